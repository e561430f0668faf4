"""Parity of the blocked engine (each step of the path a batched kernel of its own, any K) with
the FP64 oracle, through the C ABI.

Tolerances are those of the one-CTA engines (the arithmetic is the same, only the blocking and
the order of the sums differ): complex128 X and W within 1e-10, sum-rate within 1e-9; complex64
X within 1e-4 and sum-rate within 1e-3 bit/s/Hz (K <= 128); complex64 W within 1e-4 on
"blocked_fma" (FP32 FMA) and 2e-3 on "blocked", whose precoder product takes TF32 inputs (unit
roundoff 2^-11 per operand) while its Gram matrix keeps FP32 accuracy through the hi/lo split.  For the large array
(N = 4096, K = 512) the FP32 Gram matrix is a sum of 4096 products per entry: its rounding
error (about sqrt(N) u |G_ij|, 4e-6 per entry) is a sizeable fraction of dG (1.6e-5 of ||G||
per 10 ms step), so the rank of eq. 14 on that nearly flat spectrum may move by a few
components; X then moves by at most the dropped components' share of dG, far below the 1e-4
bound on X that still holds; the sum-rate keeps the 1e-3 bit/s/Hz bound.
"""
import numpy as np
import pytest
import torch

import types

from gpu_harness import energy_tie, oracle_rule, relerr, run_gpu, run_oracle
from oracle import lowrank, philox, rzf
from paper_2512_16543_gb300 import binding, channel
from test_gpu_parity import _check, _traj

pytestmark = pytest.mark.gpu


def test_blocked_complex128_single_trajectory():
    """8x8 UPA, K = 8: every branch (init, Woodbury, periodic re-inverse) against the oracle."""
    sc = channel.scenario_single_small()
    Hs = _traj(sc, 2, 45, seed=101)
    rule = binding.RankRule(eta=0.9, k_init=2, p=1, reinverse_period=20, seed=11)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c128",
                        engine="blocked")
    assert meta["engine"] == "blocked"
    assert meta["launches"] > 45                 # several kernels per snapshot
    _check(gpu, Hs, sc, rule, "c128", engine="blocked")
    branches = {g["info"][b]["branch"] for g in gpu for b in range(2)}
    assert {1, 2, 3} <= branches


@pytest.mark.parametrize("eta", [0.65, 0.99])
def test_blocked_lowrank_factors_match_oracle(eta):
    sc = channel.scenario_single_small()
    Hs = _traj(sc, 2, 12, seed=202)
    rule = binding.RankRule(eta=eta, k_init=2, p=1, reinverse_period=0, seed=3)
    gpu, _ = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c128", trace=True,
                     engine="blocked")
    nwb = 0
    for b in range(2):
        ref = run_oracle(Hs[:, b].numpy(), sc.alpha, sc.sigma2, sc.p_t, rule, instance=b)
        for t in range(1, 12):
            inf = gpu[t]["info"][b]
            assert inf["branch"] == ref[t].branch and inf["r"] == ref[t].r
            sig = gpu[t]["sig"][b][:inf["d"]]
            np.testing.assert_allclose(sig, np.asarray(ref[t].sigma_hat) ** 2,
                                       rtol=1e-9, atol=1e-12 * sig[0])
            if inf["branch"] == 1:
                nwb += 1
                r = inf["r"]
                prod = gpu[t]["L"][b][:, :r] @ gpu[t]["Rh"][b][:r]
                assert relerr(prod, ref[t].lowrank_product) < 1e-9
    assert nwb > 5


@pytest.mark.parametrize("engine", ["blocked", "blocked_fma"])
def test_blocked_complex64_batched(engine):
    """16x16 UPA, K = 32, p = 8, r <= 16 on the blocked engine against the oracle."""
    sc = channel.scenario_batched_256x32()
    Hs = _traj(sc, 3, 25, seed=303)
    rule = binding.RankRule(eta=0.9, k_init=2, p=8, r_max=16, reinverse_period=20, seed=5)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64", engine=engine)
    assert meta["engine"] == engine
    assert _check(gpu, Hs, sc, rule, "c64", engine=engine) <= 3


def test_blocked_agrees_with_fma_engine():
    """Same snapshots on the one-CTA FMA kernel and on the blocked engine: in FP64 the same
    branches and ranks and X to 1e-12; in FP32 X to 1e-4."""
    sc = channel.LeoScenario(n_x=25, n_y=4, K=17, disc_radius=50e3)
    Hs = _traj(sc, 3, 12, seed=77)
    rule = binding.RankRule(eta=0.85, k_init=2, p=3, r_max=8, reinverse_period=5, seed=8)
    for prec, tol in (("c128", 1e-12), ("c64", 1e-4)):
        a, _ = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision=prec, engine="simt")
        b, _ = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision=prec,
                       engine="blocked_fma")
        for ga, gb in zip(a, b):
            for i in range(3):
                if prec == "c128":
                    assert ga["info"][i]["branch"] == gb["info"][i]["branch"]
                    assert ga["info"][i]["r"] == gb["info"][i]["r"]
                assert relerr(gb["X"][i], ga["X"][i]) < tol
                assert relerr(gb["W"][i], ga["W"][i]) < tol


@pytest.mark.parametrize("K,N,prec,engine", [(100, 300, "c128", "auto"),
                                             (128, 512, "c64", "auto"),
                                             (128, 512, "c64", "blocked_fma"),
                                             (65, 97, "c64", "auto"), (64, 96, "c128", "auto"),
                                             (200, 250, "c64", "auto")])
def test_blocked_beyond_one_cta(K, N, prec, engine):
    """K above the one-CTA limit (and K = 64 in complex128, whose one-CTA footprint exceeds
    shared memory): the automatic choice is the blocked engine; ragged last pivot block
    (K not a multiple of 32) and ragged N."""
    sc = channel.LeoScenario(n_x=N, n_y=1, K=K, disc_radius=100e3)
    Hs = _traj(sc, 2, 6, seed=500 + K)
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=32, reinverse_period=4, seed=2)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision=prec, engine=engine)
    assert meta["engine"] == ("blocked" if engine == "auto" else engine)
    _check(gpu, Hs, sc, rule, prec, engine=meta["engine"])


def test_blocked_uneven_class_1024x128():
    """The largest class of the uneven population (32x32 UPA, N = 1024, K = 128) with the
    bench's rule (p = 8, k_init = 2, r_max = 64, eta = 0.65, re-inverse every 20), through the
    fused Algorithm 1 path of the blocked engine, against the oracle: two instances over ten
    snapshots, Woodbury updates included."""
    sc = channel.LeoScenario(n_x=32, n_y=32, K=128, disc_radius=50e3)
    Hs = _traj(sc, 2, 10, seed=1024)
    rule = binding.RankRule(eta=0.65, k_init=2, p=8, r_max=64, reinverse_period=20, seed=77)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64")
    assert meta["engine"] == "blocked"
    assert _check(gpu, Hs, sc, rule, "c64", engine="blocked") <= 2
    assert sum(g["info"][b]["branch"] == 1 for g in gpu for b in range(2)) >= 12


def test_blocked_full_inversion_method():
    sc = channel.LeoScenario(n_x=50, n_y=4, K=96, disc_radius=100e3)
    Hs = _traj(sc, 2, 3, seed=9)
    rule = binding.RankRule()
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64", method="full",
                        keep_state=False, engine="blocked")
    assert meta["engine"] == "blocked"
    assert all(g["info"][b]["branch"] == 5 for g in gpu for b in range(2))
    _check(gpu, Hs, sc, rule, "c64", method="full", engine="blocked")


def test_blocked_batch_invariance_with_instance_ids():
    sc = channel.scenario_batched_256x32()
    Hs = _traj(sc, 4, 5, seed=12).to(torch.complex64)
    rule = binding.RankRule(eta=0.8, k_init=2, p=8, r_max=16, seed=9)
    ids = [70, 71, 72, 73]
    batch, _ = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, ids=ids, engine="blocked")
    alone, _ = run_gpu(Hs[:, 2:3].contiguous(), sc.alpha, sc.sigma2, sc.p_t, rule, ids=[72],
                       engine="blocked")
    for t in range(5):
        np.testing.assert_array_equal(batch[t]["W"][2], alone[t]["W"][0])
        np.testing.assert_array_equal(batch[t]["X"][2], alone[t]["X"][0])


def test_blocked_not_positive_definite_is_reported():
    K, N = 70, 80
    H = np.ones((K, N), dtype=np.complex128) * 0.1
    H[5] = 0.0
    h = binding.WBRZF(1, N, K, [0.0], [0.1], precision="c128")
    h.full_inverse(torch.from_numpy(H[None].copy()).cuda())
    assert h.last_engine == "blocked"
    assert h.step_info()[0]["status"] & 1
    h.close()


def test_large_array_against_oracle():
    """64x64 UPA (N = 4096), K = 512, adaptive rank up to 64, complex64: one instance, the
    initial inverse and three updates against the oracle.  dG's spectrum is nearly flat here
    (the leading 64 of 512 singular values hold about half its energy) and a sketch of
    d = 72 columns captures about a third of it, so eta = 0.25 is met at a rank in the 40s
    and the updates take the Woodbury branch, while at eta = 0.9 Algorithm 1 ends unmet at
    r = d = 72 > r_max and every update is a direct inverse (branch RANK), as in the oracle.

    The rank of a Woodbury update is checked against the oracle's Algorithm 1 run on the dG
    the GPU itself formed (G_t - G_{t-1} from its complex64 states, the same Philox test
    matrices): equal, or an energy tie at 1e-3 of the target.  Against the oracle's own dG it
    may differ by a few components: the FP32 Gram matrix's rounding (about sqrt(N) u of each
    entry, 4e-6 here) is a sizeable fraction of dG (1.6e-5 of ||G|| per 10 ms step), and on a
    flat spectrum that moves the cumulative energies by about as much as a component holds."""
    sc = channel.scenario_large_4096x512()
    Hs = _traj(sc, 1, 4, seed=7)
    H64 = Hs[:, 0].numpy().astype(np.complex64).astype(np.complex128)
    for eta, branch in ((0.25, 1), (0.9, 4)):
        rule = binding.RankRule(eta=eta, k_init=2, p=8, r_max=64, reinverse_period=20, seed=5)
        gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64")
        assert meta["engine"] == "blocked"
        ref = run_oracle(H64, sc.alpha, sc.sigma2, sc.p_t, rule)
        for t in range(4):
            inf = gpu[t]["info"][0]
            assert inf["status"] == 0
            assert inf["branch"] == ref[t].branch == (2 if t == 0 else branch)
            if branch == 1 and t > 0:
                dG = gpu[t]["G"][0].astype(np.complex128) - gpu[t - 1]["G"][0].astype(np.complex128)
                rr = oracle_rule(rule).resolved(sc.K)
                lr = lowrank.arsvd(dG, rr.eta, rr.k_init, rr.p, rr.i_max,
                                   lambda it, d, t=t: philox.omega(sc.K, d, seed=rr.seed, step=t,
                                                                   instance=0, it=it))
                own = types.SimpleNamespace(sigma_hat=lr.sigma_hat, r=lr.k_est,
                                            dA_fro2=float(np.sum(np.abs(dG) ** 2)))
                assert inf["r"] == lr.k_est or energy_tie(own, 1e-3, eta, inf["r"]), (
                    inf["r"], lr.k_est, ref[t].r)
            assert relerr(gpu[t]["X"][0], ref[t].X) < 1e-4
            assert relerr(gpu[t]["W"][0], ref[t].W) < 2e-3      # TF32 precoder product
            assert abs(gpu[t]["rate"][0] - ref[t].sum_rate) < 1e-3
        if branch == 4:                           # direct inverse: X G = I to FP32 level
            G = rzf.gram(H64[3], sc.alpha)
            assert np.max(np.abs(gpu[3]["X"][0] @ G - np.eye(sc.K))) < 1e-4


@pytest.mark.parametrize("K,N,eta,engine,fp64", [(64, 128, 0.9, "simt", False),
                                                 (64, 128, 0.9, "blocked", False),
                                                 (64, 128, 0.97, "blocked", False),
                                                 (65, 97, 0.95, "blocked", False),
                                                 (128, 256, 0.8, "blocked", False),
                                                 (128, 256, 0.85, "blocked", False),
                                                 (64, 128, 0.9, "blocked", True),
                                                 (65, 97, 0.95, "blocked", True)])
def test_sketch_wider_than_a_warp(K, N, eta, engine, fp64):
    """A wide user disc and a high eta drive Algorithm 1 to sketch widths d = 40, 64 and 72,
    wider than the 32 lanes of the warp that factors CholQR's Gram matrix and rotates the
    eigensolver's pairs, with Woodbury ranks 23 to 42 (above the fused Woodbury kernel's first
    cap of 24, and at K = 128 around its second cap of 40): the one-CTA FMA engine, the blocked engine's fused kernels (both launches) and
    its per-step kernels, in FP32 and with the FP64 small solves, against the oracle.  The
    one-CTA engine's shared memory holds d = 40 at K = 64 with r_max = 32."""
    sc = channel.LeoScenario(n_x=N, n_y=1, K=K, disc_radius=200e3)
    Hs = _traj(sc, 2, 4, seed=7)
    rule = binding.RankRule(eta=eta, k_init=2, p=8, r_max=32 if engine == "simt" else 48,
                            reinverse_period=0, seed=4)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64", engine=engine,
                        fp64_small=fp64)
    assert meta["engine"] == engine
    assert _check(gpu, Hs, sc, rule, "c64", engine=engine) <= 2
    infos = [g["info"][b] for g in gpu[1:] for b in range(2)]
    assert max(i["d"] for i in infos) > 32
    assert any(i["branch"] == 1 and i["r"] > (20 if engine == "simt" else 24) for i in infos)
