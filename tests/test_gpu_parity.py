"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Tolerances (relative Frobenius errors of X = G^-1 and W, absolute sum-rate gaps):
  * complex128 path: FP64 on both sides, every branch and rank identical, X and W within
    1e-10, sum-rate within 1e-9 bit/s/Hz.
  * complex64, tensor-core engine: the Gram matrix uses the hi/lo TF32 split (FP32-faithful,
    same X tolerance); the precoder product H^H X takes TF32 inputs (unit roundoff 2^-11 per
    operand, FP32 accumulation).  W's tolerance (tf32_w_tol) is then computed per snapshot from
    the data: the FP64 product of the GPU's own X, W_x, differs from the oracle's W by the
    X error alone (computed exactly); the GPU's W differs from W_x by the TF32 rounding of the
    operands, which the exact rounding of H and s X gives (three times it, for the operands
    whose rounding differs with the GPU's s), plus FP32 accumulation.  (test_gpu_lowprec_products
    pins the product itself to the rounded operands.)  The blocked engine's complex64 products
    are the same on tensor cores.  The SINR and sum-rate come from G and X, not from W, and
    keep the FP32 tolerance.
  * complex64 path: FP32 arithmetic.  The Gram matrix is accumulated in FP32 (u = 6e-8), so
    dG = G_t - G_{t-1} (about 5e-5 of ||G|| per 10 ms step on these channels) carries a
    relative error of a few 1e-3; through the Woodbury chain and the periodic re-inversion X
    and W stay within 1e-4, sum-rate within 1e-3 bit/s/Hz.  The rank decided by eq. 14 may
    differ by one only where the oracle's cumulative energy lies within 1e-3 of the target.
  * Method gap: WB-arSVD vs the exact-SVD oracle within 0.05 bit/s/Hz at every step.
"""
import numpy as np
import pytest
import torch

from gpu_harness import energy_tie, relerr, run_gpu, run_oracle
from oracle import method as om
from oracle import rzf
from paper_2512_16543_gb300 import binding, channel

pytestmark = pytest.mark.gpu


def _traj(sc, B, T, seed, t0=0):
    p = channel.draw_trajectories(sc, B, seed)
    return channel.trajectory(p, T, t0=t0, dtype=torch.complex128)


def tf32_round(x: np.ndarray) -> np.ndarray:
    """FP32 -> TF32 as the kernels convert (cvt.rna: nearest, ties away from zero)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def bf16_round(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 as the kernels convert (nearest, ties to even)."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def tf32_w_tol(H, X_gpu, W_ref, p_t, rnd=tf32_round, x_tol=0.0) -> float:
    """Relative Frobenius tolerance of the GPU's W = s H^H X from low-precision operands
    (rounded by `rnd`: TF32 or BF16) against the oracle's W_ref (H: the complex64 channel as
    complex128; X_gpu: the GPU's X): ||W_x - W_ref|| / ||W_ref|| with W_x the FP64 product of
    X_gpu (the X error), plus three times the error of the product of rounded H and s X_gpu
    (the operand rounding), plus twice the FP32 accumulation error 2^-24 sqrt(2K), each of the
    last two times the cancellation factor || |H^H| |X| || / ||H^H X|| where it applies.
    Callers without the GPU's X pass the oracle's and x_tol, the X tolerance, which then
    enters times the cancellation factor."""
    X = X_gpu.astype(np.complex128)
    P = H.conj().T @ X
    s = np.sqrt(p_t) / np.linalg.norm(P)
    W_x = s * P
    x_part = np.linalg.norm(W_x - W_ref) / np.linalg.norm(W_ref)
    H32, SX = H.astype(np.complex64), (s * X).astype(np.complex64)
    Hr = (rnd(H32.real) + 1j * rnd(H32.imag)).astype(np.complex128)
    Sr = (rnd(SX.real) + 1j * rnd(SX.imag)).astype(np.complex128)
    e_round = np.linalg.norm(Hr.conj().T @ Sr - W_x) / np.linalg.norm(W_x)
    cancel = np.linalg.norm(np.abs(H).T @ np.abs(X)) / np.linalg.norm(P)
    return (3 * e_round + x_part + cancel * x_tol +
            2 * 2.0 ** -24 * np.sqrt(2 * H.shape[0]) * cancel)


def _check(gpu, Hs, sc, rule, prec, *, ids=None, r_tie_tol=1e-3, x_tol=None, w_tol=None,
           rate_tol=None, alpha=None, sigma2=None, method="wb", engine="simt"):
    T, B = Hs.shape[:2]
    x_tol = x_tol or (1e-10 if prec == "c128" else 1e-4)
    tf32_w = prec == "c64" and engine in ("tensor", "blocked")   # W from TF32 inputs
    w_tol_given = w_tol is not None
    w_tol = w_tol or (1e-10 if prec == "c128" else (2e-3 if tf32_w else 1e-4))
    rate_tol = rate_tol or (1e-9 if prec == "c128" else 1e-3)
    alpha = sc.alpha if alpha is None else alpha
    sigma2 = sc.sigma2 if sigma2 is None else sigma2
    mism = 0
    for b in range(B):
        inst = b if ids is None else ids[b]
        Hb = Hs[:, b].numpy()
        if prec == "c64":
            Hb = Hb.astype(np.complex64).astype(np.complex128)   # the values the GPU sees
        ref = run_oracle(Hb, alpha, sigma2, sc.p_t, rule, instance=inst, method=method)
        for t in range(T):
            g = gpu[t]
            inf = g["info"][b]
            assert inf["status"] == 0, (t, b, inf)
            if inf["branch"] != ref[t].branch or inf["r"] != ref[t].r:
                tie = energy_tie(ref[t], r_tie_tol, rule.eta, inf["r"])
                assert prec == "c64" and tie, (t, b, inf, ref[t].branch, ref[t].r)
                mism += 1
            if "X" in g:
                assert relerr(g["X"][b], ref[t].X) < x_tol, (t, b, relerr(g["X"][b], ref[t].X))
            if tf32_w and not w_tol_given:
                wt = tf32_w_tol(Hb[t], g["X"][b] if "X" in g else ref[t].X, ref[t].W, sc.p_t)
            else:
                wt = w_tol
            assert relerr(g["W"][b], ref[t].W) < wt, (t, b, relerr(g["W"][b], ref[t].W), wt)
            assert abs(g["rate"][b] - ref[t].sum_rate) < rate_tol, (t, b, g["rate"][b],
                                                                    ref[t].sum_rate)
            np.testing.assert_allclose(g["sinr"][b], ref[t].sinr, rtol=max(1e-5, rate_tol))
    return mism


def test_single_trajectory_complex128_full_length():
    """8x8 UPA, K = 8, 100 snapshots at 10 ms, re-inverse every 20, p = 1, k_init = 2."""
    sc = channel.scenario_single_small()
    Hs = _traj(sc, 1, 100, seed=101)
    rule = binding.RankRule(eta=0.9, k_init=2, p=1, reinverse_period=20, seed=11)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c128")
    assert _check(gpu, Hs, sc, rule, "c128") == 0
    assert meta["launches"] == 100
    branches = [g["info"][0]["branch"] for g in gpu]
    assert branches[0] == 2 and branches[20] == 3 and branches.count(1) >= 90
    # method gap against the exact truncated SVD (the paper's intent, eq. 14)
    ex = run_oracle(Hs[:, 0].numpy(), sc.alpha, sc.sigma2, sc.p_t, rule, lowrank_mode="exact")
    assert max(abs(g["rate"][0] - e.sum_rate) for g, e in zip(gpu, ex)) <= 0.05
    # and against conventional full-inversion RZF
    full = run_oracle(Hs[:, 0].numpy(), sc.alpha, sc.sigma2, sc.p_t, rule, method="full")
    assert max(abs(g["rate"][0] - f.sum_rate) for g, f in zip(gpu, full)) <= 0.05


@pytest.mark.parametrize("eta", [0.65, 0.9, 0.99])
def test_lowrank_factors_match_oracle(eta):
    """The arSVD product L R^H = U_r Sigma_r V_r^H and sigma_hat^2 of every Woodbury step."""
    sc = channel.scenario_single_small()
    Hs = _traj(sc, 2, 15, seed=202)
    rule = binding.RankRule(eta=eta, k_init=2, p=1, reinverse_period=0, seed=3)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c128", trace=True)
    nwb = 0
    for b in range(2):
        ref = run_oracle(Hs[:, b].numpy(), sc.alpha, sc.sigma2, sc.p_t, rule, instance=b)
        for t in range(1, 15):
            inf = gpu[t]["info"][b]
            assert inf["branch"] == ref[t].branch and inf["r"] == ref[t].r
            r = inf["r"]
            sig = gpu[t]["sig"][b][:inf["d"]]
            np.testing.assert_allclose(sig, np.asarray(ref[t].sigma_hat) ** 2,
                                       rtol=1e-9, atol=1e-12 * sig[0])
            if inf["branch"] == 1:
                nwb += 1
                prod = gpu[t]["L"][b][:, :r] @ gpu[t]["Rh"][b][:r]
                assert relerr(prod, ref[t].lowrank_product) < 1e-9
    assert nwb > 10


@pytest.mark.parametrize("engine", ["simt", "tensor"])
def test_batched_shapes_complex64(engine):
    """16x16 UPA, K = 32, p = 8, r <= 16: FP32 path against the oracle, on both engines."""
    sc = channel.scenario_batched_256x32()
    Hs = _traj(sc, 3, 30, seed=303)
    rule = binding.RankRule(eta=0.9, k_init=2, p=8, r_max=16, reinverse_period=20, seed=5)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64", engine=engine)
    assert meta["engine"] == engine
    mism = _check(gpu, Hs, sc, rule, "c64", engine=engine)
    assert mism <= 3


def test_engines_agree():
    """The tensor-core and FMA kernels agree on the same snapshots: branches and ranks, X to
    the FP32 level, W to the TF32 level."""
    sc = channel.scenario_batched_256x32()
    Hs = _traj(sc, 4, 25, seed=313)
    rule = binding.RankRule(eta=0.8, k_init=2, p=8, r_max=16, reinverse_period=20, seed=6)
    g1, m1 = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, engine="simt")
    g2, m2 = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, engine="tensor")
    assert m1["engine"] == "simt" and m2["engine"] == "tensor"
    same = 0
    for a, b in zip(g1, g2):
        for i in range(4):
            same += a["info"][i]["r"] == b["info"][i]["r"]
            assert relerr(b["X"][i], a["X"][i]) < 1e-4
            assert relerr(b["W"][i], a["W"][i]) < 2e-3
            assert abs(a["rate"][i] - b["rate"][i]) < 1e-3
    assert same >= 0.95 * 25 * 4


@pytest.mark.parametrize("K,N", [(1, 5), (3, 1), (5, 37), (17, 100), (32, 33), (64, 96),
                                 (8, 1000), (2, 2), (31, 290), (32, 160)])
@pytest.mark.parametrize("prec,engine", [("c128", "simt"), ("c64", "simt"), ("c64", "tensor"),
                                         ("c128", "blocked"), ("c64", "blocked"),
                                         ("c64", "blocked_fma")])
def test_edge_shapes(K, N, prec, engine):
    """Ragged N (not a multiple of the 32-column staging chunk or of the 128-antenna tile),
    K > N, K = 1, K = 64; the tensor engine needs K <= 32 and even N and must refuse others;
    the blocked engine takes every shape."""
    sc = channel.LeoScenario(n_x=N, n_y=1, K=K, disc_radius=50e3)
    Hs = _traj(sc, 2, 6, seed=400 + K + N)
    rule = binding.RankRule(eta=0.9, k_init=2, p=2, r_max=min(K, 16), reinverse_period=4,
                            seed=1)
    if K == 64 and prec == "c128" and engine == "simt":
        # three resident 64 x 64 complex128 matrices plus workspaces exceed one CTA's
        # shared memory: the one-CTA kernel must refuse the shape instead of running it
        with pytest.raises(binding.WbrzfError) as e:
            run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision=prec, engine=engine)
        assert e.value.code == 6
        return
    if engine == "tensor" and (K > 32 or N % 2):
        with pytest.raises(binding.WbrzfError) as e:
            run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision=prec, engine=engine)
        assert e.value.code == 6
        return
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision=prec, engine=engine)
    assert meta["engine"] == engine
    _check(gpu, Hs, sc, rule, prec, engine=engine)


def test_keep_branch_on_unchanged_channel():
    sc = channel.scenario_single_small()
    Hs = _traj(sc, 1, 3, seed=5)
    Hs[2] = Hs[1]
    rule = binding.RankRule(eta=0.9, reinverse_period=0, seed=2)
    gpu, _ = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c128")
    assert gpu[2]["info"][0]["branch"] == 0 and gpu[2]["info"][0]["r"] == 0
    np.testing.assert_array_equal(gpu[2]["X"], gpu[1]["X"])


def test_woodbury_exact_for_exact_low_rank_change():
    """Only user 3's channel changes: rank(dG) <= 2, eta ~ 1, so X_t = G_t^-1 (eq. 12 exact)."""
    rng = np.random.default_rng(9)
    K, N = 6, 24
    H0 = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))) / np.sqrt(2 * N)
    H1 = H0.copy()
    H1[3] += 0.05 * (rng.standard_normal(N) + 1j * rng.standard_normal(N)) / np.sqrt(N)
    Hs = torch.from_numpy(np.stack([H0, H1])[:, None])
    rule = binding.RankRule(eta=1.0 - 1e-12, k_init=2, p=2, reinverse_period=0, seed=4)
    gpu, _ = run_gpu(Hs, 0.5, 0.1, 1.0, rule, precision="c128")
    inf = gpu[1]["info"][0]
    assert inf["branch"] == 1 and inf["r"] == 2
    A1 = rzf.gram(H1, 0.5)
    assert np.max(np.abs(gpu[1]["X"][0] @ A1 - np.eye(K))) < 1e-10


def test_full_inversion_method_matches_oracle():
    sc = channel.scenario_batched_256x32()
    Hs = _traj(sc, 2, 4, seed=6)
    rule = binding.RankRule()
    for engine in ("simt", "tensor"):
        gpu, _ = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64", method="full",
                         keep_state=False, engine=engine)
        for t in range(4):
            for b in range(2):
                assert gpu[t]["info"][b]["branch"] == 5
        _check(gpu, Hs, sc, rule, "c64", method="full", engine=engine)


def test_rank_switch_forces_direct_inverse():
    sc = channel.scenario_single_small()
    Hs = _traj(sc, 1, 5, seed=8)
    rule = binding.RankRule(eta=0.9, switch_ratio=0.0, reinverse_period=0, seed=1)
    gpu, _ = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c128")
    for t in range(1, 5):
        assert gpu[t]["info"][0]["branch"] == 4
        A = rzf.gram(Hs[t, 0].numpy(), sc.alpha)
        assert np.max(np.abs(gpu[t]["X"][0] @ A - np.eye(sc.K))) < 1e-11


@pytest.mark.parametrize("engine", ["simt", "tensor"])
def test_batch_invariance_with_instance_ids(engine):
    """An instance gives the same bits alone and inside a batch (same identity)."""
    sc = channel.scenario_batched_256x32()
    Hs = _traj(sc, 5, 6, seed=12).to(torch.complex64)
    rule = binding.RankRule(eta=0.8, k_init=2, p=8, r_max=16, seed=9)
    ids = [40, 41, 42, 43, 44]
    batch, _ = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, ids=ids, engine=engine)
    alone, _ = run_gpu(Hs[:, 3:4].contiguous(), sc.alpha, sc.sigma2, sc.p_t, rule, ids=[43],
                       engine=engine)
    for t in range(6):
        np.testing.assert_array_equal(batch[t]["W"][3], alone[t]["W"][0])
        np.testing.assert_array_equal(batch[t]["X"][3], alone[t]["X"][0])


def test_not_positive_definite_is_reported():
    """alpha = 0 and a user with an all-zero channel: G is singular, the direct inverse meets
    a zero pivot and the instance reports WBRZF_STATUS_NOT_PD."""
    K, N = 4, 8
    H = np.ones((K, N), dtype=np.complex128) * 0.1
    H[1] = 0.0
    Hs = torch.from_numpy(H[None, None].copy())
    h = binding.WBRZF(1, N, K, [0.0], [0.1], precision="c128")
    h.full_inverse(Hs[0].cuda())
    info = h.step_info()
    assert info[0]["status"] & 1
    with pytest.raises(binding.WbrzfError):
        h.step_info(raise_on_numerical=True)
    h.close()


def test_update_before_full_inverse_is_rejected():
    h = binding.WBRZF(1, 16, 4, [0.4], [0.1], precision="c64")
    H = torch.zeros(1, 4, 16, dtype=torch.complex64, device="cuda")
    with pytest.raises(binding.WbrzfError) as e:
        h.update(H)
    assert e.value.code == 2
    h.close()


def test_full_size_batched_sampled_parity():
    """1024 trajectories of 16x16 UPA, K = 32, in the launch configuration the bench times;
    four sampled instances are recomputed by the oracle."""
    sc = channel.scenario_batched_256x32()
    B, T = 1024, 25
    params = channel.draw_trajectories(sc, B, seed=2512)
    rule = binding.RankRule(eta=0.9, k_init=2, p=8, r_max=16, reinverse_period=20, seed=77)
    h = binding.WBRZF(B, sc.N, sc.K, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule)
    sample = [0, 333, 700, 1023]
    Hs_s, Ws_s, rates_s = [], [], []
    for t in range(T):
        H = channel.channel_at(params, t, device="cuda", dtype=torch.complex64)
        W = h.full_inverse(H) if t == 0 else h.update(H)
        _, rate = h.sum_rate()
        Hs_s.append(H[sample].cpu())
        Ws_s.append(W[sample].cpu().numpy())
        rates_s.append(rate[sample].cpu().numpy())
    info = h.step_info()
    assert all(i["status"] == 0 for i in info)
    assert h.last_engine == "tensor"
    h.close()
    Hs = torch.stack(Hs_s)
    for j, b in enumerate(sample):
        ref = run_oracle(Hs[:, j].numpy().astype(np.complex128), sc.alpha, sc.sigma2, sc.p_t,
                         rule, instance=b)
        for t in range(T):
            assert relerr(Ws_s[t][j], ref[t].W) < 2e-3
            assert abs(rates_s[t][j] - ref[t].sum_rate) < 1e-3


def test_full_size_batched_full_length_at_bench_eta():
    """The batched configuration over its full 500 snapshots (5 s of orbit, 25 periodic
    re-inversions) at the bench's eta = 0.65, in the launch configuration the bench times:
    sampled instances recomputed by the oracle stay within the complex64 tolerances at every
    snapshot, so the Woodbury updates between re-inversions do not drift."""
    sc = channel.scenario_batched_256x32()
    B, T = 1024, 500
    params = channel.draw_trajectories(sc, B, seed=2512)
    rule = binding.RankRule(eta=0.65, k_init=2, p=8, r_max=16, reinverse_period=20, seed=77)
    h = binding.WBRZF(B, sc.N, sc.K, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule)
    sample = [5, 511, 1000]
    Hs_s, Ws_s, rates_s, branches = [], [], [], []
    for t in range(T):
        H = channel.channel_at(params, t, device="cuda", dtype=torch.complex64)
        W = h.full_inverse(H) if t == 0 else h.update(H)
        _, rate = h.sum_rate()
        Hs_s.append(H[sample].cpu())
        Ws_s.append(W[sample].cpu().numpy())
        rates_s.append(rate[sample].cpu().numpy())
        if t % 50 == 49:
            info = h.step_info()
            assert all(i["status"] == 0 for i in info), t
            branches.append({i["branch"] for i in info})
    assert h.last_engine == "tensor"
    h.close()
    assert any(1 in b for b in branches)            # Woodbury updates were taken
    Hs = torch.stack(Hs_s)
    for j, b in enumerate(sample):
        ref = run_oracle(Hs[:, j].numpy().astype(np.complex128), sc.alpha, sc.sigma2, sc.p_t,
                         rule, instance=b)
        assert sum(r.branch == 1 for r in ref) > T // 2
        for t in range(T):
            assert relerr(Ws_s[t][j], ref[t].W) < 2e-3, (t, b)
            assert abs(rates_s[t][j] - ref[t].sum_rate) < 1e-3, (t, b)


@pytest.mark.parametrize("prec,engine,tol", [("c128", "simt", 1e-9), ("c128", "blocked", 1e-9),
                                             ("c64", "tensor", 1e-3), ("c64", "blocked", 1e-3)])
def test_sum_rate_in_fp64(prec, engine, tol):
    """The per-instance sum-rate summed in FP64 (wbrzf_sum_rate_f64): within the engine's
    sum-rate tolerance of the oracle, equal to the FP32 report after rounding, and in complex128
    beyond FP32's resolution of it (the FP32 copy is off by up to half an ulp, 2^-24 R)."""
    sc = channel.LeoScenario(n_x=16, n_y=8, K=16, disc_radius=50e3)
    Hs = _traj(sc, 3, 4, seed=64)
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=8, reinverse_period=3, seed=6)
    dt = torch.complex64 if prec == "c64" else torch.complex128
    h = binding.WBRZF(3, sc.N, sc.K, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule,
                      precision=prec, workspace_for="blocked")
    h.set_engine(engine)
    refs = [run_oracle(Hs[:, b].numpy().astype(np.complex64).astype(np.complex128)
                       if prec == "c64" else Hs[:, b].numpy(), sc.alpha, sc.sigma2, sc.p_t,
                       rule, instance=b) for b in range(3)]
    for t in range(4):
        H = Hs[t].to(device="cuda", dtype=dt).contiguous()
        h.full_inverse(H) if t == 0 else h.update(H)
        r64 = h.sum_rate64().cpu().numpy()
        r32 = h.sum_rate()[1].cpu().numpy()
        assert r64.dtype == np.float64
        np.testing.assert_array_equal(r64.astype(np.float32), r32)
        for b in range(3):
            assert abs(r64[b] - refs[b][t].sum_rate) < tol, (t, b, r64[b], refs[b][t].sum_rate)
            if prec == "c128":
                assert abs(r64[b] - refs[b][t].sum_rate) < 2.0 ** -30 * refs[b][t].sum_rate
    h.close()


@pytest.mark.parametrize("engine,shortcut", [("tensor", False), ("tensor", True),
                                             ("simt", True)])
def test_energy_shortcut_keeps_parity(engine, shortcut):
    """A wide disc and eta = 0.9 at K = 32 make Algorithm 1 iterate (d = 10 .. 24): with the
    energy test taken without the eigensolver (tensor kernel's launch choice; always in the
    FMA kernel) or with the full test, the branches, ranks and results meet the oracle."""
    sc = channel.LeoScenario(n_x=16, n_y=16, K=32, disc_radius=200e3)
    Hs = _traj(sc, 3, 5, seed=320)
    rule = binding.RankRule(eta=0.9, k_init=2, p=8, r_max=32, reinverse_period=0, seed=7)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64", engine=engine,
                        energy_shortcut=shortcut)
    assert meta["engine"] == engine
    assert _check(gpu, Hs, sc, rule, "c64", engine=engine) <= 2
    assert max(g["info"][b]["iters"] for g in gpu[1:] for b in range(3)) >= 3
    assert any(g["info"][b]["branch"] == 1 for g in gpu[1:] for b in range(3))
