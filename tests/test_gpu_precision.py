"""Precision modes of the blocked engine: BF16 precoder product, one Newton refinement of X.

BF16 operands carry a unit roundoff of 2^-9, four times TF32's.  W is held, snapshot by
snapshot, to the tolerance computed from the data as for TF32 (tf32_w_tol with BF16
rounding: the X error, three times the exact error of the rounded operands' product, FP32
accumulation), and to 8e-3 overall (the largest error measured against FP64 on the uneven
workload is 7.5e-3).  X is untouched by that mode (its Gram matrix stays FP32-faithful) and
keeps 1e-4.  The Newton
step X <- X (2 I - G X) squares the residual I - G X: with it the residual stays at the square
of one snapshot's truncation residual (about (5e-5)^2 in FP64 at eta = 0.65) or at FP32
rounding (1e-4 entrywise at K = 32), while without it the truncation error accumulates from
snapshot to snapshot.
"""
import numpy as np
import pytest
import torch

from gpu_harness import relerr, run_gpu, run_oracle
from oracle import rzf
from paper_2512_16543_gb300 import binding, channel
from test_gpu_parity import _traj, bf16_round, tf32_w_tol

pytestmark = pytest.mark.gpu


def _run(Hs, sc, rule, prec, engine, bf16=False, refine=0):
    T, B, K, N = Hs.shape
    dt = torch.complex64 if prec == "c64" else torch.complex128
    h = binding.WBRZF(B, N, K, sc.alpha, sc.sigma2, rule=rule, precision=prec,
                      workspace_for="blocked")
    h.set_engine(engine)
    h.set_precision_mode(bf16, refine)
    out = []
    for t in range(T):
        H = Hs[t].to(device="cuda", dtype=dt).contiguous()
        W = h.full_inverse(H) if t == 0 else h.update(H)
        G, X = h.state()
        out.append((W.cpu().numpy(), G.cpu().numpy(), X.cpu().numpy(), h.step_info()))
    h.close()
    return out


def test_bf16_precoder_product_against_the_oracle():
    sc = channel.LeoScenario(n_x=16, n_y=8, K=48, disc_radius=80e3)
    Hs = _traj(sc, 2, 8, seed=81)
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=16, reinverse_period=4, seed=3)
    gpu = _run(Hs, sc, rule, "c64", "blocked", bf16=True)
    for b in range(2):
        Hb = Hs[:, b].numpy().astype(np.complex64).astype(np.complex128)
        ref = run_oracle(Hb, sc.alpha, sc.sigma2, sc.p_t, rule, instance=b)
        for t in range(8):
            W, _, X, info = gpu[t]
            assert relerr(X[b], ref[t].X) < 1e-4
            tol = min(8e-3, tf32_w_tol(Hb[t], X[b], ref[t].W, sc.p_t, rnd=bf16_round))
            e = relerr(W[b], ref[t].W)
            assert e < tol, (t, b, e, tol)
            assert e > 1e-5            # the BF16 product is really in use
    # the TF32 product of the same engine is several times closer
    gpu32 = _run(Hs, sc, rule, "c64", "blocked")
    ref = run_oracle(Hs[:, 0].numpy().astype(np.complex64).astype(np.complex128), sc.alpha,
                     sc.sigma2, sc.p_t, rule, instance=0)
    assert relerr(gpu32[5][0][0], ref[5].W) < relerr(gpu[5][0][0], ref[5].W)


@pytest.mark.parametrize("prec,engine,tol", [("c64", "blocked", 1e-4),
                                             ("c128", "blocked_fma", 1e-7)])
def test_refinement_keeps_x_at_the_inverse(prec, engine, tol):
    sc = channel.scenario_batched_256x32()
    Hs = _traj(sc, 2, 14, seed=82)
    # eta = 0.65 and no periodic re-inversion: the truncation error accumulates in X
    rule = binding.RankRule(eta=0.65, k_init=2, p=8, r_max=16, reinverse_period=0, seed=4)
    plain = _run(Hs, sc, rule, prec, engine)
    refined = _run(Hs, sc, rule, prec, engine, refine=1)
    I = np.eye(sc.K)
    drift, resid = [], []
    for t in range(1, 14):
        for b in range(2):
            G = rzf.gram(Hs[t, b].numpy().astype(np.complex64 if prec == "c64" else
                                                 np.complex128).astype(np.complex128),
                         sc.alpha)
            Xr = refined[t][2][b].astype(np.complex128)
            Xp = plain[t][2][b].astype(np.complex128)
            resid.append(np.abs(Xr @ G - I).max())
            assert resid[-1] < tol, (t, b)
            drift.append(np.abs(Xp @ G - I).max())
            assert refined[t][3][b]["branch"] == plain[t][3][b]["branch"]
    assert max(drift) > 10 * max(resid)    # without the step the iterate leaves the inverse


def test_precision_mode_needs_the_blocked_engine():
    h = binding.WBRZF(2, 64, 8, 0.8, 0.1, precision="c64")
    h.set_precision_mode(False, 1)
    H = torch.zeros(2, 8, 64, dtype=torch.complex64, device="cuda")
    with pytest.raises(binding.WbrzfError) as e:
        h.full_inverse(H)
    assert e.value.code == 6
    h.close()
    h = binding.WBRZF(1, 64, 8, 0.8, 0.1, precision="c128", workspace_for="blocked")
    with pytest.raises(binding.WbrzfError) as e:
        h.set_precision_mode(True, 0)                  # BF16 products are complex64 only
    assert e.value.code == 6
    h.close()
