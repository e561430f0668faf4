"""The blocked engine's FP64 small-solve mode (complex64 handles): the eigensolver of
Algorithm 1's small SVD of B, the capacitance inverse of eq. 12 and every direct inverse of G
in FP64, the large products unchanged.

Parity with the FP64 oracle holds at the complex64 tolerances of the other blocked tests (the
FP32 / TF32 products dominate the error).  What the mode changes is pinned where it is the
whole error: a direct inverse in FP64 rounded once to complex64 is the inverse of the G the
library holds to the rounding of X (2^-24 relative per entry), whatever G's condition number,
while the FP32 block inverse's error grows with it.
"""
import numpy as np
import pytest
import torch

from gpu_harness import relerr, run_gpu
from paper_2512_16543_gb300 import binding, channel
from test_gpu_parity import _check, _traj

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("K,N,p,r_max", [(16, 64, 4, 8), (32, 256, 8, 16), (65, 97, 4, 32),
                                         (128, 512, 8, 64)])
def test_fp64_small_solves_match_the_oracle(K, N, p, r_max):
    """Every branch (init, Woodbury, periodic re-inverse; ragged K = 65) against the oracle at
    the complex64 tolerances; the rank may differ only on an energy tie."""
    sc = channel.LeoScenario(n_x=N, n_y=1, K=K, disc_radius=50e3)
    Hs = _traj(sc, 2, 9, seed=640 + K)
    rule = binding.RankRule(eta=0.8, k_init=2, p=p, r_max=r_max, reinverse_period=4, seed=9)
    gpu, meta = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64",
                        engine="blocked", fp64_small=True)
    assert meta["engine"] == "blocked"
    assert _check(gpu, Hs, sc, rule, "c64", engine="blocked") <= 2
    branches = {g["info"][b]["branch"] for g in gpu for b in range(2)}
    assert {1, 2, 3} <= branches


def _ill_conditioned(B, K, N, seed):
    """Gaussian H with N = K: the smallest singular value of a square Gaussian matrix is about
    1 / sqrt(K) of its scale, so H H^H + alpha I with a small alpha has a condition number of
    order 1e4 .. 1e5."""
    g = torch.Generator().manual_seed(seed)
    re = torch.randn(B, K, N, generator=g, dtype=torch.float64)
    im = torch.randn(B, K, N, generator=g, dtype=torch.float64)
    return torch.complex(re, im).to(torch.complex64) / np.sqrt(2 * N)


@pytest.mark.parametrize("K", [24, 64, 128])
def test_fp64_direct_inverse_is_the_rounded_inverse(K):
    B = 3
    H = _ill_conditioned(B, K, K, seed=K)
    alpha, sigma2, p_t = 1e-4, 1e-4, 1.0
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=min(16, K), reinverse_period=2,
                            seed=1)
    err = {}
    for small64 in (True, False):
        h = binding.WBRZF(B, K, K, alpha, sigma2, p_t=p_t, rule=rule, precision="c64",
                          workspace_for="blocked")
        h.set_engine("blocked")
        if small64:
            h.set_fp64_small_solves(True)
        h.full_inverse(H.cuda())
        G, X = h.state()
        G = G.cpu().numpy().astype(np.complex128)
        X = X.cpu().numpy().astype(np.complex128)
        assert all(i["status"] == 0 for i in h.step_info())
        h.close()
        conds = [np.linalg.cond(G[b]) for b in range(B)]
        err[small64] = [relerr(X[b], np.linalg.inv(G[b])) for b in range(B)]
    assert min(conds) > 1e3, conds
    # FP64 inverse rounded once: 2^-24 per entry (relative), a factor 2 for the sum of squares
    assert max(err[True]) < 2 * 2.0 ** -24, err[True]
    # the FP32 block inverse is far from it on such a G
    assert min(err[False]) > 10 * max(err[True]), (err[False], err[True])


def test_fp64_periodic_reinverse_is_the_rounded_inverse():
    """Algorithm 2's periodic re-inversion (every 2nd snapshot here) in FP64 mode: X equals the
    rounded FP64 inverse of that snapshot's G."""
    sc = channel.LeoScenario(n_x=16, n_y=4, K=32, disc_radius=50e3)
    Hs = _traj(sc, 2, 5, seed=31)
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=16, reinverse_period=2, seed=3)
    gpu, _ = run_gpu(Hs, sc.alpha, sc.sigma2, sc.p_t, rule, precision="c64", engine="blocked",
                     fp64_small=True)
    seen = 0
    for g in gpu:
        for b in range(2):
            if g["info"][b]["branch"] in (2, 3):           # init, periodic
                G = g["G"][b].astype(np.complex128)
                assert relerr(g["X"][b].astype(np.complex128), np.linalg.inv(G)) < 2 * 2.0 ** -24
                seen += 1
    assert seen >= 4


def test_fp64_small_solves_unsupported_cases():
    sc = channel.LeoScenario(n_x=8, n_y=4, K=8, disc_radius=50e3)
    rule = binding.RankRule(eta=0.9, k_init=2, p=2, reinverse_period=0, seed=1)
    h = binding.WBRZF(2, 32, 8, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule, precision="c128")
    with pytest.raises(RuntimeError):
        h.set_fp64_small_solves(True)                      # complex128: already FP64
    h.close()
    h = binding.WBRZF(2, 32, 8, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule, precision="c64",
                      workspace_for="blocked")
    h.set_engine("simt")
    h.set_fp64_small_solves(True)
    H = channel.channel_at(channel.draw_trajectories(sc, 2, seed=1), 0, device="cuda",
                           dtype=torch.complex64)
    with pytest.raises(RuntimeError):
        h.full_inverse(H)                                  # the mode runs on the blocked engine
    h.set_engine("blocked")
    h.full_inverse(H)
    h.close()
