"""The low-precision precoder product W = s H^H X of the tensor-core engines, pinned exactly.

The oracle-parity tests hold W to 2e-3 (TF32) or 8e-3 (BF16), or to a multiple of the
entrywise rounding bound where the sum over users cancels: there the GPU's W also inherits
the FP32 differences of X, so the bound has to cover operand rounding and X together.  Here
the product is isolated.  The handle is loaded (wbrzf_set_state) with the oracle's G and
X = G^-1 rounded to complex64, and updated on the same channel with dg_floor_rel = 1, so the
branch is KEEP and X is exactly the loaded one.  The reference is the product that the
tensor cores are specified to form: each operand rounded like the kernels round it --
TF32 round-to-nearest-away (cvt.rna.tf32) of H and of the FP32 product s X, or BF16
round-to-nearest-even -- with s = sqrt(P_t) / ||H^H X||_F from the oracle, multiplied and
summed in FP64.  What remains is FP32 accumulation (2K terms, about 2^-24 sqrt(2K) of
|| |H^H| |sX| ||) and the operand roundings that flip where the GPU's s (from FP32 sums)
and the oracle's s fall on either side of a rounding boundary: each flip moves one operand
by one unit in the last place (2^-10 relative for TF32, 2^-7 for BF16) on a fraction f of
about |ds / s| / 2^-11 of the entries; with |ds / s| <= 1e-6 that is f <= 2e-3, giving
sqrt(f) 2^-10 <= 5e-5 (TF32) and 4e-4 (BF16) of || |H^H| |sX| ||.  The tolerance is that,
with a factor of two, times the cancellation factor || |H^H| |X| || / ||H^H X|| (>= 1).
"""
import numpy as np
import pytest
import torch

from gpu_harness import relerr
from oracle import rzf
from paper_2512_16543_gb300 import binding, channel
from test_gpu_parity import _traj

pytestmark = pytest.mark.gpu


def tf32_rna(x: np.ndarray) -> np.ndarray:
    """FP32 -> TF32 (10 stored mantissa bits), round to nearest, ties away from zero."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)


def bf16_rne(x: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 (7 stored mantissa bits), round to nearest, ties to even."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def reference_product(H32: np.ndarray, X32: np.ndarray, p_t: float, rnd):
    """s H^H X from operands rounded by `rnd` (H's components, and the FP32 products s X)."""
    H = H32.astype(np.complex128)
    X = X32.astype(np.complex128)
    s = np.float32(np.sqrt(p_t / np.linalg.norm(H.conj().T @ X) ** 2))
    Hr = rnd(H32.real) + 1j * rnd(H32.imag)
    Sx = rnd(s * X32.real.astype(np.float32)) + 1j * rnd(s * X32.imag.astype(np.float32))
    W = Hr.astype(np.complex128).conj().T @ Sx.astype(np.complex128)
    cancel = np.linalg.norm(np.abs(H).T @ np.abs(X)) / np.linalg.norm(H.conj().T @ X)
    return W, max(1.0, float(cancel))


def _keep_step(H32, sc, engine, bf16=False):
    """Load the oracle's G and X rounded to complex64, then one KEEP update on H."""
    B, K, N = H32.shape
    Gs = np.stack([rzf.gram(H32[b].astype(np.complex128), sc.alpha) for b in range(B)])
    Xs = np.stack([np.linalg.inv(G) for G in Gs])
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=min(K, 16), reinverse_period=0,
                            dg_floor_rel=1.0, seed=1)
    h = binding.WBRZF(B, N, K, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule, precision="c64",
                      workspace_for="blocked" if engine == "blocked" else "auto")
    h.set_engine(engine)
    if bf16:
        h.set_precision_mode(True, 0)
    X32 = Xs.astype(np.complex64)
    h.restore(torch.from_numpy(Gs.astype(np.complex64)), torch.from_numpy(X32), [1] * B)
    W = h.update(torch.from_numpy(H32).cuda())
    info = h.step_info()
    assert h.last_engine == engine
    W = W.cpu().numpy()
    h.close()
    assert all(i["branch"] == 0 and i["status"] == 0 for i in info), info
    return W, X32


SHAPES = [(1, 6), (3, 2), (5, 38), (17, 100), (31, 290), (32, 160), (32, 256)]


@pytest.mark.parametrize("K,N", SHAPES + [(64, 96), (128, 512)])
@pytest.mark.parametrize("engine", ["tensor", "blocked"])
def test_tf32_precoder_product_is_the_rounded_product(K, N, engine):
    if engine == "tensor" and K > 32:
        pytest.skip("the tensor engine takes K <= 32")
    sc = channel.LeoScenario(n_x=N, n_y=1, K=K, disc_radius=50e3)
    H32 = _traj(sc, 2, 1, seed=900 + K + N)[0].numpy().astype(np.complex64)
    W, X32 = _keep_step(H32, sc, engine)
    for b in range(2):
        ref, cancel = reference_product(H32[b], X32[b], sc.p_t, tf32_rna)
        tol = 2 * (5e-5 + 2.0 ** -24 * np.sqrt(2 * K)) * cancel
        assert relerr(W[b], ref) < tol, (b, relerr(W[b], ref), tol)


@pytest.mark.parametrize("K,N", [(5, 38), (17, 100), (48, 128), (128, 512)])
def test_bf16_precoder_product_is_the_rounded_product(K, N):
    sc = channel.LeoScenario(n_x=N, n_y=1, K=K, disc_radius=50e3)
    H32 = _traj(sc, 2, 1, seed=950 + K + N)[0].numpy().astype(np.complex64)
    W, X32 = _keep_step(H32, sc, "blocked", bf16=True)
    for b in range(2):
        ref, cancel = reference_product(H32[b], X32[b], sc.p_t, bf16_rne)
        tol = 2 * (4e-4 + 2.0 ** -24 * np.sqrt(2 * K)) * cancel
        assert relerr(W[b], ref) < tol, (b, relerr(W[b], ref), tol)
        # the same operands rounded to TF32 instead are far from the GPU's BF16 product
        ref32, _ = reference_product(H32[b], X32[b], sc.p_t, tf32_rna)
        assert relerr(W[b], ref32) > 4 * relerr(W[b], ref)
