"""wbrzf_rzf_noalloc: RZF precoders for callers that cannot allocate device memory.

Such callers (code inside a CUDA-graph stream capture, allocation-free real-time loops,
plug-ins whose framework owns all device memory) get the conventional full-inversion RZF
result without handing the library a workspace: the per-instance scratch comes from a fixed
array inside the library.  This test calls the entry point through the C ABI twice in a row
on different channels and checks each result against the workspace-based entry point
(a WBRZF_METHOD_FULL_INVERSE handle on the FMA engine, the kernel both share), within the
tolerances the other parity tests use.
It lives in its own file so that it is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2512_16543_gb300 import binding, channel

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-4}


def _noalloc(H, alpha, sigma2, p_t, prec):
    L = binding.lib()
    f = L.wbrzf_rzf_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    B, K, N = H.shape
    W = torch.empty(B, N, K, dtype=H.dtype, device=H.device)
    rate = torch.empty(B, dtype=torch.float32, device=H.device)
    code = f(B, N, K, binding.C128 if prec == "c128" else binding.C64, H.data_ptr(), alpha,
             sigma2, p_t, W.data_ptr(), rate.data_ptr(),
             torch.cuda.current_stream().cuda_stream)
    return code, W, rate


@pytest.mark.parametrize("prec,shape", [("c128", (5, 8, 64)), ("c64", (7, 32, 256))])
def test_noalloc_matches_workspace_entry_point_twice(prec, shape):
    B, K, N = shape
    sc = channel.LeoScenario(n_x=N // 8, n_y=8, K=K)
    dt = torch.complex128 if prec == "c128" else torch.complex64
    params = channel.draw_trajectories(sc, B, seed=31 + K)
    ref = binding.WBRZF(B, N, K, sc.alpha, sc.sigma2, p_t=sc.p_t, method="full",
                        precision=prec)
    ref.set_engine("simt")               # the kernel the allocation-free call runs
    for t in (0, 40):                    # two calls in a row, different channels
        H = channel.channel_at(params, t, device="cuda", dtype=dt)
        code, W, rate = _noalloc(H, sc.alpha, sc.sigma2, sc.p_t, prec)
        assert code == 0
        W_ref = ref.update(H)
        _, rate_ref = ref.sum_rate()
        torch.cuda.synchronize()
        a, b = W.cpu().numpy(), W_ref.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL[prec]
        np.testing.assert_allclose(rate.cpu().numpy(), rate_ref.cpu().numpy(),
                                   rtol=TOL[prec], atol=1e-6)
    ref.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    H = torch.zeros(1, dtype=torch.complex64, device="cuda")
    code, _, _ = _noalloc(H.view(1, 1, 1), 0.1, 0.1, 1.0, "c64")
    assert code == 0
    f = binding.lib().wbrzf_rzf_noalloc
    too_many = 4097                           # WBRZF_NOALLOC_MAX_BATCH + 1
    code = f(too_many, 8, 4, binding.C64, H.data_ptr(), 0.1, 0.1, 1.0, H.data_ptr(), None,
             None)
    assert code == 6                          # WBRZF_ERR_UNSUPPORTED, nothing launched
