"""wbrzf_rzf_noalloc: RZF precoders for callers that cannot allocate device memory.

Such callers (code inside a CUDA-graph stream capture, allocation-free real-time loops,
plug-ins whose framework owns all device memory) get the conventional full-inversion RZF
result without handing the library a workspace: the per-instance scratch comes from a fixed
array inside the library.  These tests call the entry point through the C ABI: twice in a row
on different channels, checking each result against the workspace-based entry point (a
WBRZF_METHOD_FULL_INVERSE handle on the FMA engine, the kernel both share) within the
tolerances the other parity tests use; once recorded into a CUDA graph by stream capture and
replayed on new channels; and with a singular Gram matrix, whose instance must read NaN.
They live in their own file so that they are collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2512_16543_gb300 import binding, channel

pytestmark = pytest.mark.gpu

TOL = {"c128": 1e-10, "c64": 1e-4}


def _fn():
    f = binding.lib().wbrzf_rzf_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                  ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_void_p]
    return f


def _call(H, W, rate, alpha, sigma2, p_t, prec):
    B, K, N = H.shape
    return _fn()(B, N, K, binding.C128 if prec == "c128" else binding.C64, H.data_ptr(),
                 alpha, sigma2, p_t, W.data_ptr(), rate.data_ptr(),
                 torch.cuda.current_stream().cuda_stream)


def _noalloc(H, alpha, sigma2, p_t, prec):
    B, K, N = H.shape
    W = torch.empty(B, N, K, dtype=H.dtype, device=H.device)
    rate = torch.empty(B, dtype=torch.float32, device=H.device)
    return _call(H, W, rate, alpha, sigma2, p_t, prec), W, rate


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


def test_noalloc_replays_from_a_captured_graph():
    """One warm-up call (it resolves the scratch address on this device), then the call is
    recorded into a CUDA graph on a side stream and replayed on two new channels written into
    the same input buffer: each replay matches the workspace-based entry point."""
    B, K, N = 6, 16, 128
    sc = channel.LeoScenario(n_x=16, n_y=8, K=K)
    params = channel.draw_trajectories(sc, B, seed=97)
    H = channel.channel_at(params, 0, device="cuda", dtype=torch.complex64).contiguous()
    W = torch.empty(B, N, K, dtype=torch.complex64, device="cuda")
    rate = torch.empty(B, dtype=torch.float32, device="cuda")
    assert _call(H, W, rate, sc.alpha, sc.sigma2, sc.p_t, "c64") == 0
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=torch.cuda.Stream(), capture_error_mode="thread_local"):
        code = _call(H, W, rate, sc.alpha, sc.sigma2, sc.p_t, "c64")
    assert code == 0
    ref = binding.WBRZF(B, N, K, sc.alpha, sc.sigma2, p_t=sc.p_t, method="full",
                        precision="c64")
    ref.set_engine("simt")
    for t in (7, 23):
        H.copy_(channel.channel_at(params, t, device="cuda", dtype=torch.complex64))
        graph.replay()
        W_ref = ref.update(H)
        _, rate_ref = ref.sum_rate()
        torch.cuda.synchronize()
        a, b = W.cpu().numpy(), W_ref.cpu().numpy()
        assert np.linalg.norm(a - b) / np.linalg.norm(b) <= TOL["c64"]
        np.testing.assert_allclose(rate.cpu().numpy(), rate_ref.cpu().numpy(),
                                   rtol=TOL["c64"], atol=1e-6)
    ref.close()


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_noalloc_marks_a_failed_instance_with_nan(prec):
    """alpha = 0 (zero forcing) and an instance with an all-zero user channel: its G is
    singular, the direct inverse meets a zero pivot, and since this entry point returns no
    step info, that instance's precoder and sum-rate read NaN; the other instance is
    unaffected.  A non-finite p_t is rejected before anything runs."""
    B, K, N = 2, 4, 16
    rng = np.random.default_rng(5)
    Hn = (rng.standard_normal((B, K, N)) + 1j * rng.standard_normal((B, K, N))) / np.sqrt(2 * N)
    Hn[1, 2] = 0.0
    dt = torch.complex64 if prec == "c64" else torch.complex128
    H = torch.from_numpy(Hn).to(device="cuda", dtype=dt).contiguous()
    code, W, rate = _noalloc(H, 0.0, 0.1, 1.0, prec)
    assert code == 0
    torch.cuda.synchronize()
    W, rate = W.cpu().numpy(), rate.cpu().numpy()
    assert np.all(np.isfinite(W[0])) and np.isfinite(rate[0])
    assert np.all(np.isnan(W[1])) and np.isnan(rate[1])
    code, _, _ = _noalloc(H, 0.1, 0.1, float("inf"), prec)
    assert code == 1                          # WBRZF_ERR_INVALID_ARG
