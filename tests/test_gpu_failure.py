"""Failure detection on the GPU without a GPU fault.

The tensor-core kernels bound every wait on a shared-memory mbarrier (for TMA copies and MMAs)
by a %globaltimer deadline; on expiry the CTA records WBRZF_STATUS_TIMEOUT and finishes.  Here
that wait runs out on purpose -- on an mbarrier nothing ever arrives on -- and the host reads
the status; afterwards the same context runs the tensor-core step kernel with clean statuses.
Numerical failures (a Gram matrix that is not positive definite, a singular capacitance) have
their own tests in the parity files.
"""
import ctypes

import pytest
import torch

from paper_2512_16543_gb300 import binding, channel

pytestmark = pytest.mark.gpu

WBRZF_STATUS_TIMEOUT = 4
WAIT_NS = 200_000_000          # the kernels' per-wait deadline


def _selftest():
    f = binding.lib().wbrzf_selftest_bounded_wait
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    return f


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    f = _selftest()
    out = torch.zeros(2, dtype=torch.int64, device="cuda")
    assert f(out.data_ptr(), torch.cuda.current_stream().cuda_stream) == 0
    torch.cuda.synchronize()
    status, waited = out.cpu().tolist()
    assert status == WBRZF_STATUS_TIMEOUT
    assert WAIT_NS <= waited < 25 * WAIT_NS
    assert f(None, None) == 1                          # null output: invalid argument
    assert f(out.data_ptr() + 4, None) == 1            # misaligned output

    sc = channel.scenario_batched_256x32()
    params = channel.draw_trajectories(sc, 4, seed=5)
    rule = binding.RankRule(eta=0.9, k_init=2, p=8, r_max=16, reinverse_period=20, seed=3)
    h = binding.WBRZF(4, sc.N, sc.K, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule)
    h.set_engine("tensor")
    for t in range(3):
        H = channel.channel_at(params, t, device="cuda", dtype=torch.complex64)
        W = h.full_inverse(H) if t == 0 else h.update(H)
    torch.cuda.synchronize()
    assert h.last_engine == "tensor"
    assert all(i["status"] == 0 for i in h.step_info())
    assert bool(torch.isfinite(torch.view_as_real(W)).all())
    h.close()
