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


def test_step_info_reports_a_timed_out_instance_with_its_own_code():
    """A TIMEOUT status bit in any instance's step info makes wbrzf_step_info_get return
    WBRZF_ERR_TIMEOUT (7), ahead of WBRZF_ERR_NUMERICAL (4) for other non-zero statuses.  The
    bit is planted on the host side of the contract: written into the step-info record of the
    handle's workspace (the common layout: G, X, then the 32-byte records, each region
    256-byte aligned; status at byte 28), not produced by a GPU wait."""
    sc = channel.scenario_batched_256x32()
    params = channel.draw_trajectories(sc, 3, seed=6)
    h = binding.WBRZF(3, sc.N, sc.K, sc.alpha, sc.sigma2, p_t=sc.p_t)
    h.full_inverse(channel.channel_at(params, 0, device="cuda", dtype=torch.complex64))
    assert [i["status"] for i in h.step_info()] == [0, 0, 0]
    kk = 3 * sc.K * sc.K * 8
    al = lambda x: (x + 255) // 256 * 256
    o_info = al(al(kk) + kk)
    status = h.workspace[o_info:o_info + 3 * 32].view(3, 32)[:, 28:32]
    status[1].copy_(torch.tensor([4, 0, 0, 0], dtype=torch.uint8))        # TIMEOUT
    status[2].copy_(torch.tensor([1, 0, 0, 0], dtype=torch.uint8))        # NOT_PD
    info = h.step_info()
    assert [i["status"] for i in info] == [0, 4, 1]
    with pytest.raises(binding.WbrzfError) as e:
        h.step_info(raise_on_numerical=True)
    assert e.value.code == 7
    status[1].zero_()
    with pytest.raises(binding.WbrzfError) as e:
        h.step_info(raise_on_numerical=True)
    assert e.value.code == 4
    h.close()
