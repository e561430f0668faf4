"""Masked steps: only the instances of the active mask take a snapshot.

Each instance keeps its own snapshot index t, so an instance that takes its k-th update in a
step where any other set of instances is active gives the same bits as the same instance
updated alone, and (complex128) the oracle run over that instance's own snapshots.  Inactive
instances keep their state, step info, snapshot index and W rows.
"""
import numpy as np
import pytest
import torch

from gpu_harness import relerr, run_oracle
from paper_2512_16543_gb300 import binding, channel

pytestmark = pytest.mark.gpu

CASES = [("simt", "c128"), ("simt", "c64"), ("tensor", "c64"), ("blocked", "c64"),
         ("blocked_fma", "c64"), ("blocked", "c128")]


def _mask_at(step, B):
    # instance 0 every step, 1 every other step, 2 every third, 3 never after the init
    return [1, int(step % 2 == 0), int(step % 3 == 0), 0][:B]


@pytest.mark.parametrize("engine,prec", CASES)
def test_masked_updates_match_alone_and_keep_inactive(engine, prec):
    sc = channel.scenario_single_small() if prec == "c128" else channel.scenario_batched_256x32()
    B, S = 4, 9
    dt = torch.complex128 if prec == "c128" else torch.complex64
    params = channel.draw_trajectories(sc, B, seed=61)
    Hs = channel.trajectory(params, S + 1, dtype=dt)              # [S+1, B, K, N]
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=min(sc.K, 16), reinverse_period=4,
                            seed=21)
    wsf = "blocked" if engine.startswith("blocked") else "auto"
    h = binding.WBRZF(B, sc.N, sc.K, sc.alpha, sc.sigma2, rule=rule, precision=prec,
                      workspace_for=wsf)
    h.set_engine(engine)
    h.full_inverse(Hs[0].cuda().contiguous())
    cnt = [1] * B                        # next snapshot index of each instance's trajectory
    W = torch.full((B, sc.N, sc.K), 7 + 7j, dtype=dt, device="cuda")
    seen = {b: [] for b in range(B)}     # (W, X) after each update the instance takes
    for step in range(S):
        m = _mask_at(step, B)
        H = torch.randn(B, sc.K, sc.N, dtype=dt, device="cuda")      # rows of inactive: noise
        for b in range(B):
            if m[b]:
                H[b] = Hs[cnt[b], b].cuda()
        G0, X0 = h.state()
        info0 = h.step_info()
        W.fill_(7 + 7j)
        h.update(H, W, active=torch.tensor(m, dtype=torch.uint8, device="cuda"))
        G1, X1 = h.state()
        info1 = h.step_info()
        torch.cuda.synchronize()
        for b in range(B):
            if m[b]:
                cnt[b] += 1
                seen[b].append((W[b].cpu().numpy(), X1[b].cpu().numpy()))
            else:
                assert torch.equal(G1[b], G0[b]) and torch.equal(X1[b], X0[b])
                assert bool((W[b] == 7 + 7j).all())
                assert info1[b] == info0[b]
    assert h.steps() == cnt
    h.close()
    # each instance alone, plain updates over its own snapshots
    for b in range(B):
        a = binding.WBRZF(1, sc.N, sc.K, sc.alpha, sc.sigma2, rule=rule, precision=prec,
                          workspace_for=wsf)
        a.set_engine(engine)
        a.set_instance_ids([b])
        a.full_inverse(Hs[0, b:b + 1].cuda().contiguous())
        for k, (Wm, Xm) in enumerate(seen[b]):
            Wa = a.update(Hs[k + 1, b:b + 1].cuda().contiguous())
            _, Xa = a.state()
            np.testing.assert_array_equal(Wa[0].cpu().numpy(), Wm)
            np.testing.assert_array_equal(Xa[0].cpu().numpy(), Xm)
        a.close()
        if prec == "c128" and engine == "simt" and seen[b]:
            ref = run_oracle(Hs[:len(seen[b]) + 1, b].numpy(), sc.alpha, sc.sigma2, sc.p_t, rule,
                             instance=b)
            for k, (Wm, _) in enumerate(seen[b]):
                assert relerr(Wm, ref[k + 1].W) < 1e-10


def test_masked_full_inverse_reinitialises_only_the_masked_instances():
    sc = channel.scenario_single_small()
    B = 3
    params = channel.draw_trajectories(sc, B, seed=5)
    Hs = channel.trajectory(params, 4, dtype=torch.complex128).cuda()
    h = binding.WBRZF(B, sc.N, sc.K, sc.alpha, sc.sigma2, precision="c128")
    h.full_inverse(Hs[0].contiguous())
    h.update(Hs[1].contiguous())
    h.update(Hs[2].contiguous())
    assert h.steps() == [3, 3, 3]
    _, X0 = h.state()
    h.full_inverse(Hs[3].contiguous(), active=torch.tensor([0, 1, 0], dtype=torch.uint8,
                                                            device="cuda"))
    _, X1 = h.state()
    assert h.steps() == [3, 1, 3]
    assert torch.equal(X1[0], X0[0]) and torch.equal(X1[2], X0[2])
    A = Hs[3, 1] @ Hs[3, 1].conj().T + sc.alpha * torch.eye(sc.K, dtype=torch.complex128,
                                                             device="cuda")
    assert float((X1[1] @ A - torch.eye(sc.K, device="cuda")).abs().max()) < 1e-11
    h.close()
