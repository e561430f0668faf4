"""Continuous-batching server: results alone and in the mix, admission by HBM footprint,
states waiting for memory admitted as retires free it."""
import numpy as np
import pytest
import torch

from gpu_harness import relerr, run_oracle
from paper_2512_16543_gb300 import binding, channel, serving
from test_gpu_parity import tf32_w_tol

pytestmark = pytest.mark.gpu

CLASSES = [(256, 32), (512, 64)]                 # (N, K): 16x16 and 32x16 UPA
ARR = {256: (16, 16), 512: (32, 16)}


def _states(n_per_class, T, seed):
    """Per state: class, scenario, snapshots [T, K, N] (complex64, device)."""
    out = []
    for ci, (N, K) in enumerate(CLASSES):
        sc = channel.LeoScenario(n_x=ARR[N][0], n_y=ARR[N][1], K=K)
        p = channel.draw_trajectories(sc, n_per_class, seed=seed + ci)
        Hs = channel.trajectory(p, T, dtype=torch.complex64).cuda()
        for j in range(n_per_class):
            out.append((ci, sc, Hs[:, j].contiguous()))
    return out


def _serve(states, order, rule, bursts):
    """Submit the requests of `order` (state ids) in bursts of the given sizes, pumping
    between bursts, so that requests join launches already in flight."""
    srv = serving.BeamServer([(N, K, 8) for N, K in CLASSES], rule, keep_results=True)
    for sid in sorted(set(order)):
        ci, sc, _ = states[sid]
        assert srv.admit(sid, ci, sc.alpha, sc.sigma2)
    nxt = {sid: 0 for sid in set(order)}
    reqs, i = [], 0
    for b in bursts:
        for sid in order[i:i + b]:
            r = serving.Request(sid, states[sid][2][nxt[sid]])
            nxt[sid] += 1
            srv.submit(r)
            reqs.append(r)
        i += b
        srv.pump()
    srv.drain()
    srv.close()
    return reqs, srv


def test_each_result_is_the_same_alone_and_in_the_mix():
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=16, reinverse_period=5, seed=13)
    states = _states(4, 9, seed=300)
    g = torch.Generator().manual_seed(5)
    order = []
    for _ in range(6):                       # every state 6 requests, interleaved at random
        order += torch.randperm(len(states), generator=g).tolist()
    bursts = [3, 1, 5, 2, 7, 4, 6, 3, 5, 2, 4, 6]
    mix, srv = _serve(states, order, rule, bursts)
    assert all(r.done is not None for r in mix)
    assert srv.classes[0].launches > 2 and srv.classes[1].launches > 2
    for sid in (0, 3, 5, 7):
        alone, _ = _serve(states, [sid] * 6, rule, [1] * 6)
        mine = [r for r in mix if r.state == sid]
        assert len(mine) == len(alone) == 6
        for a, m in zip(alone, mine):
            assert torch.equal(a.W, m.W), sid
            assert a.sum_rate == m.sum_rate
    # and one state against the FP64 oracle (its first request is the full inverse)
    ci, sc, Hs = states[1]
    mine = [r for r in mix if r.state == 1]
    Hn = Hs[:6].cpu().numpy().astype(np.complex128)
    ref = run_oracle(Hn, sc.alpha, sc.sigma2, sc.p_t, rule, instance=1)
    for t, r in enumerate(mine):
        tol = tf32_w_tol(Hn[t], ref[t].X, ref[t].W, sc.p_t, x_tol=1e-4)
        assert relerr(r.W.cpu().numpy(), ref[t].W) < tol
        assert abs(r.sum_rate - ref[t].sum_rate) < 1e-3


def test_admission_respects_the_hbm_budget():
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=16, seed=1)
    probe = serving.BeamServer([(256, 32, 8)], rule)
    per = probe.classes[0].per_state_bytes
    probe.close()
    srv = serving.BeamServer([(256, 32, 8)], rule, budget_bytes=3 * per + per // 2)
    sc = channel.scenario_batched_256x32()
    ok = [srv.admit(s, 0, sc.alpha, sc.sigma2) for s in range(5)]
    assert ok == [True, True, True, False, False]
    H = channel.channel_at(channel.draw_trajectories(sc, 1, seed=2), 0,
                           dtype=torch.complex64, device="cuda")[0]
    assert not srv.submit(serving.Request(4, H))
    assert srv.rejected == 1
    srv.retire(1)
    assert srv.admit(4, 0, sc.alpha, sc.sigma2)
    assert srv.used_bytes <= 3 * per + per // 2
    srv.close()


def test_a_state_waiting_for_memory_is_served_after_a_retire():
    """Budget for two states: a third state's admission waits (not rejected), its requests
    are held while the first two are served, and after a retire frees memory it is admitted
    and served; its results equal the same state served alone, and its latency includes the
    wait."""
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=16, reinverse_period=5, seed=3)
    probe = serving.BeamServer([(256, 32, 4)], rule)
    per = probe.classes[0].per_state_bytes
    probe.close()
    states = _states(3, 4, seed=910)[:3]           # three states of the (256, 32) class
    srv = serving.BeamServer([(256, 32, 4)], rule, budget_bytes=2 * per + per // 2,
                             keep_results=True)
    got = [srv.admit(sid, 0, states[sid][1].alpha, states[sid][1].sigma2, wait=True)
           for sid in range(3)]
    assert got == [True, True, False] and srv.waiting and srv.rejected == 0
    reqs = []
    for t in range(3):
        for sid in range(3):
            r = serving.Request(sid, states[sid][2][t], arrival=0.0)
            assert srv.submit(r)                     # held, not rejected, for state 2
            reqs.append(r)
    srv.drain()
    assert all(r.done is not None for r in reqs if r.state != 2)
    assert all(r.done is None for r in reqs if r.state == 2)
    srv.retire(0)
    assert srv.admitted_after_wait == 1 and not srv.waiting
    assert srv.used_bytes <= 2 * per + per // 2
    srv.drain()
    srv.close()
    mine = [r for r in reqs if r.state == 2]
    assert all(r.done is not None for r in mine)
    assert min(r.done for r in mine) > max(r.done for r in reqs if r.state == 0)
    alone = serving.BeamServer([(256, 32, 4)], rule, keep_results=True)
    assert alone.admit(2, 0, states[2][1].alpha, states[2][1].sigma2)
    ref = []
    for t in range(3):
        r = serving.Request(2, states[2][2][t])
        alone.submit(r)
        ref.append(r)
        alone.drain()
    alone.close()
    for a, m in zip(ref, mine):
        assert torch.equal(a.W, m.W)
        assert a.sum_rate == m.sum_rate
