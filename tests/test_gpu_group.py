"""CUDA-graph replay and groups of handles (uneven batches).

A replayed step reads everything from device memory (H's contents, per-instance snapshot
index, state), so replay must give the same bits as enqueueing; a group steps its members on
streams of their own and must give each member the same bits as stepping it alone.
"""
import numpy as np
import pytest
import torch

from gpu_harness import relerr, run_oracle
from paper_2512_16543_gb300 import binding, channel
from test_gpu_parity import tf32_w_tol

pytestmark = pytest.mark.gpu


def _handle(sc, B, prec, rule, engine, seed_ids=0):
    wsf = "blocked" if engine.startswith("blocked") else "auto"
    h = binding.WBRZF(B, sc.N, sc.K, sc.alpha, sc.sigma2, rule=rule, precision=prec,
                      workspace_for=wsf)
    if engine != "auto":
        h.set_engine(engine)
    return h


@pytest.mark.parametrize("engine,prec", [("simt", "c128"), ("tensor", "c64"), ("blocked", "c64"),
                                         ("blocked_fma", "c128")])
def test_graph_replay_gives_the_enqueued_bits(engine, prec):
    sc = channel.scenario_batched_256x32() if prec == "c64" else channel.scenario_single_small()
    B, T = 3, 9
    dt = torch.complex64 if prec == "c64" else torch.complex128
    Hs = channel.trajectory(channel.draw_trajectories(sc, B, seed=9), T, dtype=dt).cuda()
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=min(16, sc.K), reinverse_period=4,
                            seed=3)
    a = _handle(sc, B, prec, rule, engine)
    g = _handle(sc, B, prec, rule, engine)
    g.set_graph(True)
    Hbuf = torch.empty_like(Hs[0])          # the graph is keyed on fixed buffers
    Wa = torch.empty(B, sc.N, sc.K, dtype=dt, device="cuda")
    Wg = torch.empty_like(Wa)
    for t in range(T):
        Hbuf.copy_(Hs[t])
        if t == 0:
            a.full_inverse(Hbuf, Wa)
            g.full_inverse(Hbuf, Wg)
        else:
            a.update(Hbuf, Wa)
            g.update(Hbuf, Wg)
        torch.cuda.synchronize()
        assert torch.equal(Wa, Wg), t
        assert torch.equal(a.state()[1], g.state()[1]), t
        assert a.step_info() == g.step_info()
    assert a.launches == g.launches and a.last_engine == g.last_engine
    assert a.steps() == g.steps()
    a.close()
    g.close()


def test_graph_replay_with_conditional_blocks_at_k128():
    """The blocked engine at K = 128 (N = 256) under CUDA-graph replay, where Algorithm 1's
    iterations beyond the fused kernel's sketch widths, the batched Woodbury products and the
    direct inverse are IF nodes of the graph, skipped when no instance needs them: eta = 0.99
    makes some instances iterate past the fused widths, and the periodic re-inversion (every 3
    snapshots) switches the direct inverse on and off.  Replay gives the enqueued bits."""
    sc = channel.LeoScenario(n_x=16, n_y=16, K=128, disc_radius=100e3)
    B, T = 4, 8
    Hs = channel.trajectory(channel.draw_trajectories(sc, B, seed=128), T,
                            dtype=torch.complex64).cuda()
    rule = binding.RankRule(eta=0.99, k_init=2, p=8, r_max=64, reinverse_period=3, seed=5)
    a = _handle(sc, B, "c64", rule, "blocked")
    g = _handle(sc, B, "c64", rule, "blocked")
    g.set_graph(True)
    Hbuf = torch.empty_like(Hs[0])
    Wa = torch.empty(B, sc.N, sc.K, dtype=torch.complex64, device="cuda")
    Wg = torch.empty_like(Wa)
    iters = set()
    for t in range(T):
        Hbuf.copy_(Hs[t])
        if t == 0:
            a.full_inverse(Hbuf, Wa)
            g.full_inverse(Hbuf, Wg)
        else:
            a.update(Hbuf, Wa)
            g.update(Hbuf, Wg)
        torch.cuda.synchronize()
        assert torch.equal(Wa, Wg), t
        assert torch.equal(a.state()[1], g.state()[1]), t
        info = a.step_info()
        assert info == g.step_info()
        iters |= {i["iters"] for i in info}
    assert max(iters) >= 3           # iterations beyond the fused widths (d <= 24) were taken
    a.close()
    g.close()


def _classes():
    return [(channel.LeoScenario(n_x=8, n_y=8, K=8), 3, "simt"),
            (channel.scenario_batched_256x32(), 4, "tensor"),
            (channel.LeoScenario(n_x=20, n_y=10, K=80, disc_radius=100e3), 2, "blocked")]


@pytest.mark.parametrize("graph", [False, True])
def test_group_gives_each_member_its_own_bits(graph):
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=16, reinverse_period=5, seed=8)
    T = 7
    cls = _classes()
    Hs = [channel.trajectory(channel.draw_trajectories(sc, B, seed=40 + i), T,
                             dtype=torch.complex64).cuda() for i, (sc, B, _) in enumerate(cls)]
    mk = lambda: [_handle(sc, B, "c64", rule, e) for sc, B, e in cls]   # noqa: E731
    solo, members = mk(), mk()
    grp = binding.WBRZFGroup(members)
    grp.set_graph(graph)
    Hb = [torch.empty_like(H[0]) for H in Hs]
    Wg = [torch.empty(B, sc.N, sc.K, dtype=torch.complex64, device="cuda") for sc, B, _ in cls]
    for t in range(T):
        for i in range(len(cls)):
            Hb[i].copy_(Hs[i][t])
        (grp.full_inverse if t == 0 else grp.update)(Hb, Wg)
        torch.cuda.synchronize()
        for i, h in enumerate(solo):
            W = h.full_inverse(Hs[i][t].contiguous()) if t == 0 else h.update(Hs[i][t].contiguous())
            torch.cuda.synchronize()
            assert torch.equal(W, Wg[i]), (t, i)
            assert torch.equal(h.state()[1], members[i].state()[1]), (t, i)
    assert [h.last_engine for h in members] == ["simt", "tensor", "blocked"]
    grp.close()
    for h in solo + members:
        h.close()


def test_group_autotune_chooses_an_accepted_engine_and_keeps_parity():
    rule = binding.RankRule(eta=0.9, k_init=2, p=4, r_max=16, reinverse_period=20, seed=8)
    cls = _classes()
    Hs = [channel.trajectory(channel.draw_trajectories(sc, B, seed=70 + i), 4,
                             dtype=torch.complex64).cuda() for i, (sc, B, _) in enumerate(cls)]
    members = [_handle(sc, B, "c64", rule, "blocked") for sc, B, _ in cls]   # any engine fits
    grp = binding.WBRZFGroup(members)
    Ws = [torch.empty(B, sc.N, sc.K, dtype=torch.complex64, device="cuda") for sc, B, _ in cls]
    chosen = grp.autotune([H[0] for H in Hs], [H[1] for H in Hs], Ws, reps=2)
    for h, e in zip(members, chosen):           # the launch shape is one of the grid's
        cap, jmin = h.blocked_tuning
        assert cap in (32, 64) and jmin in (12, 65) if e.startswith("blocked") else True
    assert chosen[0] in ("tensor", "simt", "blocked", "blocked_fma")
    assert chosen[1] in ("tensor", "simt", "blocked", "blocked_fma")
    assert chosen[2] in ("blocked", "blocked_fma")                  # K = 80: blocked only
    outs = []
    for t in range(1, 4):
        grp.update([H[t] for H in Hs], Ws)
        torch.cuda.synchronize()
        outs.append([W.cpu().numpy() for W in Ws])
    for i, (sc, B, _) in enumerate(cls):
        tf32 = chosen[i] in ("tensor", "blocked")
        for b in range(B):
            Hb = Hs[i][:, b].cpu().numpy().astype(np.complex128)
            ref = run_oracle(Hb, sc.alpha, sc.sigma2, sc.p_t, rule, instance=b)
            for t in range(1, 4):
                tol = (tf32_w_tol(Hb[t], ref[t].X, ref[t].W, sc.p_t, x_tol=1e-4) if tf32
                       else 1e-4)
                assert relerr(outs[t - 1][i][b], ref[t].W) < tol, (i, b, t, chosen[i])
    grp.close()
    for h in members:
        h.close()


def test_blocked_launch_shapes_keep_results():
    """The batched GEMMs' tile cap changes no result (each output's k-sum keeps its order):
    bitwise equal W and X with 64- and 32-wide tiles and the automatic choice.  The one-warp and the CTA-wide
    eigensolvers both meet the oracle at the complex64 tolerances."""
    sc = channel.LeoScenario(n_x=16, n_y=8, K=96, disc_radius=100e3)
    Hs = channel.trajectory(channel.draw_trajectories(sc, 3, seed=96), 5, dtype=torch.complex128)
    rule = binding.RankRule(eta=0.9, k_init=2, p=8, r_max=32, reinverse_period=3, seed=2)
    outs = {}
    for cap, jmin in ((64, 12), (32, 12), (0, 12), (64, 65)):
        h = binding.WBRZF(3, sc.N, sc.K, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule,
                          workspace_for="blocked")
        h.set_engine("blocked")
        h.set_blocked_tuning(cap, jmin)
        assert h.blocked_tuning == (cap, jmin)
        rec = []
        for t in range(5):
            H = Hs[t].to(device="cuda", dtype=torch.complex64)
            W = h.full_inverse(H) if t == 0 else h.update(H)
            rec.append((W.cpu().numpy(), h.state()[1].cpu().numpy(), h.step_info()))
        outs[(cap, jmin)] = rec
        h.close()
    for t in range(5):
        np.testing.assert_array_equal(outs[(64, 12)][t][0], outs[(32, 12)][t][0])
        np.testing.assert_array_equal(outs[(64, 12)][t][1], outs[(32, 12)][t][1])
        np.testing.assert_array_equal(outs[(64, 12)][t][0], outs[(0, 12)][t][0])
        np.testing.assert_array_equal(outs[(64, 12)][t][1], outs[(0, 12)][t][1])
    for key in ((64, 12), (64, 65)):
        for b in range(3):
            Hb = Hs[:, b].numpy().astype(np.complex64).astype(np.complex128)
            ref = run_oracle(Hb, sc.alpha, sc.sigma2, sc.p_t, rule, instance=b)
            for t in range(5):
                W, X, info = outs[key][t]
                assert relerr(X[b], ref[t].X) < 1e-4, (key, t, b)
                assert relerr(W[b], ref[t].W) < tf32_w_tol(Hb[t], X[b], ref[t].W, sc.p_t)
    with pytest.raises(binding.WbrzfError):
        h = binding.WBRZF(1, sc.N, sc.K, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule)
        try:
            h.set_blocked_tuning(48, 12)
        finally:
            h.close()
