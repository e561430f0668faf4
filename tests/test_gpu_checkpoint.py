"""Checkpoint / resume through the C ABI: a handle restored from another handle's exported
state (G, X and the per-instance snapshot indices) continues bit for bit like the original --
the kernels reduce in a fixed order, and the restored t keys Algorithm 1's random draws and
the periodic re-inversion."""
import pytest
import torch

from paper_2512_16543_gb300 import binding, channel

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,engine,K,N", [("c64", "tensor", 32, 256), ("c128", "simt", 8, 64),
                                             ("c64", "blocked", 64, 128)])
def test_restored_handle_continues_like_the_original(prec, engine, K, N):
    B = 6
    sc = channel.LeoScenario(n_x=N // 8, n_y=8, K=K)
    dt = torch.complex64 if prec == "c64" else torch.complex128
    params = channel.draw_trajectories(sc, B, seed=11 + K)
    rule = binding.RankRule(eta=0.9, k_init=2, p=8 if K >= 32 else 1, r_max=min(16, K),
                            reinverse_period=7, seed=5)
    ids = [100 + 3 * i for i in range(B)]

    def make():
        h = binding.WBRZF(B, N, K, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule, precision=prec,
                          workspace_for="blocked" if engine == "blocked" else "auto")
        h.set_engine(engine)
        h.set_instance_ids(ids)
        return h

    Hs = [channel.channel_at(params, t, device="cuda", dtype=dt) for t in range(12)]
    a = make()
    a.full_inverse(Hs[0])
    for t in range(1, 6):
        a.update(Hs[t])
    G, X, steps = a.checkpoint()
    G, X = G.clone(), X.clone()
    assert steps == [6] * B                            # the next snapshot index

    b = make()
    with pytest.raises(binding.WbrzfError) as e:       # nothing to update from yet
        b.update(Hs[6])
    assert e.value.code == 2
    b.restore(G, X, steps)
    assert b.steps() == steps
    branches = set()
    for t in range(6, 12):
        Wa, Wb = a.update(Hs[t]), b.update(Hs[t])
        ra, rb = a.sum_rate()[1], b.sum_rate()[1]
        torch.cuda.synchronize()
        assert torch.equal(Wa, Wb), t
        assert torch.equal(ra, rb), t
        ia, ib = a.step_info(), b.step_info()
        assert [(x["branch"], x["r"], x["status"]) for x in ia] == \
               [(x["branch"], x["r"], x["status"]) for x in ib]
        branches |= {x["branch"] for x in ia}
    assert 1 in branches and 3 in branches             # Woodbury and the periodic re-inverse
    assert b.steps() == a.steps()
    a.close()
    b.close()


def test_restore_rejects_bad_input():
    h = binding.WBRZF(2, 64, 8, 0.1, 0.1, precision="c128")
    G = torch.zeros(2, 8, 8, dtype=torch.complex128, device="cuda")
    with pytest.raises(binding.WbrzfError) as e:
        h.restore(G, G, [0, -1])
    assert e.value.code == 1
    with pytest.raises(ValueError):
        h.restore(G[:1], G, [0, 0])
    h.close()
