"""The shared synthetic-channel generator (Section II eqs. 1-3 readings)."""
import math

import numpy as np
import torch

from paper_2512_16543_gb300 import channel as ch


def test_shapes_dtype_and_reproducibility():
    sc = ch.scenario_single_small()
    p1 = ch.draw_trajectories(sc, 3, seed=11)
    p2 = ch.draw_trajectories(sc, 3, seed=11)
    H1 = ch.channel_at(p1, 5)
    H2 = ch.channel_at(p2, 5)
    assert H1.shape == (3, sc.K, sc.N) and H1.dtype == torch.complex128
    assert torch.equal(H1, H2)
    assert not torch.equal(H1, ch.channel_at(ch.draw_trajectories(sc, 3, seed=12), 5))
    assert ch.channel_at(p1, 5, dtype=torch.complex64).dtype == torch.complex64


def test_los_part_is_unit_norm_steering_times_gain():
    sc = ch.LeoScenario(n_x=4, n_y=4, K=3, k_rician_db=300.0)   # K_R -> infinity: pure LOS
    p = ch.draw_trajectories(sc, 2, seed=1)
    H = ch.channel_at(p, 0).numpy()
    xy = p.user_xy.numpy()
    dist = np.sqrt(xy[..., 0] ** 2 + xy[..., 1] ** 2 + sc.h_alt ** 2)
    np.testing.assert_allclose(np.linalg.norm(H, axis=-1), sc.h_alt / dist, rtol=1e-12)
    # every element has the same modulus (a = N^-1/2 exp(j kappa . r_m))
    ref = np.broadcast_to((sc.h_alt / dist)[..., None] / math.sqrt(sc.N), H.shape)
    np.testing.assert_allclose(np.abs(H), ref, rtol=1e-12)


def test_steering_phase_matches_geometry():
    sc = ch.LeoScenario(n_x=2, n_y=1, K=1, k_rician_db=300.0)
    p = ch.draw_trajectories(sc, 1, seed=2)
    H = ch.channel_at(p, 3).numpy()[0, 0]
    x, y = p.user_xy.numpy()[0, 0]
    xs = sc.v * sc.dt * 3
    d = np.array([x - xs, y, -sc.h_alt])
    u = d / np.linalg.norm(d)
    # elements at x = -lambda/4 and +lambda/4: phase difference kappa_x * lambda / 2 = pi u_x
    dphi = np.angle(H[1] / H[0])
    assert abs(dphi - math.pi * u[0]) < 1e-9


def test_rician_power_split_and_parameters():
    sc = ch.scenario_batched_256x32()
    assert sc.N == 256 and sc.K == 32
    assert abs(sc.alpha - 32 / 10.0) < 1e-12 and abs(sc.sigma2 - 0.1) < 1e-12
    p = ch.draw_trajectories(sc, 64, seed=3)
    g = p.g_nlos.numpy()
    assert abs(np.mean(np.sum(np.abs(g) ** 2, axis=-1)) - 1.0) < 0.02   # E||g||^2 = 1


def test_device_argument_and_subset():
    sc = ch.scenario_single_small()
    p = ch.draw_trajectories(sc, 4, seed=4)
    full = ch.channel_at(p, 2)
    sub = ch.channel_at(p, 2, index=torch.tensor([1, 3]))
    assert torch.equal(sub, full[[1, 3]])
    T = ch.trajectory(p, 3, t0=2)
    assert torch.equal(T[0], full)


def test_uneven_population_is_seeded_and_spans_the_ranges():
    a = ch.uneven_population(600, seed=4)
    b = ch.uneven_population(600, seed=4)
    assert sum(c.batch for c in a) == 600 and len(a) == 12
    idx = torch.cat([c.index for c in a])
    assert torch.equal(torch.sort(idx).values, torch.arange(600))
    for ca, cb in zip(a, b):
        assert torch.equal(ca.index, cb.index) and torch.equal(ca.radius, cb.radius)
        assert torch.equal(ca.params.user_xy, cb.params.user_xy)
        assert ca.scenario.N in (256, 512, 1024) and ca.scenario.K in (16, 32, 64, 128)
        assert float(ca.radius.min()) >= 20e3 and float(ca.radius.max()) <= 200e3
        assert float(ca.snr_db.min()) >= 0.0 and float(ca.snr_db.max()) <= 20.0
        # users lie inside their instance's own disc
        r = ca.params.user_xy.norm(dim=-1)
        assert bool((r <= ca.radius[:, None] + 1e-6).all())
        np.testing.assert_allclose(ca.alpha, [ca.scenario.K * s for s in ca.sigma2])


def test_dft_codebook_and_beam_users():
    sc = ch.scenario_paper_hybrid()
    cb = ch.dft_codebook(sc)
    np.testing.assert_allclose((cb.conj().T @ cb).numpy(), np.eye(sc.N), atol=1e-12)
    p = ch.draw_beam_users(sc, 3, seed=8)
    beams = ch.best_power_beams(ch.steering_at(p, 0), cb)
    for b in range(3):                     # one user per beam cell at mid-pass
        assert len(set(beams[b].tolist())) == sc.K
    He, Ht, F = ch.hybrid_channels(p, 5, cb)
    assert He.shape == (3, sc.K, sc.K) and Ht.dtype == torch.complex128
    # H_eff is the steering part seen through the selected beams
    A = ch.steering_at(p, 5)
    np.testing.assert_allclose(He.numpy(), (A @ F).numpy(), atol=1e-12)
