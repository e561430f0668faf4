"""Pins of the hybrid-beamforming oracle (Section II eq. 4 and eq. 5, Section VI eq. 15)."""
import math

import numpy as np

from oracle import hybrid, rzf


def _rand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def test_dft_codebook_is_unitary():
    # half-wavelength 2-D DFT: the N beams are orthonormal (a wrong grid or spacing breaks it)
    for nx, ny in ((4, 4), (2, 3), (8, 2)):
        F = hybrid.dft_codebook(nx, ny)
        assert np.max(np.abs(F.conj().T @ F - np.eye(nx * ny))) < 1e-12


def test_a_user_on_the_grid_picks_its_own_beam():
    F = hybrid.dft_codebook(4, 4)
    A = np.stack([F[:, 5], F[:, 10], 0.8 * F[:, 3] + 0.6 * F[:, 12]])
    beams = hybrid.best_power_beams(A, F)
    assert beams == [5, 10, 3]          # the third: |0.8|^2 > |0.6|^2


def test_single_user_closed_form():
    # K = N_RF = 1: R = log2(1 + P_t |h f|^2 / sigma^2) whatever alpha
    rng = np.random.default_rng(1)
    F = hybrid.dft_codebook(3, 3)
    a = F[:, 4:5].T.copy()
    h = a + 0.3 * _rand(rng, 1, 9)
    for alpha in (0.0, 0.5, 7.0):
        out = hybrid.hybrid_rzf(a, h, 3, 3, alpha, P_t=2.0, sigma2=0.25)
        f = out["F_RF"][:, 0]
        assert out["beams"] == [4]
        assert abs(out["sum_rate"] - math.log2(1 + 2.0 * abs(h[0] @ f) ** 2 / 0.25)) < 1e-12


def test_a_full_unitary_analog_stage_leaves_rzf_unchanged():
    # N_RF = N with all N orthonormal beams: F_RF F_BB = H^H (H H^H + alpha I)^{-1} up to the
    # scale, so precoder and sum-rate equal the fully digital RZF of eq. 5
    rng = np.random.default_rng(2)
    nx, ny, K = 3, 2, 4
    F = hybrid.dft_codebook(nx, ny)
    H = _rand(rng, K, nx * ny)
    F_BB, _ = hybrid.digital_precoder(H @ F, F, 0.4, 1.5)
    ref = rzf.full_inversion_rzf(H, 0.4, 1.5, 0.2)
    assert np.max(np.abs(F @ F_BB - ref["W"])) < 1e-12
    assert abs(hybrid.sum_rate_through_beams(H, F, F_BB, 0.2) - ref["sum_rate"]) < 1e-12


def test_power_constraint_and_zero_forcing_through_beams():
    # ||F_RF F_BB||_F^2 = P_t; alpha -> 0 on the geometric channel itself: no interference, so
    # R = K log2(1 + s^2 / sigma^2) with s the common diagonal gain
    rng = np.random.default_rng(3)
    F = hybrid.dft_codebook(4, 4)
    beams = [1, 6, 11, 14]
    A = np.stack([F[:, b] + 0.2 * _rand(rng, 16) for b in beams])
    out = hybrid.hybrid_rzf(A, A, 4, 4, 1e-12, P_t=3.0, sigma2=0.1)
    assert out["beams"] == beams
    assert abs(np.linalg.norm(out["F_RF"] @ out["F_BB"]) ** 2 - 3.0) < 1e-10
    g = out["H_eff"] @ out["F_BB"]
    s = abs(g[0, 0])
    assert np.max(np.abs(g - s * np.eye(4))) < 1e-9
    assert abs(out["sum_rate"] - 4 * math.log2(1 + s * s / 0.1)) < 1e-8
