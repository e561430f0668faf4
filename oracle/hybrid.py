"""Hybrid beamforming of Section II (oracle, FP64): test infrastructure only.

The satellite steers one analog beam per user from a DFT codebook, chosen by best power, and
computes the RZF digital precoder on the effective channel (Section II eq. 4 and eq. 5):

  H_eff = H~ F_RF (K x N_RF), H~ = [h~_1 ... h~_K]^T the array-manifold vectors a(theta, phi)
          that the satellite knows from positions;
  F_BB  = H_eff^H (H_eff H_eff^H + alpha I_K)^{-1}, scaled so that ||F_RF F_BB||_F^2 = P_t;
  R_sum = sum_n log2(1 + |g_nn|^2 / (sum_{i != n} |g_ni|^2 + sigma^2)) (Section VI eq. 15) with
          g_ni = (H F_RF F_BB)_{n i}, H the Rician channel of eqs. 1-3, user n's channel row n.

The paper does not spell out the codebook's grid.  The reading used here, and pinned by the
tests through its orthonormality: an n_x x n_y uniform planar array at half-wavelength spacing,
element m = m_y n_x + m_x at (m_x - (n_x - 1)/2, m_y - (n_y - 1)/2) half-wavelengths, and beam
(p, q) (column p n_y + q) steering to the direction cosines (u_x, u_y) = (-1 + 2p/n_x,
-1 + 2q/n_y), entry exp(j pi (x_m u_x + y_m u_y)) / sqrt(N).  Plain loops, written from those
definitions.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

from . import rzf


def dft_codebook(n_x: int, n_y: int) -> np.ndarray:
    """The N x N codebook (N = n_x n_y) described above."""
    N = n_x * n_y
    F = np.zeros((N, N), dtype=np.complex128)
    for p in range(n_x):
        for q in range(n_y):
            ux = -1.0 + 2.0 * p / n_x
            uy = -1.0 + 2.0 * q / n_y
            col = p * n_y + q
            for my in range(n_y):
                for mx in range(n_x):
                    x = mx - (n_x - 1) / 2.0
                    y = my - (n_y - 1) / 2.0
                    F[my * n_x + mx, col] = cmath.exp(1j * math.pi * (x * ux + y * uy)) / math.sqrt(N)
    return F


def best_power_beams(A: np.ndarray, F: np.ndarray) -> list[int]:
    """For each user (row k of the array-manifold matrix A, K x N) the codebook column f with
    the largest beamforming power |a_k^H f|^2 (the first one on ties)."""
    beams = []
    for k in range(A.shape[0]):
        best, arg = -1.0, 0
        for m in range(F.shape[1]):
            pw = abs(np.vdot(A[k], F[:, m])) ** 2
            if pw > best:
                best, arg = pw, m
        beams.append(arg)
    return beams


def analog_precoder(F: np.ndarray, beams: list[int]) -> np.ndarray:
    """F_RF = [f_{beam_1} ... f_{beam_K}] (N x N_RF, N_RF = K)."""
    return np.stack([F[:, b] for b in beams], axis=1)


def digital_precoder(H_eff: np.ndarray, F_RF: np.ndarray, alpha: float, P_t: float):
    """F_BB = H_eff^H A^{-1} (eq. 5, A = H_eff H_eff^H + alpha I, inverted by Gauss-Jordan) scaled
    so that ||F_RF F_BB||_F^2 = P_t; returns (F_BB, scale)."""
    A = rzf.gram(H_eff, alpha)
    X = rzf.inverse_gauss_jordan(A)
    F_BB = rzf.rzf_unnormalised(H_eff, X)
    s = math.sqrt(P_t) / np.linalg.norm(F_RF @ F_BB)
    return s * F_BB, s


def sum_rate_through_beams(H: np.ndarray, F_RF: np.ndarray, F_BB: np.ndarray,
                           sigma2: float) -> float:
    """R_sum of eq. 15 with gains g = H F_RF F_BB (H: K x N, user n's channel in row n)."""
    g = H @ F_RF @ F_BB
    K = g.shape[0]
    R = 0.0
    for n in range(K):
        sig = abs(g[n, n]) ** 2
        intf = sum(abs(g[n, i]) ** 2 for i in range(K) if i != n)
        R += math.log2(1.0 + sig / (intf + sigma2))
    return R


def hybrid_rzf(A: np.ndarray, H: np.ndarray, n_x: int, n_y: int, alpha: float, P_t: float,
               sigma2: float, F: np.ndarray | None = None) -> dict:
    """The whole hybrid step for one snapshot: beams from the array-manifold vectors A (K x N),
    the digital RZF precoder from H_eff = A F_RF, and the sum-rate on the channel H (K x N)
    through the same beams.  F: the codebook dft_codebook(n_x, n_y), if already built."""
    if F is None:
        F = dft_codebook(n_x, n_y)
    beams = best_power_beams(A, F)
    F_RF = analog_precoder(F, beams)
    H_eff = A @ F_RF
    F_BB, s = digital_precoder(H_eff, F_RF, alpha, P_t)
    return {"beams": beams, "F_RF": F_RF, "H_eff": H_eff, "F_BB": F_BB, "scale": s,
            "sum_rate": sum_rate_through_beams(H, F_RF, F_BB, sigma2)}
