"""Low-rank approximation of the Gram perturbation (oracle, FP64).

Section IV, eqs. 13-14: the truncated SVD keeps the smallest number r of leading singular
triplets of dA whose squared singular values reach a fraction eta of ||dA||_F^2.

Section IV-A, Algorithm 1 (adaptive randomized SVD): with E_target = eta ||dA||_F^2 and a
working rank k0 starting at k_init, each iteration takes d = min(k0 + p, K), draws a Gaussian
Omega (K x d), forms the sketch Y = dA Omega, an orthonormal basis Q = orth(Y) (thin QR),
the projection B = Q^H dA, and the SVD B = U_hat Sigma_hat V_hat^H.  If some r <= d makes
the leading r squared singular values of B reach E_target, the factors
U_r = Q U_hat[:, :r], Sigma_r, V_r = V_hat[:, :r] and k_est = r are returned; otherwise k0
doubles.  After I_max iterations without success all d components of the last iteration are
returned with k_est = d.

Library primitives used as single steps: numpy.linalg.qr for the thin QR and numpy.linalg.svd
for the SVDs.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable

import numpy as np


def energy_rank(sigma: np.ndarray, E_target: float) -> int | None:
    """Smallest r >= 1 with sum_{j<=r} sigma_j^2 >= E_target (sigma sorted descending).

    Returns None when even all of sigma falls short (eq. 14, Algorithm 1).
    """
    cum = 0.0
    for r, s in enumerate(np.asarray(sigma, dtype=np.float64), start=1):
        cum += float(s) * float(s)
        if cum >= E_target:
            return r
    return None


@dataclass
class LowRank:
    """dA ~= U diag(S) V^H with rank k_est = len(S)."""

    U: np.ndarray          # K x r
    S: np.ndarray          # r
    V: np.ndarray          # K x r
    k_est: int
    iters: int = 0         # Algorithm 1 iterations used (0 for the exact SVD)
    met: bool = True       # energy target reached
    last_d: int = 0        # sketch width of the last iteration
    sigma_hat: np.ndarray | None = None   # singular values of the last B

    def product(self) -> np.ndarray:
        return (self.U * self.S) @ self.V.conj().T


def truncated_svd(dA: np.ndarray, eta: float) -> LowRank:
    """Exact SVD of dA (eq. 13) truncated by the energy rule (eq. 14)."""
    dA = np.asarray(dA, dtype=np.complex128)
    U, S, Vh = np.linalg.svd(dA)
    E_target = eta * float(np.sum(np.abs(dA) ** 2))
    r = energy_rank(S, E_target)
    if r is None:            # only possible through rounding when eta == 1
        r = len(S)
    return LowRank(U[:, :r], S[:r], Vh[:r].conj().T, k_est=r, iters=0, met=True,
                   last_d=dA.shape[0], sigma_hat=S)


def arsvd(dA: np.ndarray, eta: float, k_init: int, p: int, i_max: int,
          draw_omega: Callable[[int, int], np.ndarray]) -> LowRank:
    """Algorithm 1.  draw_omega(it, d) returns the K x d test matrix of iteration `it`
    (0-based); it is the only source of randomness."""
    dA = np.asarray(dA, dtype=np.complex128)
    K = dA.shape[0]
    E_target = eta * float(np.sum(np.abs(dA) ** 2))
    k0 = k_init
    U_approx = S_hat = V_hat = None
    d = 0
    for it in range(i_max):
        d = min(k0 + p, K)
        Om = np.asarray(draw_omega(it, d), dtype=np.complex128)
        assert Om.shape == (K, d)
        Y = dA @ Om
        Q, _ = np.linalg.qr(Y, mode="reduced")
        B = Q.conj().T @ dA
        U_hat, S_hat, V_hat_h = np.linalg.svd(B, full_matrices=False)
        V_hat = V_hat_h.conj().T
        U_approx = Q @ U_hat
        r = energy_rank(S_hat, E_target)
        if r is not None:
            return LowRank(U_approx[:, :r], S_hat[:r], V_hat[:, :r], k_est=r,
                           iters=it + 1, met=True, last_d=d, sigma_hat=S_hat)
        k0 = 2 * k0
    return LowRank(U_approx[:, :d], S_hat[:d], V_hat[:, :d], k_est=d, iters=i_max,
                   met=False, last_d=d, sigma_hat=S_hat)
