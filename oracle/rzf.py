"""Gram matrix, direct inverses, RZF precoder and sum-rate (oracle, FP64).

Section II, eq. 5:  F_BB = H^H (H H^H + alpha I_K)^{-1} = H^H A^{-1}, with alpha >= 0, and the
precoder scaled so that ||F_RF F_BB||_F^2 = P_t.  The arrays here are fully digital
(F_RF = I), so the constraint reads ||W||_F^2 = P_t.

Section VI, eq. 15:  R_sum = sum_n log2(1 + |g_nn|^2 / (sum_{i != n} |g_ni|^2 + sigma_n^2)),
where g_ni is the gain of user n's channel on precoder column i.  H = [h_1 ... h_K]^T (eq. 1)
stores user n's channel as row n, so g_ni = (H W)_{n i}; that is the reading under which
zero forcing (alpha -> 0) removes all inter-user interference.
"""
from __future__ import annotations

import numpy as np


def gram(H: np.ndarray, alpha: float) -> np.ndarray:
    """A = H H^H + alpha I_K (eq. 5)."""
    H = np.asarray(H, dtype=np.complex128)
    K = H.shape[0]
    return H @ H.conj().T + alpha * np.eye(K, dtype=np.complex128)


def inverse_gauss_jordan(A: np.ndarray) -> np.ndarray:
    """Direct inverse by Gauss-Jordan elimination with partial (row) pivoting.

    Reduces [A | I] to [I | A^{-1}] one pivot column at a time.  Raises
    numpy.linalg.LinAlgError on an exactly zero pivot column.
    """
    A = np.asarray(A, dtype=np.complex128)
    K = A.shape[0]
    M = np.concatenate([A.copy(), np.eye(K, dtype=np.complex128)], axis=1)
    for c in range(K):
        p = c + int(np.argmax(np.abs(M[c:, c])))
        if M[p, c] == 0:
            raise np.linalg.LinAlgError("singular matrix")
        if p != c:
            M[[c, p]] = M[[p, c]]
        M[c] = M[c] / M[c, c]
        for r in range(K):
            if r != c and M[r, c] != 0:
                M[r] = M[r] - M[r, c] * M[c]
    return M[:, K:]


def cholesky_lower(A: np.ndarray) -> np.ndarray:
    """Lower factor L with A = L L^H for Hermitian positive definite A (column by column)."""
    A = np.asarray(A, dtype=np.complex128)
    K = A.shape[0]
    L = np.zeros_like(A)
    for j in range(K):
        d = A[j, j].real - np.sum(np.abs(L[j, :j]) ** 2)
        if not d > 0:
            raise np.linalg.LinAlgError("matrix is not positive definite")
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, K):
            L[i, j] = (A[i, j] - np.sum(L[i, :j] * L[j, :j].conj())) / L[j, j]
    return L


def inverse_cholesky(A: np.ndarray) -> np.ndarray:
    """A^{-1} = L^{-H} L^{-1} from the Cholesky factor (forward substitution for L^{-1})."""
    L = cholesky_lower(A)
    K = L.shape[0]
    Linv = np.zeros_like(L)
    for j in range(K):               # column j of L^{-1}: solve L y = e_j
        y = np.zeros(K, dtype=np.complex128)
        y[j] = 1.0 / L[j, j]
        for i in range(j + 1, K):
            y[i] = -np.sum(L[i, j:i] * y[j:i]) / L[i, i]
        Linv[:, j] = y
    return Linv.conj().T @ Linv


def rzf_unnormalised(H: np.ndarray, X: np.ndarray) -> np.ndarray:
    """F_BB = H^H X with X standing for A^{-1} (eq. 5)."""
    return np.asarray(H, dtype=np.complex128).conj().T @ np.asarray(X, dtype=np.complex128)


def power_normalise(F: np.ndarray, P_t: float) -> tuple[np.ndarray, float]:
    """Scale F so that ||F||_F^2 = P_t; returns (scaled F, scale)."""
    nrm = np.linalg.norm(F)
    if nrm == 0:
        raise ValueError("zero precoder cannot be normalised")
    s = np.sqrt(P_t) / nrm
    return s * F, float(s)


def received_gains(H: np.ndarray, W: np.ndarray) -> np.ndarray:
    """g[n, i] = (H W)_{n i}: user n's channel (row n of H) on precoder column i."""
    return np.asarray(H, dtype=np.complex128) @ np.asarray(W, dtype=np.complex128)


def sinr(H: np.ndarray, W: np.ndarray, sigma2) -> np.ndarray:
    """Per-user SINR of eq. 15 (sigma2: scalar or per-user array)."""
    g = received_gains(H, W)
    p = np.abs(g) ** 2
    sig = np.diag(p)
    interference = p.sum(axis=1) - sig
    return sig / (interference + np.broadcast_to(np.asarray(sigma2, dtype=np.float64), sig.shape))


def sum_rate(H: np.ndarray, W: np.ndarray, sigma2) -> tuple[float, np.ndarray]:
    """R_sum = sum_n log2(1 + SINR_n) (eq. 15); returns (R_sum, SINR vector)."""
    s = sinr(H, W, sigma2)
    return float(np.sum(np.log2(1.0 + s))), s


def full_inversion_rzf(H: np.ndarray, alpha: float, P_t: float, sigma2):
    """The conventional method: invert A directly, precode, normalise, score."""
    A = gram(H, alpha)
    X = inverse_gauss_jordan(A)
    W, s = power_normalise(rzf_unnormalised(H, X), P_t)
    R, sn = sum_rate(H, W, sigma2)
    return {"A": A, "X": X, "W": W, "scale": s, "sum_rate": R, "sinr": sn}
