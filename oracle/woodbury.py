"""Woodbury inverse update, written exactly as eq. 12 (Section III) (oracle, FP64).

(A + U_r Sigma_r V_r^H)^{-1} = A^{-1} - A^{-1} U_r (Sigma_r^{-1} + V_r^H A^{-1} U_r)^{-1} V_r^H A^{-1},

valid when A and the r x r capacitance matrix Sigma_r^{-1} + V_r^H A^{-1} U_r are nonsingular.
The r x r inverse uses the oracle's own Gauss-Jordan elimination.
"""
from __future__ import annotations

import numpy as np

from .rzf import inverse_gauss_jordan


def woodbury_update(X: np.ndarray, U: np.ndarray, S: np.ndarray, V: np.ndarray) -> np.ndarray:
    """Return (A + U diag(S) V^H)^{-1} given X = A^{-1} (eq. 12)."""
    X = np.asarray(X, dtype=np.complex128)
    U = np.asarray(U, dtype=np.complex128)
    V = np.asarray(V, dtype=np.complex128)
    S = np.asarray(S, dtype=np.float64)
    if U.shape[1] == 0:
        return X.copy()
    XU = X @ U                                   # step 1: A^{-1} U_r
    C = np.diag(1.0 / S) + V.conj().T @ XU       # step 2: Sigma_r^{-1} + V_r^H A^{-1} U_r
    Cinv = inverse_gauss_jordan(C)               # step 3: r x r inverse
    VhX = V.conj().T @ X
    return X - XU @ Cinv @ VhX                   # steps 4-5
