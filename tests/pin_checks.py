"""Checks that pin the FP64 oracle to facts outside itself.

Each check returns an error measure (0 = exact agreement); the pin tests assert these are at
rounding level, and the mutation tests assert that a planted mistake in the oracle makes at
least one of them large.  Nothing here reuses the oracle's own library calls to verify it:
the references are closed forms, brute-force sums, independent numpy.linalg routines that the
oracle does not call for that step, and algebraic identities of the paper's equations.
"""
from __future__ import annotations

import numpy as np

from oracle import lowrank, rzf, woodbury


def rng_complex(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)


def gram_bruteforce_err(seed=0, K=3, N=4, alpha=0.7):
    """eq. 5: A[k, l] = sum_n H[k, n] conj(H[l, n]) + alpha [k == l], by explicit loops."""
    rng = np.random.default_rng(seed)
    H = rng_complex(rng, K, N)
    A = rzf.gram(H, alpha)
    ref = np.zeros((K, K), dtype=np.complex128)
    for k in range(K):
        for l in range(K):
            s = 0j
            for n in range(N):
                s += H[k, n] * np.conj(H[l, n])
            ref[k, l] = s + (alpha if k == l else 0.0)
    return float(np.max(np.abs(A - ref)))


def inverse_2x2_err(inv=None):
    """Closed form [[a, b], [c, d]]^-1 = [[d, -b], [-c, a]] / (ad - bc)."""
    inv = inv or rzf.inverse_gauss_jordan
    a, b, c, d = 1.5 + 0.5j, -0.25 + 2j, 0.75 - 1j, 2.0 + 0.1j
    M = np.array([[a, b], [c, d]])
    ref = np.array([[d, -b], [-c, a]]) / (a * d - b * c)
    return float(np.max(np.abs(inv(M) - ref)))


def inverse_vs_numpy_err(seed=1, K=7, inv=None, hpd=False):
    inv = inv or rzf.inverse_gauss_jordan
    rng = np.random.default_rng(seed)
    M = rng_complex(rng, K, K)
    if hpd:
        M = M @ M.conj().T + 0.5 * np.eye(K)
    elif K > 1:
        M[0, 0] = 0.0   # forces a row exchange in the first column
    ref = np.linalg.inv(M)
    return float(np.linalg.norm(inv(M) - ref) / np.linalg.norm(ref))


def rzf_identity_err(seed=2, K=4, N=9, alpha=0.3):
    """H (H^H A^-1) = (A - alpha I) A^-1 = I - alpha A^-1, since H H^H = A - alpha I."""
    rng = np.random.default_rng(seed)
    H = rng_complex(rng, K, N)
    A = rzf.gram(H, alpha)
    X = np.linalg.inv(A)
    F = rzf.rzf_unnormalised(H, X)
    lhs = rzf.received_gains(H, F)
    return float(np.max(np.abs(lhs - (np.eye(K) - alpha * X))))


def rzf_norm_identity_err(seed=3, K=5, N=8, alpha=0.9):
    """||H^H A^-1||_F^2 = tr(A^-1) - alpha ||A^-1||_F^2."""
    rng = np.random.default_rng(seed)
    H = rng_complex(rng, K, N)
    A = rzf.gram(H, alpha)
    X = np.linalg.inv(A)
    F = rzf.rzf_unnormalised(H, X)
    lhs = np.linalg.norm(F) ** 2
    rhs = np.trace(X).real - alpha * np.linalg.norm(X) ** 2
    return float(abs(lhs - rhs) / abs(rhs))


def single_user_rate_err(seed=4, N=6, P_t=2.0, sigma2=0.3):
    """K = 1: R = log2(1 + P_t ||h||^2 / sigma^2) for every alpha (no interference)."""
    rng = np.random.default_rng(seed)
    h = rng_complex(rng, 1, N)
    ref = np.log2(1.0 + P_t * np.linalg.norm(h) ** 2 / sigma2)
    errs = []
    for alpha in (0.0, 0.1, 10.0):
        out = rzf.full_inversion_rzf(h, alpha, P_t, sigma2)
        errs.append(abs(out["sum_rate"] - ref))
    return float(max(errs))


def sum_rate_worked_err():
    """Worked example of eq. 15.  H = [[1, 0], [0, 2]], W = [[1, 0.5], [0, 1]]:
    gains HW = [[1, 0.5], [0, 2]]; with sigma^2 = 0.25:
    SINR_1 = 1 / (0.25 + 0.25) = 2, SINR_2 = 4 / (0 + 0.25) = 16,
    R = log2(3) + log2(17)."""
    H = np.array([[1.0, 0.0], [0.0, 2.0]], dtype=np.complex128)
    W = np.array([[1.0, 0.5], [0.0, 1.0]], dtype=np.complex128)
    R, s = rzf.sum_rate(H, W, 0.25)
    return float(max(abs(R - (np.log2(3.0) + np.log2(17.0))), abs(s[0] - 2.0), abs(s[1] - 16.0)))


def zf_limit_interference(seed=5, K=3, N=6):
    """alpha -> 0 with K <= N: RZF becomes zero forcing, inter-user gains vanish."""
    rng = np.random.default_rng(seed)
    H = rng_complex(rng, K, N)
    out = rzf.full_inversion_rzf(H, 1e-12, 1.0, 1.0)
    g = rzf.received_gains(H, out["W"])
    off = g - np.diag(np.diag(g))
    return float(np.max(np.abs(off)) / np.max(np.abs(np.diag(g))))


def mrt_limit_err(seed=6, K=3, N=5):
    """alpha -> infinity: A^-1 -> I / alpha, so the normalised precoder tends to H^H."""
    rng = np.random.default_rng(seed)
    H = rng_complex(rng, K, N)
    out = rzf.full_inversion_rzf(H, 1e9, 1.0, 1.0)
    ref = H.conj().T / np.linalg.norm(H)
    return float(np.max(np.abs(out["W"] - ref)))


def energy_rank_bruteforce_err():
    """eq. 14 by hand: sigma^2 = (4, 3, 2, 1), total 10."""
    sig = np.sqrt(np.array([4.0, 3.0, 2.0, 1.0]))
    cases = [(0.4, 1), (0.7, 2), (0.71, 3), (0.9, 3), (0.91, 4), (1.0, 4)]
    bad = 0
    for eta, r in cases:
        if lowrank.energy_rank(sig, eta * 10.0) != r:
            bad += 1
    if lowrank.energy_rank(sig, 10.5) is not None:
        bad += 1
    return float(bad)


def low_rank_perturbation(seed=7, K=6, N=10, alpha=0.5, row=2):
    """A and A' differing by one user's channel row: rank(A' - A) <= 2."""
    rng = np.random.default_rng(seed)
    H = rng_complex(rng, K, N)
    H2 = H.copy()
    H2[row] += 0.3 * rng_complex(rng, N)
    return rzf.gram(H, alpha), rzf.gram(H2, alpha)


def woodbury_exact_err(seed=7):
    """eq. 12 is exact when Sigma_r carries all of dA: compare with numpy.linalg.inv(A')."""
    A, A2 = low_rank_perturbation(seed)
    dA = A2 - A
    U, S, Vh = np.linalg.svd(dA)
    r = int(np.sum(S > 1e-12 * S[0]))
    X2 = woodbury.woodbury_update(np.linalg.inv(A), U[:, :r], S[:r], Vh[:r].conj().T)
    ref = np.linalg.inv(A2)
    return float(np.linalg.norm(X2 - ref) / np.linalg.norm(ref)), r


def sherman_morrison_err(seed=8, K=5):
    """r = 1: (A + u v^H)^-1 = X - X u v^H X / (1 + v^H X u) (closed form), with a
    non-Hermitian rank-one term so U and V differ."""
    rng = np.random.default_rng(seed)
    M = rng_complex(rng, K, K)
    A = M @ M.conj().T + np.eye(K)
    u = rng_complex(rng, K)
    v = rng_complex(rng, K)
    X = np.linalg.inv(A)
    ref = X - np.outer(X @ u, v.conj() @ X) / (1.0 + v.conj() @ X @ u)
    nu, nv = np.linalg.norm(u), np.linalg.norm(v)
    got = woodbury.woodbury_update(X, (u / nu)[:, None], np.array([nu * nv]), (v / nv)[:, None])
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def arsvd_full_width_err(seed=9, K=6, eta=0.8):
    """d = K: Q spans C^K, so B has the singular values of dA and Algorithm 1 returns the
    truncated SVD of eq. 14 (same r, same U_r Sigma_r V_r^H).  Reference: numpy.linalg.svd
    of dA, which the arSVD path never computes."""
    rng = np.random.default_rng(seed)
    M = rng_complex(rng, K, K)
    dA = M + M.conj().T
    U, S, Vh = np.linalg.svd(dA)
    r_ref = int(np.searchsorted(np.cumsum(S ** 2), eta * np.sum(S ** 2) * (1 - 1e-15)) + 1)
    ref = (U[:, :r_ref] * S[:r_ref]) @ Vh[:r_ref]
    lr = lowrank.arsvd(dA, eta, k_init=K, p=0, i_max=1,
                       draw_omega=lambda it, d: rng_complex(np.random.default_rng(it + 50), K, d))
    return float(np.linalg.norm(lr.product() - ref) / np.linalg.norm(ref)), lr.k_est, r_ref


def arsvd_exact_rank_err(seed=10, K=12, s=3):
    """dA of exact rank s and sketch width d >= s: eta = 1 recovers dA exactly."""
    rng = np.random.default_rng(seed)
    L = rng_complex(rng, K, s)
    dA = L @ np.diag([3.0, -2.0, 0.5]) @ L.conj().T
    lr = lowrank.arsvd(dA, 1.0 - 1e-12, k_init=2, p=2, i_max=3,
                       draw_omega=lambda it, d: rng_complex(np.random.default_rng(100 + it), K, d))
    return float(np.linalg.norm(lr.product() - dA) / np.linalg.norm(dA)), lr.k_est
