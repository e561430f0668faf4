"""Planted mistakes: each mutation swaps one oracle function for a plausible wrong variant
(a dropped term, a wrong sign or index, a transposed operand) and checks that at least one
pin from pin_checks no longer holds.  All on the CPU; the oracle is restored afterwards."""
import numpy as np
import pytest

import pin_checks as pc
from oracle import lowrank, philox, rzf, woodbury


def _all_pins():
    """Evaluate every pin; return the list of (name, ok)."""
    res = []

    def chk(name, fn, ok):
        try:
            v = fn()
            res.append((name, bool(ok(v))))
        except Exception:
            res.append((name, False))
    chk("gram", pc.gram_bruteforce_err, lambda v: v < 1e-12)
    chk("inv2x2", pc.inverse_2x2_err, lambda v: v < 1e-12)
    chk("inv_np", pc.inverse_vs_numpy_err, lambda v: v < 1e-10)
    chk("rzf_id", pc.rzf_identity_err, lambda v: v < 1e-10)
    chk("rzf_norm", pc.rzf_norm_identity_err, lambda v: v < 1e-10)
    chk("k1_rate", pc.single_user_rate_err, lambda v: v < 1e-10)
    chk("worked", pc.sum_rate_worked_err, lambda v: v < 1e-12)
    chk("zf", pc.zf_limit_interference, lambda v: v < 1e-8)
    chk("mrt", pc.mrt_limit_err, lambda v: v < 1e-6)
    chk("energy", pc.energy_rank_bruteforce_err, lambda v: v == 0)
    chk("wb_exact", pc.woodbury_exact_err, lambda v: v[0] < 1e-10 and v[1] == 2)
    chk("sherman", pc.sherman_morrison_err, lambda v: v < 1e-10)
    chk("arsvd_full", pc.arsvd_full_width_err, lambda v: v[0] < 1e-10 and v[1] == v[2])
    chk("arsvd_rank", pc.arsvd_exact_rank_err, lambda v: v[0] < 1e-10 and v[1] == 3)
    chk("philox", lambda: [int(x) for x in philox.philox4x32_10([0, 0, 0, 0], [0, 0])],
        lambda v: v == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8])
    return res


def test_unmutated_oracle_passes_every_pin():
    bad = [n for n, ok in _all_pins() if not ok]
    assert bad == []


def _gram_no_conj(H, alpha):
    H = np.asarray(H, dtype=np.complex128)
    return H @ H.T + alpha * np.eye(H.shape[0])


def _gram_transposed(H, alpha):
    H = np.asarray(H, dtype=np.complex128)
    return np.conj(H) @ H.T + alpha * np.eye(H.shape[0])


def _gram_no_alpha(H, alpha):
    H = np.asarray(H, dtype=np.complex128)
    return H @ H.conj().T


def _gj_no_pivot(A):
    A = np.asarray(A, dtype=np.complex128)
    K = A.shape[0]
    M = np.concatenate([A.copy(), np.eye(K, dtype=np.complex128)], axis=1)
    for c in range(K):
        M[c] = M[c] / M[c, c]
        for r in range(K):
            if r != c:
                M[r] = M[r] - M[r, c] * M[c]
    return M[:, K:]


def _wb_no_sigma_inv(X, U, S, V):
    XU = X @ U
    C = V.conj().T @ XU
    return X - XU @ np.linalg.inv(C) @ (V.conj().T @ X)


def _wb_plus_sign(X, U, S, V):
    XU = X @ U
    C = np.diag(1.0 / S) + V.conj().T @ XU
    return X + XU @ np.linalg.inv(C) @ (V.conj().T @ X)


def _wb_u_for_v(X, U, S, V):
    XU = X @ U
    C = np.diag(1.0 / S) + U.conj().T @ XU
    return X - XU @ np.linalg.inv(C) @ (U.conj().T @ X)


def _gains_transposed(H, W):
    return (np.asarray(H) @ np.asarray(W)).T


def _power_no_sqrt(F, P_t):
    s = P_t / np.linalg.norm(F)
    return s * F, float(s)


def _energy_off_by_one(sigma, E_target):
    r = _orig_energy_rank(sigma, E_target)
    return None if r is None else r + 1


_orig_energy_rank = lowrank.energy_rank


def _arsvd_sketch_dropped(dA, eta, k_init, p, i_max, draw_omega):
    """Algorithm 1 with dA dropped from the sketch (Y = Omega instead of dA Omega)."""
    K = dA.shape[0]
    E_target = eta * float(np.sum(np.abs(dA) ** 2))
    k0 = k_init
    for it in range(i_max):
        d = min(k0 + p, K)
        Q, _ = np.linalg.qr(draw_omega(it, d), mode="reduced")
        B = Q.conj().T @ dA
        Uh, Sh, Vhh = np.linalg.svd(B, full_matrices=False)
        r = _orig_energy_rank(Sh, E_target)
        if r is not None:
            return lowrank.LowRank((Q @ Uh)[:, :r], Sh[:r], Vhh.conj().T[:, :r], r, it + 1)
        k0 *= 2
    return lowrank.LowRank(Q @ Uh, Sh, Vhh.conj().T, d, i_max, met=False)


def _philox_nine_rounds(ctr, key):
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    m = np.uint64(0xFFFFFFFF)
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    for rnd in range(9):
        if rnd:
            k0, k1 = (k0 + np.uint64(0x9E3779B9)) & m, (k1 + np.uint64(0xBB67AE85)) & m
        p0 = c0 * np.uint64(0xD2511F53)
        p1 = c2 * np.uint64(0xCD9E8D57)
        c0, c1, c2, c3 = (p1 >> np.uint64(32)) ^ c1 ^ k0, p1 & m, (p0 >> np.uint64(32)) ^ c3 ^ k1, p0 & m
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


MUTATIONS = [
    ("gram: conjugate dropped", rzf, "gram", _gram_no_conj),
    ("gram: transposed operand", rzf, "gram", _gram_transposed),
    ("gram: alpha I dropped", rzf, "gram", _gram_no_alpha),
    ("inverse: no pivoting", rzf, "inverse_gauss_jordan", _gj_no_pivot),
    ("woodbury: Sigma^-1 dropped", woodbury, "woodbury_update", _wb_no_sigma_inv),
    ("woodbury: wrong sign", woodbury, "woodbury_update", _wb_plus_sign),
    ("woodbury: U used for V", woodbury, "woodbury_update", _wb_u_for_v),
    ("sinr: columns for rows", rzf, "received_gains", _gains_transposed),
    ("power: P_t for sqrt(P_t)", rzf, "power_normalise", _power_no_sqrt),
    ("energy rule: off by one", lowrank, "energy_rank", _energy_off_by_one),
    ("arsvd: sketch of Omega alone", lowrank, "arsvd", _arsvd_sketch_dropped),
    ("philox: nine rounds", philox, "philox4x32_10", _philox_nine_rounds),
]


@pytest.mark.parametrize("name,mod,attr,bad", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, name, mod, attr, bad):
    monkeypatch.setattr(mod, attr, bad)
    failing = [n for n, ok in _all_pins() if not ok]
    assert failing, f"no pin caught the planted mistake '{name}'"
