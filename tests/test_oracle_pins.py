"""Pins of the FP64 oracle (CPU only).

The oracle is only trusted because these tests tie it to facts outside itself: published
known-answer vectors, closed forms, brute-force sums, independent library routines it does
not call, and invariants of the paper's equations (Sections II-V, Algorithms 1-2).
"""
import math
import os

import numpy as np
import pytest

import pin_checks as pc
from oracle import cost, lowrank, method, philox, rzf, woodbury

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


# ---------------------------------------------------------------- Philox / Omega (Alg. 1)
def test_philox_known_answers():
    for row in _rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = philox.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_box_muller_exact_map():
    xa, xb = np.uint32(0x80000000), np.uint32(0x40000000)
    ua = ((0x80000000 >> 9) + 0.5) / 2 ** 23
    ub = ((0x40000000 >> 9) + 0.5) / 2 ** 23
    z = philox.box_muller(np.array([xa]), np.array([xb]))[0]
    assert abs(abs(z) ** 2 + math.log(ua)) < 1e-15
    assert abs(np.angle(z) % (2 * math.pi) - 2 * math.pi * ub) < 1e-12


def test_omega_is_circular_standard_gaussian():
    Om = philox.omega(2000, 64, seed=123, step=3, instance=1, it=0).ravel()
    assert abs(Om.mean()) < 0.01
    assert abs(np.mean(np.abs(Om) ** 2) - 1.0) < 0.01           # E|w|^2 = 1
    assert abs(np.mean(Om ** 2)) < 0.01                           # circular: E w^2 = 0
    assert abs(np.mean(Om.real ** 2) - 0.5) < 0.01                # Re ~ N(0, 1/2)
    assert abs(np.mean(Om.real * Om.imag)) < 0.01


def test_omega_counter_layout():
    a = philox.omega(5, 7, seed=9, step=4, instance=2, it=1)
    b = philox.omega(5, 3, seed=9, step=4, instance=2, it=1)
    np.testing.assert_array_equal(a[:, :3], b)                    # entries do not depend on d
    for kw in ({"step": 5}, {"instance": 3}, {"it": 2}, {"seed": 10}):
        args = dict(seed=9, step=4, instance=2, it=1)
        args.update(kw)
        assert not np.allclose(philox.omega(5, 7, **args), a)
    # entry (i, j) uses counter (i, j // 2, t, 16 b + it), words (x0, x1) for even j
    x = philox.philox4x32_10([3, 2, 4, 16 * 2 + 1], [9, 0])
    assert a[3, 4] == philox.box_muller(x[None, 0], x[None, 1])[0]
    assert a[3, 5] == philox.box_muller(x[None, 2], x[None, 3])[0]


# ---------------------------------------------------------------- Gram, inverses, RZF (eq. 5)
def test_gram_bruteforce():
    assert pc.gram_bruteforce_err() < 1e-14


def test_inverse_closed_form_2x2():
    assert pc.inverse_2x2_err(rzf.inverse_gauss_jordan) < 1e-14
    # Hermitian positive definite [[a, b], [conj(b), d]]^-1 = [[d, -b], [-conj(b), a]] / det
    a, b, d = 2.0, 0.5 - 0.75j, 3.0
    M = np.array([[a, b], [np.conj(b), d]])
    ref = np.array([[d, -b], [-np.conj(b), a]]) / (a * d - abs(b) ** 2)
    assert np.max(np.abs(rzf.inverse_cholesky(M) - ref)) < 1e-14


def test_inverse_vs_independent_library():
    assert pc.inverse_vs_numpy_err(K=7) < 1e-12
    assert pc.inverse_vs_numpy_err(K=7, inv=rzf.inverse_cholesky, hpd=True) < 1e-12
    assert pc.inverse_vs_numpy_err(K=1) < 1e-14


def test_inverse_times_matrix_is_identity():
    rng = np.random.default_rng(11)
    H = pc.rng_complex(rng, 8, 64)
    A = rzf.gram(H, 0.8)
    for inv in (rzf.inverse_gauss_jordan, rzf.inverse_cholesky):
        assert np.max(np.abs(inv(A) @ A - np.eye(8))) < 1e-12


def test_singular_and_indefinite_raise():
    with pytest.raises(np.linalg.LinAlgError):
        rzf.inverse_gauss_jordan(np.zeros((3, 3)))
    with pytest.raises(np.linalg.LinAlgError):
        rzf.cholesky_lower(np.diag([1.0, -1.0]).astype(complex))


def test_rzf_identities():
    assert pc.rzf_identity_err() < 1e-12
    assert pc.rzf_norm_identity_err() < 1e-12


def test_power_constraint():
    rng = np.random.default_rng(12)
    H = pc.rng_complex(rng, 4, 16)
    out = rzf.full_inversion_rzf(H, 0.4, 3.0, 0.1)
    assert abs(np.linalg.norm(out["W"]) ** 2 - 3.0) < 1e-12


def test_single_user_rate_closed_form():
    assert pc.single_user_rate_err() < 1e-12


def test_sum_rate_worked_example():
    assert pc.sum_rate_worked_err() < 1e-14


def test_zero_forcing_limit():
    assert pc.zf_limit_interference() < 1e-9


def test_mrt_limit():
    assert pc.mrt_limit_err() < 1e-7


# ---------------------------------------------------------------- energy rule, SVDs (eqs. 13-14)
def test_energy_rank_bruteforce():
    assert pc.energy_rank_bruteforce_err() == 0.0


def test_truncated_svd_of_diagonal():
    dA = np.diag([0.5, -3.0, 1.0, 2.0]).astype(complex)
    # sigma^2 = 9, 4, 1, .25 (total 14.25); cumulative 9, 13, 14, 14.25
    lr = lowrank.truncated_svd(dA, 0.9)        # target 12.825: 13 >= 12.825 -> r = 2
    assert lr.k_est == 2
    assert np.max(np.abs(lr.product() - np.diag([0.0, -3.0, 0.0, 2.0]))) < 1e-14
    lr = lowrank.truncated_svd(dA, 0.92)       # target 13.11: 14 >= 13.11 > 13 -> r = 3
    assert lr.k_est == 3
    assert np.max(np.abs(lr.product() - np.diag([0.0, -3.0, 1.0, 2.0]))) < 1e-14


def test_arsvd_full_width_is_truncated_svd():
    err, k, kref = pc.arsvd_full_width_err()
    assert k == kref and err < 1e-12


def test_arsvd_exact_rank_recovery():
    err, k = pc.arsvd_exact_rank_err()
    assert k == 3 and err < 1e-12


def test_arsvd_doubling_schedule_and_fallthrough():
    K = 16
    dA = np.eye(K, dtype=complex)               # flat spectrum: only d = K meets eta = 0.9
    draws = []

    def draw(it, d):
        draws.append(d)
        return pc.rng_complex(np.random.default_rng(it), K, d)
    lr = lowrank.arsvd(dA, 0.9, k_init=2, p=1, i_max=4, draw_omega=draw)
    assert draws == [3, 5, 9, 16]               # d = min(k0 + p, K), k0 = 2, 4, 8, 16
    assert lr.met and lr.iters == 4 and lr.k_est == 15   # ceil(0.9 * 16) = 15
    draws.clear()
    lr = lowrank.arsvd(dA, 0.9, k_init=2, p=1, i_max=3, draw_omega=draw)
    assert draws == [3, 5, 9] and not lr.met and lr.k_est == 9 and lr.U.shape == (K, 9)


def test_randomized_range_finder_error_bound():
    """Halko-Martinsson-Tropp (SIAM Rev. 2011, Thm. 10.5, cited by the paper in Section IV):
    E ||dA - Q Q^H dA||_F <= (1 + k / (p - 1))^{1/2} (sum_{j > k} sigma_j^2)^{1/2} for p >= 2.
    With eta = 1 the target is unreachable, so Algorithm 1 falls through and returns all d
    components, whose product is exactly Q Q^H dA."""
    K, k, p = 24, 4, 3
    rng = np.random.default_rng(13)
    U, _ = np.linalg.qr(pc.rng_complex(rng, K, K))
    sig = 0.7 ** np.arange(K)
    dA = (U * sig) @ U.conj().T
    tail = math.sqrt(np.sum(sig[k:] ** 2))
    bound = math.sqrt(1 + k / (p - 1)) * tail
    errs = []
    for s in range(200):
        lr = lowrank.arsvd(dA, 1.0, k_init=k, p=p, i_max=1,
                           draw_omega=lambda it, d, s=s: philox.omega(K, d, seed=s, step=0,
                                                                     instance=0, it=it))
        assert not lr.met and lr.k_est == k + p
        errs.append(np.linalg.norm(dA - lr.product()))
    assert np.mean(errs) <= bound
    assert min(errs) >= math.sqrt(np.sum(sig[k + p:] ** 2)) * (1 - 1e-9)  # Eckart-Young floor


# ---------------------------------------------------------------- Woodbury (eq. 12)
def test_woodbury_exact_for_exact_low_rank():
    err, r = pc.woodbury_exact_err()
    assert r == 2 and err < 1e-12


def test_woodbury_sherman_morrison():
    assert pc.sherman_morrison_err() < 1e-12


def test_woodbury_rank_zero_is_identity():
    X = np.eye(3, dtype=complex) * 2
    out = woodbury.woodbury_update(X, np.zeros((3, 0)), np.zeros(0), np.zeros((3, 0)))
    np.testing.assert_array_equal(out, X)


# ---------------------------------------------------------------- Algorithm 2 driver
def _traj(K=6, N=16, T=12, seed=14):
    rng = np.random.default_rng(seed)
    H0 = pc.rng_complex(rng, K, N)
    D = pc.rng_complex(rng, K, N)
    return [H0 + 0.01 * t * D + 0.002 * (t ** 2) * pc.rng_complex(rng, K, N) for t in range(T)]


def test_driver_full_matches_conventional():
    Hs = _traj()
    res = method.run_trajectory(Hs, 0.5, 1.0, 0.2, method="full")
    for H, r in zip(Hs, res):
        ref = rzf.full_inversion_rzf(H, 0.5, 1.0, 0.2)
        assert r.branch == method.FULL
        assert abs(r.sum_rate - ref["sum_rate"]) < 1e-12


@pytest.mark.parametrize("mode", ["exact", "arsvd"])
def test_driver_eta_one_tracks_true_inverse(mode):
    """With eta = 1 every Woodbury step (or rank fallback) reproduces A_t^-1."""
    Hs = _traj()
    rule = method.RankRule(eta=1.0 - 1e-13, k_init=2, p=2, reinverse_period=0, seed=3,
                           switch_ratio=1.0)
    res = method.run_trajectory(Hs, 0.5, 1.0, 0.2, method="wb", rule=rule, lowrank_mode=mode)
    for H, r in zip(Hs, res):
        A = rzf.gram(H, 0.5)
        assert np.max(np.abs(r.X @ A - np.eye(len(A)))) < 1e-9
    assert res[0].branch == method.INIT
    assert any(r.branch == method.WOODBURY for r in res[1:])


def test_driver_branches():
    Hs = _traj(T=8)
    Hs[3] = Hs[2].copy()                                    # unchanged channel -> dA = 0
    rule = method.RankRule(eta=0.9, k_init=2, p=1, reinverse_period=5, seed=1)
    res = method.run_trajectory(Hs, 0.5, 1.0, 0.2, method="wb", rule=rule)
    assert [r.branch for r in res][:6] == [method.INIT, res[1].branch, res[2].branch,
                                           method.KEEP, res[4].branch, method.PERIODIC]
    np.testing.assert_array_equal(res[3].X, res[2].X)
    rule0 = method.RankRule(eta=0.9, k_init=2, p=1, reinverse_period=0, switch_ratio=0.0)
    res0 = method.run_trajectory(Hs, 0.5, 1.0, 0.2, method="wb", rule=rule0)
    assert all(r.branch in (method.INIT, method.RANK, method.KEEP) for r in res0)
    for H, r in zip(Hs, res0):
        assert np.max(np.abs(r.X @ rzf.gram(H, 0.5) - np.eye(6))) < 1e-12


def test_default_i_max():
    assert method.default_i_max(2, 16) == 4      # k0 = 2, 4, 8, 16
    assert method.default_i_max(2, 64) == 6
    assert method.default_i_max(2, 8) == 3
    assert method.default_i_max(2, 2) == 1


# ---------------------------------------------------------------- cost models (Tables I-IV)
def test_cost_model_fig1_values():
    for K, r, v in _rows("cost_model_fig1.txt"):
        assert abs(cost.normalised_wb_cost(int(K), int(r)) - float(v)) < 5e-3


def test_savings_accounting():
    K = 16
    assert cost.savings(K, [5, 5], [0, 0]) == 0.0
    assert abs(cost.savings(K, [1, 1], [4, 4]) - (1 - cost.normalised_wb_cost(K, 4))) < 1e-15
    assert cost.savings(K, [0], [0]) == 1.0
