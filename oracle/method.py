"""Per-snapshot driver: Algorithm 2 (Section V) over a trajectory (oracle, FP64).

For each snapshot t with channel H_t:
  * if no inverse exists yet, invert A_t = H_t H_t^H + alpha I directly;
  * otherwise form dA = A_t - A_{t-1} (eq. 9), approximate it with Algorithm 1 (or with the
    exact truncated SVD of eqs. 13-14), and apply the Woodbury update of eq. 12 when
    k_est / K <= switch_ratio (0.5 in the paper), else invert A_t directly;
  * precode W = H_t^H X, scale to ||W||_F^2 = P_t (eq. 5) and score eq. 15.

Readings taken where the paper leaves a choice open:
  * A periodic direct re-inversion every `reinverse_period` snapshots (0 = never) bounds the
    drift of the chained Woodbury updates; the paper re-inverts only on the rank test.
  * The working rank is capped by r_max: I_max defaults to ceil(log2(r_max / k_init)) + 1
    so the last k0 reaches r_max, and any k_est > r_max takes the direct-inverse branch like
    k_est / K > switch_ratio does.  Algorithm 1's fall-through (target not met after I_max
    iterations) returns k_est = d as printed, which then meets the same test.
  * ||dA||_F <= dg_floor_rel * ||A_t||_F skips the update (r = 0, X kept): with dA = 0 the
    energy rule would pick one zero singular value and Sigma_r^{-1} would not exist.
  * The SINR always uses the true H_t, whatever inverse the precoder was built from.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import lowrank, philox, rzf, woodbury

# Branch codes of one snapshot (the CUDA library reports the same numbers).
KEEP = 0        # dA below the floor: X unchanged
WOODBURY = 1    # rank-r Woodbury update
INIT = 2        # no inverse yet: direct inversion
PERIODIC = 3    # periodic direct re-inversion
RANK = 4        # k_est too large for the switch test or the rank cap: direct inversion
FULL = 5        # conventional method: direct inversion at every snapshot


def default_i_max(k_init: int, r_max: int) -> int:
    return max(1, int(math.ceil(math.log2(max(r_max, k_init) / k_init))) + 1)


@dataclass
class RankRule:
    eta: float = 0.9
    k_init: int = 2
    p: int = 1
    i_max: int = 0                 # 0 -> default_i_max(k_init, r_max)
    r_max: int = 0                 # 0 -> K
    switch_ratio: float = 0.5
    reinverse_period: int = 20     # 0 -> never
    seed: int = 0
    dg_floor_rel: float = 0.0

    def resolved(self, K: int) -> "RankRule":
        r_max = self.r_max if self.r_max > 0 else K
        i_max = self.i_max if self.i_max > 0 else default_i_max(self.k_init, r_max)
        return RankRule(self.eta, self.k_init, self.p, i_max, r_max, self.switch_ratio,
                        self.reinverse_period, self.seed, self.dg_floor_rel)


@dataclass
class StepResult:
    t: int
    branch: int
    r: int
    iters: int
    d: int
    X: np.ndarray
    W: np.ndarray
    scale: float
    sinr: np.ndarray
    sum_rate: float
    dA_fro2: float = 0.0
    lowrank_product: np.ndarray | None = None
    sigma_hat: np.ndarray | None = None


@dataclass
class WBState:
    A_prev: np.ndarray | None = None
    X: np.ndarray | None = None
    t: int = 0
    history: list = field(default_factory=list)


def _finish(t, branch, r, iters, d, H, X, P_t, sigma2, dA_fro2=0.0, prod=None, sig=None):
    W, s = rzf.power_normalise(rzf.rzf_unnormalised(H, X), P_t)
    R, sn = rzf.sum_rate(H, W, sigma2)
    return StepResult(t, branch, r, iters, d, X, W, s, sn, R, dA_fro2, prod, sig)


def step_full(H: np.ndarray, alpha: float, P_t: float, sigma2, t: int = 0) -> StepResult:
    """Conventional full-inversion RZF for one snapshot."""
    H = np.asarray(H, dtype=np.complex128)
    X = rzf.inverse_gauss_jordan(rzf.gram(H, alpha))
    return _finish(t, FULL, 0, 0, 0, H, X, P_t, sigma2)


def step_wb(state: WBState, H: np.ndarray, alpha: float, rule: RankRule, P_t: float, sigma2,
            *, lowrank_mode: str = "arsvd", instance: int = 0) -> StepResult:
    """One snapshot of Algorithm 2; `lowrank_mode` is "arsvd" (Algorithm 1 with the Philox
    test matrices) or "exact" (truncated SVD)."""
    H = np.asarray(H, dtype=np.complex128)
    K = H.shape[0]
    rr = rule.resolved(K)
    t = state.t
    A = rzf.gram(H, alpha)
    if state.X is None:
        res = _finish(t, INIT, 0, 0, 0, H, rzf.inverse_gauss_jordan(A), P_t, sigma2)
    elif rr.reinverse_period > 0 and t % rr.reinverse_period == 0:
        res = _finish(t, PERIODIC, 0, 0, 0, H, rzf.inverse_gauss_jordan(A), P_t, sigma2)
    else:
        dA = A - state.A_prev
        dA_fro2 = float(np.sum(np.abs(dA) ** 2))
        if math.sqrt(dA_fro2) <= rr.dg_floor_rel * float(np.linalg.norm(A)):
            res = _finish(t, KEEP, 0, 0, 0, H, state.X, P_t, sigma2, dA_fro2)
        else:
            if lowrank_mode == "exact":
                lr = lowrank.truncated_svd(dA, rr.eta)
            elif lowrank_mode == "arsvd":
                def draw(it, d):
                    return philox.omega(K, d, seed=rr.seed, step=t, instance=instance, it=it)
                lr = lowrank.arsvd(dA, rr.eta, rr.k_init, rr.p, rr.i_max, draw)
            else:
                raise ValueError(lowrank_mode)
            if lr.k_est > rr.r_max or lr.k_est / K > rr.switch_ratio:
                X = rzf.inverse_gauss_jordan(A)
                res = _finish(t, RANK, lr.k_est, lr.iters, lr.last_d, H, X, P_t, sigma2,
                              dA_fro2, lr.product(), lr.sigma_hat)
            else:
                X = woodbury.woodbury_update(state.X, lr.U, lr.S, lr.V)
                res = _finish(t, WOODBURY, lr.k_est, lr.iters, lr.last_d, H, X, P_t, sigma2,
                              dA_fro2, lr.product(), lr.sigma_hat)
    state.A_prev = A
    state.X = res.X
    state.t = t + 1
    return res


def run_trajectory(Hs, alpha: float, P_t: float, sigma2, *, method: str = "wb",
                   rule: RankRule | None = None, lowrank_mode: str = "arsvd",
                   instance: int = 0, t0: int = 0) -> list[StepResult]:
    """Run snapshots Hs[0], Hs[1], ... of one trajectory (`method`: "wb" or "full")."""
    out = []
    if method == "full":
        for s, H in enumerate(Hs):
            out.append(step_full(H, alpha, P_t, sigma2, t=t0 + s))
        return out
    state = WBState(t=t0)
    for H in Hs:
        out.append(step_wb(state, H, alpha, rule or RankRule(), P_t, sigma2,
                           lowrank_mode=lowrank_mode, instance=instance))
    return out
