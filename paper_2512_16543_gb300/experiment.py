"""Paper-style study of Section VI (Fig. 2, Table V) run on this library.

Setting (Table III, with the readings of the design notes): 18 GHz, 600 km, 16x16 UPA at
lambda/2, hybrid beamforming with N_RF = K = 16 beams (one DFT beam per user, best-power
selection re-made at every update, Section II eq. 4), users one per beam cell, K_R = 10 dB,
digital precoder updated every 50 ms over a 120 s pass (2400 updates), p = 1, k_init = 2,
Monte Carlo over independent trajectories (the batch).  The digital precoder is computed from
the geometric effective channel H_eff = A F_RF (the satellite knows positions, Section II) by
the library -- conventional RZF (a direct inverse every update) and the proposed method at each
eta -- and the sum-rate of eq. 15 is evaluated with the Rician channel seen through the same
beams, H F_RF, with the power constraint ||F_RF F_BB||_F^2 = P_t.  Algorithm 2 runs as printed
(no periodic re-inversion) unless a period is given.

Reported per eta: the computational savings of Table V from the Table I / IV cost model with
the ranks the library's Algorithm 1 chose (a direct inverse counts K^3), the mean sum-rate
degradation against conventional RZF, and quantiles of the sum-rate ECDF (Fig. 2).  The
paper's absolute link budget (P_t = 20 dBW, UT gain, noise) is replaced by an SNR parameter
(alpha = K / SNR), so sum-rates are not comparable in absolute value with the paper's; the
degradation is, and it depends on alpha: the rank-r update leaves the (1 - eta) part of dG out
of X, an error that ||G^-1||^2 <= 1 / alpha^2 amplifies and that accumulates while no direct
inverse intervenes.
"""
from __future__ import annotations

import math

import torch

from . import binding, channel

PAPER_TABLE5 = {0.9: (30.6, 1.6), 0.8: (47.7, 5.8), 0.65: (61.2, 9.5)}  # savings %, SR loss %


def op_count(K: int, r: int, direct: bool) -> float:
    """Operations of one update in the paper's cost model: a direct inverse K^3 (Table I), the
    proposed method K^2 + K^2 r + r^3 + r^2 K (Table IV)."""
    if direct:
        return float(K) ** 3
    return float(K * K + K * K * r + r ** 3 + r * r * K)


def true_sum_rate(Ht: torch.Tensor, F: torch.Tensor, W: torch.Tensor, p_t: float,
                  sigma2: float) -> torch.Tensor:
    """Sum-rate of eq. 15 for digital precoders W [B, N_RF, K] through beams F [B, N, N_RF] on
    the channel Ht = H F [B, K, N_RF], after scaling to ||F W||_F^2 = P_t."""
    W = W.to(torch.complex128)
    scale = math.sqrt(p_t) / torch.linalg.matrix_norm(F @ W)
    g = (Ht @ W) * scale[:, None, None]                       # gains (H F W)_{n i}
    p = g.abs() ** 2
    sig = torch.diagonal(p, dim1=-2, dim2=-1)
    intf = p.sum(-1) - sig
    return torch.log2(1.0 + sig / (intf + sigma2)).sum(-1)


def run(batch: int = 100, steps: int = 2400, etas=(0.9, 0.8, 0.65), seed: int = 2025,
        device="cuda", precision: str = "c64", snr_db: float = 10.0,
        reinverse_period: int = 0, per_snapshot: bool = False) -> dict:
    """reinverse_period: 0 = Algorithm 2 as printed (a direct inverse only on the rank test).
    per_snapshot: also return "sum_rates", per method (in the table's order) the sum-rate of
    every snapshot and run, a [steps, batch] nested list (snapshot 0 is the initial direct
    inverse), with "t0", the time index of snapshot 0."""
    sc = channel.scenario_paper_hybrid(snr_db=snr_db)
    K = sc.K
    cb = channel.dft_codebook(sc, device=device)
    params = channel.draw_beam_users(sc, batch, seed)
    dt = torch.complex64 if precision == "c64" else torch.complex128
    methods = [("full", None)] + [("wb", e) for e in etas]
    hs = []
    for m, e in methods:
        rule = binding.RankRule(eta=e or 0.9, k_init=2, p=1, reinverse_period=reinverse_period,
                                seed=seed)
        hs.append(binding.WBRZF(batch, K, K, sc.alpha, sc.sigma2, p_t=sc.p_t, rule=rule,
                                method=m, precision=precision, device=device))
    rates = [[] for _ in methods]
    ops = [0.0 for _ in methods]
    ranks = [[] for _ in methods]
    branches = [dict() for _ in methods]
    t0 = -(steps // 2)                                        # pass centred on t = 0
    for s in range(steps):
        He, Ht, F = channel.hybrid_channels(params, t0 + s, cb, device=device, dtype=dt)
        for i, h in enumerate(hs):
            W = h.full_inverse(He) if s == 0 else h.update(He)
            rates[i].append(true_sum_rate(Ht, F, W, sc.p_t, sc.sigma2))
            if s == 0:
                continue
            for inf in h.step_info():
                direct = inf["branch"] in (2, 3, 4, 5, 6)
                ops[i] += op_count(K, inf["r"], direct)
                if not direct:
                    ranks[i].append(inf["r"])
                name = binding.BRANCH_NAMES[inf["branch"]]
                branches[i][name] = branches[i].get(name, 0) + 1
    for h in hs:
        h.close()
    R = [torch.stack(r[1:]).flatten().cpu() for r in rates]   # updates only (not the init)
    qs = torch.tensor([0.05, 0.25, 0.5, 0.75, 0.95], dtype=torch.float64)
    full_mean = float(R[0].mean())
    table = []
    for i, (m, e) in enumerate(methods):
        row = {"method": "conventional RZF" if m == "full" else "WB-arSVD", "eta": e,
               "mean_sum_rate": float(R[i].mean()),
               "ecdf_quantiles": {f"{float(q):.2f}": float(v)
                                  for q, v in zip(qs, torch.quantile(R[i].double(), qs))},
               "savings_pct": 100.0 * (1.0 - ops[i] / ops[0]),
               "sr_degradation_pct": 100.0 * (1.0 - float(R[i].mean()) / full_mean),
               "mean_rank": (sum(ranks[i]) / len(ranks[i])) if ranks[i] else None,
               "branches": branches[i]}
        if e in PAPER_TABLE5:
            row["paper_table5"] = {"savings_pct": PAPER_TABLE5[e][0],
                                   "sr_degradation_pct": PAPER_TABLE5[e][1]}
        table.append(row)
    return {"K": K, "N": sc.N, "N_RF": K, "updates_per_run": steps - 1, "runs": batch,
            "update_period_ms": sc.dt * 1e3, "precision": precision, "snr_db": snr_db,
            "reinverse_period": reinverse_period, "table": table,
            **({"t0": t0, "sum_rates": [torch.stack(r).cpu().tolist() for r in rates]}
               if per_snapshot else {})}
