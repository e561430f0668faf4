"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and the FP64 oracle
on the same channel snapshots, and compare."""
from __future__ import annotations

import numpy as np
import torch

from oracle import method as om
from paper_2512_16543_gb300 import binding


def relerr(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def oracle_rule(rule: binding.RankRule) -> om.RankRule:
    return om.RankRule(eta=rule.eta, k_init=rule.k_init, p=rule.p, i_max=rule.i_max,
                       r_max=rule.r_max, switch_ratio=rule.switch_ratio,
                       reinverse_period=rule.reinverse_period, seed=rule.seed,
                       dg_floor_rel=rule.dg_floor_rel)


def run_gpu(Hs: torch.Tensor, alpha, sigma2, p_t, rule: binding.RankRule, *, precision="c64",
            method="wb", ids=None, trace=False, keep_state=True, device="cuda", engine="auto",
            fp64_small=False, energy_shortcut=False):
    """Hs: [T, B, K, N] complex tensor (any device).  Returns a list of per-step dicts.
    fp64_small: the blocked engine's FP64 small-solve mode."""
    T, B, K, N = Hs.shape
    dt = torch.complex64 if precision == "c64" else torch.complex128
    h = binding.WBRZF(B, N, K, alpha, sigma2, p_t=p_t, rule=rule, method=method,
                      precision=precision, device=device,
                      workspace_for="blocked" if engine.startswith("blocked") else "auto")
    if engine != "auto":
        h.set_engine(engine)
    if fp64_small:
        h.set_fp64_small_solves(True)
    if energy_shortcut:
        h.set_energy_shortcut(True)
    if ids is not None:
        h.set_instance_ids(ids)
    if trace:
        h.enable_trace()
    _, _, dmax, rcap = binding.resolved_sizes(K, rule)
    out = []
    for t in range(T):
        H = Hs[t].to(device=device, dtype=dt).contiguous()
        W = h.full_inverse(H) if t == 0 else h.update(H)
        sinr, rate = h.sum_rate()
        rec = {"W": W.cpu().numpy(), "sinr": sinr.cpu().numpy(), "rate": rate.cpu().numpy(),
               "info": h.step_info()}
        if keep_state:
            G, X = h.state()
            rec["G"] = G.cpu().numpy()
            rec["X"] = X.cpu().numpy()
        if trace:
            sig, Lm, Rh = h.trace(dmax, rcap)
            rec["sig"] = sig.cpu().numpy()
            rec["L"] = Lm.cpu().numpy()
            rec["Rh"] = Rh.cpu().numpy()
        out.append(rec)
    torch.cuda.synchronize()
    rec0 = {"launches": h.launches, "rcap": rcap, "dmax": dmax, "engine": h.last_engine}
    h.close()
    return out, rec0


def run_oracle(Hs_b: np.ndarray, alpha, sigma2, p_t, rule: binding.RankRule, *, instance=0,
               method="wb", lowrank_mode="arsvd"):
    """Hs_b: [T, K, N] complex128 snapshots of one instance."""
    return om.run_trajectory(list(Hs_b), alpha, p_t, sigma2, method=method,
                             rule=oracle_rule(rule), lowrank_mode=lowrank_mode,
                             instance=instance)


def energy_tie(ref_step, E_rel_tol, eta, r_gpu) -> bool:
    """True when the oracle's cumulative energy at rank r_gpu (or r_gpu - 1) is within
    E_rel_tol of its target, i.e. the two ranks are both defensible readings of eq. 14."""
    sig = ref_step.sigma_hat
    if sig is None:
        return False
    target = eta * ref_step.dA_fro2
    cum = np.concatenate([[0.0], np.cumsum(np.asarray(sig) ** 2)])
    for r in (r_gpu, r_gpu - 1, ref_step.r, ref_step.r - 1):
        if 0 <= r < len(cum) and abs(cum[r] - target) <= E_rel_tol * target:
            return True
    return False
