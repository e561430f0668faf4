"""Operation-count models of the paper (oracle side, used for reporting only).

Table I (Section III-A): full K x K inversion O(K^3); Woodbury update
O(K^2 + K^2 r + r^3 + r^2 K).  Table II (Section IV-A): full SVD O(K^3); arSVD
O(K^2 r + r^2 K).  Table IV (Section V): the combined WB-arSVD update is
O(K^2 + K^2 r + r^3 + r^2 K) against O(K^3) for direct inversion.  Table V reports savings
as one minus the ratio of the averaged model costs over a simulated pass.
"""
from __future__ import annotations

from typing import Iterable


def full_inverse_cost(K: int) -> float:
    return float(K) ** 3


def wb_arsvd_cost(K: int, r: int) -> float:
    K, r = float(K), float(r)
    return K * K + K * K * r + r ** 3 + r * r * K


def normalised_wb_cost(K: int, r: int) -> float:
    """Table IV cost of WB-arSVD over that of a direct inverse (the curve of Fig. 1)."""
    return wb_arsvd_cost(K, r) / full_inverse_cost(K)


def savings(K: int, branches: Iterable[int], ranks: Iterable[int]) -> float:
    """1 - (model cost of the method over a run) / (K^3 per snapshot), as in Table V.

    branches/ranks are per snapshot: Woodbury snapshots (branch 1) cost the Table IV model at
    their rank, skipped ones (branch 0) cost nothing, every other snapshot costs K^3.
    """
    total = 0.0
    n = 0
    for b, r in zip(branches, ranks):
        n += 1
        if b == 1:
            total += wb_arsvd_cost(K, r)
        elif b == 0:
            total += 0.0
        else:
            total += full_inverse_cost(K)
    return 1.0 - total / (n * full_inverse_cost(K)) if n else 0.0
