"""Merging trajectory statistics over replicas (one process per GPU).

Trajectories are independent (Sec. III: the estimator is an average over
independently sampled trajectories), so ranks run disjoint trajectory ranges
and only their statistics are combined.  The combination here is exact: each
rank reduces its per-trajectory values to (sum x, sum x^2, count) held as
exact rationals (a double is a dyadic rational, so these sums are exact Python
integers over a power of two), the ranks add them, and the mean and standard
error are rounded once at the end.  The merged result therefore does not
depend on how the trajectories were split over ranks, bit for bit.
"""
from __future__ import annotations

from fractions import Fraction
from typing import Dict, Sequence

import numpy as np


def exact_sums(values: np.ndarray) -> Dict[str, list]:
    """Column-wise exact (sum x, sum x^2) and the count of a [B, k] array (or
    [B]) of finite doubles; sums are returned as Fractions."""
    v = np.asarray(values, dtype=np.float64)
    if v.ndim == 1:
        v = v[:, None]
    if not np.all(np.isfinite(v)):
        raise ValueError("exact_sums: non-finite value")
    s1, s2 = [], []
    for c in range(v.shape[1]):
        col = [Fraction(float(x)) for x in v[:, c]]
        s1.append(sum(col, Fraction(0)))
        s2.append(sum((x * x for x in col), Fraction(0)))
    return {"sum": s1, "sum_sq": s2, "count": int(v.shape[0])}


def add_sums(a: Dict[str, list], b: Dict[str, list]) -> Dict[str, list]:
    """Sum of two exact-sum records with the same columns."""
    if len(a["sum"]) != len(b["sum"]):
        raise ValueError("add_sums: column counts differ")
    return {"sum": [x + y for x, y in zip(a["sum"], b["sum"])],
            "sum_sq": [x + y for x, y in zip(a["sum_sq"], b["sum_sq"])],
            "count": a["count"] + b["count"]}


def finalize(s: Dict[str, list]):
    """(mean, standard error of the mean) per column, each rounded once from
    the exact sums: mean = S1 / N, s.e. = sqrt((S2 - S1^2 / N) / (N - 1) / N)."""
    n = s["count"]
    mean = np.array([float(x / n) for x in s["sum"]]) if n else np.zeros(len(s["sum"]))
    se = np.zeros(len(s["sum"]))
    if n > 1:
        for c, (s1, s2) in enumerate(zip(s["sum"], s["sum_sq"])):
            var = (s2 - s1 * s1 / n) / (n - 1) / n
            se[c] = float(np.sqrt(float(var))) if var > 0 else 0.0
    return mean, se


def merge_over_ranks(dist, local: Dict[str, list]) -> Dict[str, list]:
    """Exact sums of every rank, added in rank order (torch.distributed
    all_gather_object: the Fractions travel as pickled integers)."""
    gathered: list = [None] * dist.get_world_size()
    dist.all_gather_object(gathered, local)
    out = gathered[0]
    for g in gathered[1:]:
        out = add_sums(out, g)
    return out


def merged_observables(dist, per_traj: Sequence[np.ndarray]):
    """Merge the per-trajectory observables of this rank's handles ([B_i, k]
    arrays with the same k) over all ranks; returns (mean, s.e.) per column."""
    local = None
    for a in per_traj:
        s = exact_sums(a)
        local = s if local is None else add_sums(local, s)
    return finalize(merge_over_ranks(dist, local))
