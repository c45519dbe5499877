"""Bank regions for the prescreen: templates sorted by chirp mass
M_c = (m1 m2)^(3/5) / (m1 + m2)^(1/5) and split into equal-count groups;
filtering orders built from region scores.  Host-side bookkeeping only."""

from __future__ import annotations

import numpy as np


def chirp_mass(m1, m2):
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2


def bank_regions(m1, m2, regions: int):
    """(list of template-index arrays, one per region, in increasing chirp mass;
    upper chirp-mass boundaries of regions 0 .. regions-2)."""
    mc = chirp_mass(m1, m2)
    order = np.argsort(mc, kind="stable")
    groups = np.array_split(order, regions)
    bounds = np.array([mc[g[-1]] for g in groups[:-1]])
    return groups, bounds


def region_index(mc, bounds):
    """Region of chirp mass(es) `mc` given the region boundaries."""
    return np.searchsorted(bounds, np.asarray(mc, dtype=np.float64), side="left")


def ranked_order(scores, groups, top_k: int | None = None):
    """Template order for cui_filter_bank: regions by descending score, the
    first `top_k` of them (all by default), templates of each region in bank
    order."""
    ranked = np.argsort(-np.asarray(scores), kind="stable")
    if top_k is not None:
        ranked = ranked[:top_k]
    if len(ranked) == 0:
        return np.zeros(0, dtype=np.int32)
    return np.concatenate([groups[r] for r in ranked]).astype(np.int32)
