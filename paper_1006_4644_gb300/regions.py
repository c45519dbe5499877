"""Chirp mass M_c = (m1 m2)^(3/5) / (m1 + m2)^(1/5) of bank points, the key
that orders the bank for sharding (shard.py).  The prescreen's region
ranking runs in the library (cui_prescreen_rank)."""

from __future__ import annotations

import numpy as np


def chirp_mass(m1, m2):
    m1 = np.asarray(m1, dtype=np.float64)
    m2 = np.asarray(m2, dtype=np.float64)
    return (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2
