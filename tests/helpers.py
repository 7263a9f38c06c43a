"""Shared test helpers: oracle grids from workload descriptors, comparisons."""
from __future__ import annotations

import numpy as np

from paper_2501_14030_gb300 import workloads as W


def oracle_grid(desc: dict):
    import oracle as O
    return O.grid_from_desc(desc)


def default_dt_eta(og, cfl: float = 0.5):
    """dt = cfl min ds; eta dt = 2 pi cfl / n0 (the damping reading)."""
    import oracle as O
    return O.default_dt_eta(og, cfl)


def region_masks(og):
    import oracle as O
    kind = og.field("kind")
    return {"interior": kind == O.INTERIOR, "outer": kind == O.OUTER,
            "inner": kind == O.INNER}


def rel_err(a: np.ndarray, b: np.ndarray, mask=None) -> float:
    """max |a - b| / max |b| over mask (0 if b vanishes there)."""
    if mask is not None:
        a, b = a[mask], b[mask]
    if a.size == 0:
        return 0.0
    den = np.abs(b).max()
    num = np.abs(a - b).max()
    if den == 0.0:
        return float(num)
    return float(num / den)
