"""Writes oracle_small_equal_mass.txt: the oracle's relaxation of the small
equal-mass workload (SinhSymTP 32x16x2, order 4, CFL 0.5, damping
eta dt = 2 pi CFL / n0, residual 1e-10 checked every 50 steps) -- its step
count, final norm and u at sampled interior points.

A regression record of the oracle against its own earlier output, not an
independent pin: a change of the oracle's arithmetic shows up here and must
name the passage that justifies it.  Calls only oracle/ (and the seeded
workload definitions).  Run from the repository root:
    python tests/golden/make_oracle_reference.py
"""
from __future__ import annotations

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_2501_14030_gb300 import workloads as W  # noqa: E402
from tests.helpers import default_dt_eta, oracle_grid  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                   "oracle_small_equal_mass.txt")
# interior samples (i2, i1, i0) in padded indices: near the inner boundary,
# near the punctures' focus, mid-grid and next to the outer boundary
SAMPLES = [(2, 2, 2), (2, 2, 17), (3, 9, 2), (3, 10, 20), (2, 17, 9),
           (3, 5, 33), (2, 12, 30), (3, 2, 25), (2, 9, 12), (3, 14, 5)]


def compute():
    desc, punc = W.small_equal_mass()
    og = oracle_grid(desc)
    alpha, beta = og.source(punc)
    dt, eta = default_dt_eta(og)
    u, v = og.zeros(), og.zeros()
    iters, norm, status = og.relax(alpha, beta, u, v, eta=eta, dt=dt, tol=1e-10,
                                   check_every=50)
    return iters, norm, status, {s: float(u[s]) for s in SAMPLES}


def main():
    iters, norm, status, samples = compute()
    assert status == 0
    with open(OUT, "w") as f:
        f.write("# Written by tests/golden/make_oracle_reference.py (oracle only).\n")
        f.write("# Small equal-mass workload, SinhSymTP 32x16x2, order 4: steps,\n")
        f.write("# final residual norm, then u at padded indices i2 i1 i0.\n")
        f.write(f"steps {iters}\n")
        f.write(f"norm {norm:.17e}\n")
        for (i2, i1, i0), val in samples.items():
            f.write(f"u {i2} {i1} {i0} {val:.17e}\n")


if __name__ == "__main__":
    main()
