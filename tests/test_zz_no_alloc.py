"""The allocation-free residual entry point (nrr_residual_noalloc).

Callers that cannot call cudaMalloc -- for example an application whose own
memory manager owns the whole device -- get the residual norm of their u
through nrr_residual_noalloc, whose only scratch is a static device array.
This test calls it through the C ABI several times in a row, on grids of all
three coordinate families it takes and FD orders 4, 8 and 10, and checks each
result against the grid-based nrr_residual and against the CPU oracle's
residual and norm, within the residual tolerance of the other parity tests
(1e-12 relative).  Consecutive calls use different block counts, so leftovers
from an earlier call in the shared scratch would show up as a mismatch.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2501_14030_gb300 import nrr, workloads as W
from tests.helpers import oracle_grid

pytestmark = pytest.mark.gpu

TOL = 1e-12

CASES = [
    ("q4 SinhSymTP 128x128x16 o8", W.q4_sinhsymtp_128),
    ("SinhSymTP 44x26x6 o8",
     lambda: (W.grid_desc("sinhsymtp", (44, 26, 6), 8), W.spinning_q4_pair())),
    ("Spherical 32x16x4 o8",
     lambda: (W.grid_desc("spherical", (32, 16, 4), 8, rmax=24.0),
              W.spinning_q4_pair())),
    ("Cartesian 24^3 o10",
     lambda: (W.grid_desc("cartesian", (24, 24, 24), 10, xmax=12.0),
              W.spinning_q4_pair())),
    ("SinhSymTP 36x20x4 o10",
     lambda: (W.grid_desc("sinhsymtp", (36, 20, 4), 10), W.equal_mass_pair())),
    ("SinhSymTP 32x16x2 o4", W.small_equal_mass),
]


def _reference(desc, punc, u):
    g = nrr.Grid(desc)
    g.set_punctures(punc)
    g.set_state(u)
    H = torch.zeros_like(u)
    n = g.residual(100.0, H)
    g.close()
    return n, H


def _noalloc(desc, punc, u):
    norm = torch.full((1,), -1.0, dtype=torch.float64, device=u.device)
    H = torch.zeros_like(u)
    nrr.residual_noalloc(desc, punc, u, norm, H, r_int=100.0)
    torch.cuda.synchronize()
    return norm.item(), H


def test_noalloc_residual_matches_grid_residual_and_oracle(gpu):
    for seed, (name, make) in enumerate(CASES):
        desc, punc = make()
        u_np = W.smooth_random_field(desc, seed=100 + seed, amplitude=0.2,
                                     noise=0.01)
        u = torch.from_numpy(u_np).cuda()
        n_ref, H_ref = _reference(desc, punc, u)
        n, H = _noalloc(desc, punc, u)
        assert abs(n - n_ref) <= TOL * n_ref, (name, n, n_ref)
        Hr, Hn = H_ref.cpu().numpy(), H.cpu().numpy()
        assert np.abs(Hn - Hr).max() <= TOL * np.abs(Hr).max(), name
        # the oracle: its residual at interior points and its norm
        og = oracle_grid(desc)
        alpha, beta = og.source(punc)
        H_or = og.residual(alpha, beta, og.fill_inner_ghosts(u_np))
        n_or = og.norm(H_or, 100.0)
        assert abs(n - n_or) <= TOL * n_or, (name, n, n_or)
        assert np.abs(Hn - H_or).max() <= TOL * np.abs(H_or).max(), name


def test_noalloc_rejects_oversized_grid(gpu):
    """n0*n1 above the static scratch's capacity is refused with a clear
    error.  u has the grid's full size, so nothing would be read out of
    range even if the check were missing."""
    desc = W.grid_desc("cartesian", (4096, 1025, 2), 4)
    u = torch.zeros(W.padded_shape(desc), dtype=torch.float64, device="cuda")
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(nrr.NrrError) as e:
        nrr.residual_noalloc(desc, W.spinning_q4_pair(), u, norm)
    assert e.value.status == nrr.ERR_INVALID_ARG
    assert "static scratch" in str(e.value)
    del u
    torch.cuda.empty_cache()
