"""The allocation-free residual entry point (nrr_residual_noalloc).

Callers that cannot call cudaMalloc -- for example an application whose own
memory manager owns the whole device -- get the residual norm of their u
through nrr_residual_noalloc, whose only scratch is a static device array.
This test calls it through the C ABI twice in a row, on two different grids,
and checks each result against the grid-based nrr_residual within the
residual tolerance of the other parity tests (1e-12 relative).  The second
call uses fewer blocks than the first, so leftovers from the first call in
the shared scratch would show up as a mismatch.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2501_14030_gb300 import nrr, workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12


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


def test_noalloc_residual_matches_grid_residual_twice(gpu):
    cases = [W.q4_sinhsymtp_128(),
             (W.grid_desc("sinhsymtp", (44, 26, 6), 8), W.spinning_q4_pair())]
    for seed, (desc, punc) in enumerate(cases):
        u = torch.from_numpy(W.smooth_random_field(
            desc, seed=100 + seed, amplitude=0.2, noise=0.01)).cuda()
        n_ref, H_ref = _reference(desc, punc, u)
        n, H = _noalloc(desc, punc, u)
        assert abs(n - n_ref) <= TOL * n_ref, (desc["n"], n, n_ref)
        Hr, Hn = H_ref.cpu().numpy(), H.cpu().numpy()
        assert np.abs(Hn - Hr).max() <= TOL * np.abs(Hr).max()


def test_noalloc_rejects_oversized_grid(gpu):
    desc = W.grid_desc("cartesian", (4096, 1025, 2), 4)
    u = torch.zeros(1, dtype=torch.float64, device="cuda")
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(nrr.NrrError) as e:
        nrr.residual_noalloc(desc, W.spinning_q4_pair(), u, norm)
    assert e.value.status == nrr.ERR_INVALID_ARG
    assert "static scratch" in str(e.value)
