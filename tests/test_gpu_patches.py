"""GPU parity of the two-patch system (an outer grid and an inner Cartesian
box coupled by Lagrange interpolation; the paper's Sec. 5 multiple patches
and Sec. 6 multipatch grids) against the oracle's two-patch system, through
the C ABI.

- aligned boxes (interpolation is injection): the coupled GPU trajectory
  equals the GPU single-grid trajectory, and the oracle's;
- Spherical outer patch with a Cartesian box around the punctures: fixed-step
  trajectories of both patches agree with the oracle to 1e-12, the
  receivers stay interpolated from their donors, and the coupled relaxation
  converges after the oracle's number of steps to the oracle's u (1e-10);
- set-up errors: a hole too large for the box, an inner grid that is not
  Cartesian.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2501_14030_gb300 import nrr, workloads as W
from tests.helpers import oracle_grid, rel_err

pytestmark = pytest.mark.gpu

PUNC = W.spinning_q4_pair()
SPH = W.grid_desc("spherical", (32, 16, 16), 4, rmax=48.0)
BOX = W.grid_desc("cartesian", (24, 24, 24), 4, xmax=8.0)
HOLE = 3.0


def _pair(outer_desc, inner_desc, hole, q=4):
    go, gi = nrr.Grid(outer_desc), nrr.Grid(inner_desc)
    go.set_punctures(PUNC)
    gi.set_punctures(PUNC)
    ps = nrr.PatchSet(go, gi, hole, q)
    return go, gi, ps


def _oracle_pair(outer_desc, inner_desc, hole, q=4):
    import oracle as O
    a, b = oracle_grid(outer_desc), oracle_grid(inner_desc)
    ds = min(a.dsmin, b.dsmin)
    a.set_speed_reference(ds)
    b.set_speed_reference(ds)
    sa, sb = a.source(PUNC), b.source(PUNC)
    la, lb = O.Link(a, b, 1, hole=hole, q=q), O.Link(b, a, 0, q=q)
    return a, b, sa, sb, la, lb


def _state(g):
    u = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    v = torch.empty_like(u)
    g.get_state(u, v)
    return u.cpu().numpy(), v.cpu().numpy()


def test_aligned_boxes_give_the_single_grid_trajectory(gpu):
    """Box nodes on the outer Cartesian nodes (spacing 1 in both): the
    coupled trajectory from rest equals the single outer grid's trajectory
    in both patches (to rounding), and the oracle's coupled trajectory."""
    import oracle as O
    outer = W.grid_desc("cartesian", (32, 32, 32), 4, xmax=16.0)
    inner = W.grid_desc("cartesian", (16, 16, 16), 4, xmax=8.0)
    go, gi, ps = _pair(outer, inner, 5.0)
    assert (ps.outer_receivers, ps.inner_receivers) == (10 ** 3, 20 ** 3 - 16 ** 3)
    dt, eta = ps.timestep(0.5)
    single = nrr.Grid(outer)
    single.set_punctures(PUNC)
    dts, etas = single.timestep(0.5)
    assert (dt, eta) == (dts, etas)
    for g in (go, gi, single):
        z = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        g.set_state(z, z)
    ps.step(40, dt, eta)
    single.step(40, dt, eta)
    us, vs = _state(single)
    ua, va = _state(go)
    ub, vb = _state(gi)
    sl = (slice(8, 28), slice(8, 28), slice(8, 28))
    scale = np.abs(us).max()
    assert np.abs(ua - us).max() <= 1e-14 * scale
    assert np.abs(ub - us[sl]).max() <= 1e-14 * scale
    assert np.abs(vb - vs[sl]).max() <= 1e-14 * np.abs(vs).max()
    a, b, sa, sb, la, lb = _oracle_pair(outer, inner, 5.0)
    uo, vo, ui, vi = a.zeros(), a.zeros(), b.zeros(), b.zeros()
    for _ in range(40):
        O.patch_rk4_step(a, sa, b, sb, la, lb, eta, dt, uo, vo, ui, vi)
    assert rel_err(ua, uo) <= 1e-12 and rel_err(ub, ui) <= 1e-12
    for x in (ps, go, gi, single):
        x.close()


def test_sphere_and_box_trajectory_matches_oracle(gpu):
    import oracle as O
    go, gi, ps = _pair(SPH, BOX, HOLE)
    a, b, sa, sb, la, lb = _oracle_pair(SPH, BOX, HOLE)
    assert (ps.outer_receivers, ps.inner_receivers) == (la.n, lb.n)
    assert ps.ds_ref == pytest.approx(min(a.dsmin, b.dsmin), rel=1e-13)
    dt, eta = ps.timestep(0.5)
    for g in (go, gi):
        z = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        g.set_state(z, z)
    uo, vo, ui, vi = a.zeros(), a.zeros(), b.zeros(), b.zeros()
    for k in range(2):
        ps.step(15, dt, eta)
        for _ in range(15):
            O.patch_rk4_step(a, sa, b, sb, la, lb, eta, dt, uo, vo, ui, vi)
        ua, va = _state(go)
        ub, vb = _state(gi)
        for got, ref in ((ua, uo), (va, vo), (ub, ui), (vb, vi)):
            assert rel_err(got, ref) <= 1e-12, (k, rel_err(got, ref))
    # the receivers hold the interpolation of their donors
    for link, donor, recv in ((la, ub, ua), (la, vb, va), (lb, ua, ub), (lb, va, vb)):
        idx = link.arrays()[0]
        want = np.zeros_like(recv)
        link.apply(donor, want)
        assert np.abs(want.ravel()[idx] - recv.ravel()[idx]).max() <= \
            1e-13 * np.abs(recv).max()
    for x in (ps, go, gi):
        x.close()


def test_sphere_and_box_relaxation_matches_oracle(gpu):
    import oracle as O
    go, gi, ps = _pair(SPH, BOX, HOLE)
    a, b, sa, sb, la, lb = _oracle_pair(SPH, BOX, HOLE)
    dt, eta = ps.timestep(0.5)
    r = ps.relax(tol=1e-10, check_every=50)
    assert r["status"] == 0 and r["norm"] < 1e-10
    uo, vo, ui, vi = a.zeros(), a.zeros(), b.zeros(), b.zeros()
    it, nrm, st = O.patch_relax(a, sa, b, sb, la, lb, uo, vo, ui, vi, eta=eta,
                                dt=dt, tol=1e-10, check_every=50,
                                max_iters=20000)
    assert st == 0 and it == r["iters"], (it, r)
    ua, _ = _state(go)
    ub, _ = _state(gi)
    assert rel_err(ua, uo) <= 1e-10 and rel_err(ub, ui) <= 1e-10
    # the coupled residual norm agrees with the oracle's
    Ha, Hb = a.residual(*sa, a.fill_inner_ghosts(ua)), b.residual(*sb, ub)
    n_or = O.patch_norm(a, Ha, la, b, Hb, lb, 100.0)
    assert ps.residual(100.0) == pytest.approx(n_or, rel=1e-10)
    for x in (ps, go, gi):
        x.close()


def test_patchset_rejects_bad_setups(gpu):
    go = nrr.Grid(SPH)
    gi = nrr.Grid(BOX)
    go.set_punctures(PUNC)
    with pytest.raises(nrr.NrrError) as e:
        nrr.PatchSet(go, gi, HOLE)          # punctures missing on the box
    assert e.value.status == nrr.ERR_STATE
    gi.set_punctures(PUNC)
    with pytest.raises(nrr.NrrError) as e:
        nrr.PatchSet(go, gi, 6.0)           # hole reaches the box's donors
    assert e.value.status == nrr.ERR_INVALID_ARG and "hole" in str(e.value)
    with pytest.raises(nrr.NrrError) as e:
        nrr.PatchSet(gi, go, HOLE)          # inner patch not Cartesian
    assert e.value.status == nrr.ERR_INVALID_ARG
    go.close()
    gi.close()


def test_patch_relax_chunk_graph_equals_kernel_by_kernel_steps(gpu):
    """The coupled relaxation replays each full chunk (RK4 steps of both
    patches with their links, then the norm) as one captured CUDA graph;
    a last, shorter chunk is launched kernel by kernel.  From rest, 120
    steps in chunks of 50 (two graph replays and a 20-step tail) give
    bit-for-bit the state of 120 steps launched one kernel at a time."""
    go, gi, ps = _pair(SPH, BOX, HOLE)
    r = ps.relax(tol=1e-30, max_iters=120, check_every=50, raise_on_error=False)
    assert r["iters"] == 120
    got = _state(go) + _state(gi)
    go2, gi2, ps2 = _pair(SPH, BOX, HOLE)
    for g in (go2, gi2):
        z = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        g.set_state(z, z)
    dt, eta = ps2.timestep(0.5)
    ps2.step(120, dt, eta)
    want = _state(go2) + _state(gi2)
    for a, b in zip(got, want):
        assert np.array_equal(a, b)
    # a second relaxation reuses the cached graph and stays reproducible
    r2 = ps.relax(tol=1e-30, max_iters=120, check_every=50, raise_on_error=False)
    assert r2["iters"] == 120
    for a, b in zip(_state(go) + _state(gi), want):
        assert np.array_equal(a, b)
    for obj in (ps, go, gi, ps2, go2, gi2):
        obj.close()


def test_patch_defect_correction_reaches_the_fp64_coupled_solution(gpu):
    """Defect correction on the coupled system (FP32 increments of both
    patches, FP32 links, FP64 defect and update): converges to the coupled
    residual 1e-10, the oracle confirms that residual on the GPU's state, and
    driven on to 1e-12 it agrees with the FP64 coupled solution driven to
    1e-12."""
    import oracle as O
    go, gi, ps = _pair(SPH, BOX, HOLE)
    r = ps.relax(tol=1e-10, mode="fp32_dc")
    assert r["status"] == nrr.OK and r["norm"] < 1e-10 and r["outer_iters"] > 0
    uo, _ = _state(go)
    ui, _ = _state(gi)
    a, b, sa, sb, la, lb = _oracle_pair(SPH, BOX, HOLE)
    Ha, Hb = a.residual(*sa, a.fill_inner_ghosts(uo)), b.residual(*sb, ui)
    onorm = O.patch_norm(a, Ha, la, b, Hb, lb, 100.0)
    assert onorm < 1e-10 and onorm == pytest.approx(r["norm"], rel=1e-8)
    r_dc = ps.relax(tol=1e-12, mode="fp32_dc", initial=nrr.INIT_CURRENT)
    assert r_dc["status"] == nrr.OK
    dc = _state(go)[0], _state(gi)[0]
    go2, gi2, ps2 = _pair(SPH, BOX, HOLE)
    r64 = ps2.relax(tol=1e-12, mode="fp64")
    assert r64["status"] == nrr.OK
    ref = _state(go2)[0], _state(gi2)[0]
    # a residual of 1e-12 fixes u to about 1e-10 of its scale (the box's
    # difference is a near-uniform offset of ~8e-12 against max |u| = 0.085)
    scale = max(np.max(np.abs(w)) for w in ref)
    for u, w in zip(dc, ref):
        assert np.max(np.abs(u - w)) <= 2e-10 * scale
    for obj in (ps, go, gi, ps2, go2, gi2):
        obj.close()


def test_patch_relax_modes_refused(gpu):
    go, gi, ps = _pair(SPH, BOX, HOLE)
    for mode in ("fp32",):
        with pytest.raises(nrr.NrrError) as e:
            ps.relax(tol=1e-10, mode=mode)
        assert e.value.status == nrr.ERR_INVALID_ARG
    with pytest.raises(nrr.NrrError):
        ps.relax(tol=1e-10, mode="fp32_dc", inner_steps=-1)
    for obj in (ps, go, gi):
        obj.close()
