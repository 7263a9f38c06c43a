"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

FP64 tolerances: 1e-12 relative per RHS evaluation and per trajectory
(max-norm relative to the oracle field's maximum, per region), 1e-10
relative on converged u.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2501_14030_gb300 import nrr, workloads as W
from tests.helpers import default_dt_eta, oracle_grid, rel_err, region_masks

pytestmark = pytest.mark.gpu

Q4 = W.spinning_q4_pair()
CASES = {
    # small equal-mass case, 4th order
    "sinh_32x16x2_o4": W.small_equal_mass(),
    # several tiles with ragged edges, 8th and 10th order
    "sinh_44x26x6_o8": (W.grid_desc("sinhsymtp", (44, 26, 6), 8), Q4),
    "sinh_36x20x10_o10": (W.grid_desc("sinhsymtp", (36, 20, 10), 10), Q4),
    "sph_40x22x8_o8": (W.grid_desc("spherical", (40, 22, 8), 8, rmax=64.0), Q4),
    "cart_26x20x22_o4": (W.grid_desc("cartesian", (26, 20, 22), 4, xmax=32.0), Q4),
    "cart_20x18x24_o8": (W.grid_desc("cartesian", (20, 18, 24), 8, xmax=32.0), Q4),
    "sinhsph_40x22x8_o8": (W.grid_desc("sinhspherical", (40, 22, 8), 8), Q4),
    "sinhsph_36x20x6_o4": (W.grid_desc("sinhspherical", (36, 20, 6), 4,
                                       amax=200.0, sinhwaa=0.2), Q4),
    # SinhCylindrical (rho, z, phi): outer points beyond the side and both
    # ends, ragged tiles
    "sinhcyl_40x26x8_o8": (W.grid_desc("sinhcylindrical", (40, 26, 8), 8,
                                       amax=100.0, sinhwaa=0.3, zmax=100.0,
                                       sinhwz=0.3), Q4),
    "sinhcyl_22x18x6_o4": (W.grid_desc("sinhcylindrical", (22, 18, 6), 4,
                                       amax=60.0, sinhwaa=0.3, zmax=40.0,
                                       sinhwz=0.25), Q4),
    # full-size q=4 grid
    "sinh_128x128x16_o8": W.q4_sinhsymtp_128(),
}
# The larger full-size q=4 grids (SinhSymTP 256x256x32, Spherical 128x64x32,
# Cartesian 256^3, order 8): RHS and residual parity over every point.
FULL = {
    "sinh_256x256x32_o8": W.q4_sinhsymtp_256(),
    "sinhsph_128x64x16_o8": W.q4_sinhspherical_128(),
    "sph_128x64x32_o8": W.q4_spherical_128(),
    "cart_256x256x256_o8": W.q4_cartesian_256(),
}
ALL = {**CASES, **FULL}


def _dev(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _setup(name):
    desc, punc = ALL[name]
    og = oracle_grid(desc)
    alpha, beta = og.source(punc)
    g = nrr.Grid(desc)
    g.set_punctures(punc)
    return desc, punc, og, alpha, beta, g


@pytest.mark.parametrize("name", list(CASES))
def test_timestep_matches_oracle(gpu, name):
    desc, punc, og, alpha, beta, g = _setup(name)
    dt, eta = g.timestep(0.5)
    dto, etao = default_dt_eta(og)
    assert abs(dt - dto) <= 1e-13 * dto
    assert abs(eta - etao) <= 1e-13 * etao


@pytest.mark.parametrize("name", list(ALL))
def test_rhs_parity_fp64(gpu, name):
    desc, punc, og, alpha, beta, g = _setup(name)
    u = W.smooth_random_field(desc, seed=11, amplitude=0.2, noise=0.01)
    v = W.smooth_random_field(desc, seed=12, amplitude=0.1, noise=0.01)
    dt, eta = default_dt_eta(og)
    ku_o, kv_o = og.rhs(alpha, beta, eta, og.fill_inner_ghosts(u),
                        og.fill_inner_ghosts(v))
    # The device gets the raw fields: inner ghosts hold unrelated values, so
    # any read of ghost memory instead of the image shows up as a mismatch.
    ku, kv = torch.empty_like(_dev(u)), torch.empty_like(_dev(u))
    g.rhs(_dev(u), _dev(v), ku, kv, eta, mode="fp64")
    ku, kv = ku.cpu().numpy(), kv.cpu().numpy()
    for region, m in region_masks(og).items():
        assert rel_err(ku, ku_o, m) <= 1e-12, (region, rel_err(ku, ku_o, m))
        assert rel_err(kv, kv_o, m) <= 1e-12, (region, rel_err(kv, kv_o, m))


@pytest.mark.parametrize("name", ["sinh_32x16x2_o4", "sinh_44x26x6_o8",
                                  "cart_26x20x22_o4", "sinh_128x128x16_o8"])
def test_source_parity(gpu, name):
    """At u = v = 0 the RHS is c^2 beta: the Bowen-York source on device."""
    desc, punc, og, alpha, beta, g = _setup(name)
    z = np.zeros(og.shape)
    ku_o, kv_o = og.rhs(alpha, beta, 1.0, z, z)
    ku, kv = torch.empty_like(_dev(z)), torch.empty_like(_dev(z))
    g.rhs(_dev(z), _dev(z), ku, kv, 1.0, mode="fp64")
    m = region_masks(og)["interior"]
    assert rel_err(kv.cpu().numpy(), kv_o, m) <= 1e-12


@pytest.mark.parametrize("name", list(ALL))
def test_residual_and_norm_parity(gpu, name):
    desc, punc, og, alpha, beta, g = _setup(name)
    u = W.smooth_random_field(desc, seed=21, amplitude=0.2, noise=0.01)
    H_o = og.residual(alpha, beta, og.fill_inner_ghosts(u))
    for r_int in (100.0, 1.0e9):
        n_o = og.norm(H_o, r_int)
        g.set_state(_dev(u))
        H = torch.empty_like(_dev(u))
        n = g.residual(r_int, H)
        assert abs(n - n_o) <= 1e-12 * n_o, (r_int, n, n_o)
        m = region_masks(og)["interior"]
        assert rel_err(H.cpu().numpy(), H_o, m) <= 1e-12


@pytest.mark.parametrize("name,steps", [("sinh_32x16x2_o4", 200),
                                        ("sinh_44x26x6_o8", 60),
                                        ("sinhcyl_40x26x8_o8", 60),
                                        ("sinhcyl_22x18x6_o4", 100),
                                        ("sinhsph_40x22x8_o8", 60),
                                        ("sinh_36x20x10_o10", 40),
                                        ("sph_40x22x8_o8", 60),
                                        ("cart_26x20x22_o4", 60),
                                        ("sinh_128x128x16_o8", 8)])
def test_trajectory_parity_fp64(gpu, name, steps):
    """Fixed-step trajectories from the same state agree to 1e-12."""
    desc, punc, og, alpha, beta, g = _setup(name)
    dt, eta = default_dt_eta(og)
    u = og.fill_inner_ghosts(W.smooth_random_field(desc, seed=31, amplitude=0.1))
    v = og.zeros()
    g.set_state(_dev(u), _dev(v))
    g.step(steps, dt, eta, mode="fp64")
    for _ in range(steps):
        og.rk4_step(alpha, beta, eta, dt, u, v)
    ug, vg = torch.empty_like(_dev(u)), torch.empty_like(_dev(u))
    g.get_state(ug, vg)
    assert rel_err(ug.cpu().numpy(), u) <= 1e-12
    assert rel_err(vg.cpu().numpy(), v) <= 1e-12


@pytest.mark.parametrize("name", ["sinh_32x16x2_o4", "sph_40x22x8_o8",
                                  "cart_26x20x22_o4", "sinhsph_36x20x6_o4",
                                  "sinhcyl_22x18x6_o4", "sinhcyl_40x26x8_o8"])
def test_relax_converged_parity(gpu, name):
    """Full solves to 1e-10: same step count, u within 1e-10."""
    desc, punc, og, alpha, beta, g = _setup(name)
    dt, eta = default_dt_eta(og)
    res = g.relax(mode="fp64", tol=1e-10, check_every=50)
    uo, vo = og.zeros(), og.zeros()
    it, n_o, st = og.relax(alpha, beta, uo, vo, eta=eta, dt=dt, tol=1e-10,
                           check_every=50)
    assert st == 0 and res["status"] == 0
    assert it == res["iters"], (it, res)
    u = np.zeros(og.shape)
    g.get_state(u)
    assert rel_err(u, uo) <= 1e-10
    assert og.norm(og.residual(alpha, beta, u)) < 1e-10


@pytest.mark.slow
def test_relax_full_size_converged_parity(gpu):
    """The q=4 128x128x16 order-8 FP64 solve to 1e-10 against the oracle's
    own solve of it (about a minute on the host cores): the same number of
    RK4 steps and u within 1e-10 of the oracle's u."""
    desc, punc, og, alpha, beta, g = _setup("sinh_128x128x16_o8")
    dt, eta = default_dt_eta(og)
    res = g.relax(mode="fp64", tol=1e-10, check_every=50)
    uo, vo = og.zeros(), og.zeros()
    it, n_o, st = og.relax(alpha, beta, uo, vo, eta=eta, dt=dt, tol=1e-10,
                           check_every=50, max_iters=20000)
    assert st == 0 and res["status"] == 0
    assert it == res["iters"], (it, res["iters"])
    u = np.zeros(og.shape)
    g.get_state(u)
    assert rel_err(u, uo) <= 1e-10, rel_err(u, uo)


@pytest.mark.slow
def test_trajectory_parity_full_size_1000_steps(gpu):
    """1000 RK4 steps on the full 128x128x16 grid from the same state.  Both
    sides round differently in every stage (the device folds c^2 and the
    metric into per-column weights and contracts multiply-adds; the oracle
    rounds every operation of the per-point formula), so the difference of
    the two trajectories grows with the step count K, at most linearly in
    this damped system: bound K x 4e-15 (relative to max |u|), i.e. 2e-12 at
    step 500 and 4e-12 at step 1000.  Short trajectories (<= 200 steps) are
    held to 1e-12 above."""
    desc, punc, og, alpha, beta, g = _setup("sinh_128x128x16_o8")
    dt, eta = default_dt_eta(og)
    u = og.fill_inner_ghosts(W.smooth_random_field(desc, seed=32, amplitude=0.1))
    v = og.zeros()
    g.set_state(_dev(u), _dev(v))
    for half in range(2):
        g.step(500, dt, eta, mode="fp64")
        for _ in range(500):
            og.rk4_step(alpha, beta, eta, dt, u, v)
        ug, vg = torch.empty_like(_dev(u)), torch.empty_like(_dev(u))
        g.get_state(ug, vg)
        bound = 500 * (half + 1) * 4e-15
        eu, ev = rel_err(ug.cpu().numpy(), u), rel_err(vg.cpu().numpy(), v)
        print("trajectory step %d: rel. diff u %.3e, v %.3e" % (
            500 * (half + 1), eu, ev))
        assert eu <= bound and ev <= bound, (half, eu, ev)


def test_relax_full_size_residual_checked_by_oracle(gpu):
    """128x128x16 FP64 solve to 1e-10; the oracle re-evaluates the residual
    of the returned u (a size-independent check)."""
    desc, punc, og, alpha, beta, g = _setup("sinh_128x128x16_o8")
    res = g.relax(mode="fp64", tol=1e-10, check_every=50)
    u = np.zeros(og.shape)
    g.get_state(u)
    n_o = og.norm(og.residual(alpha, beta, u))
    assert res["norm"] < 1e-10
    assert n_o < 1.02e-10, n_o
    assert abs(n_o - res["norm"]) <= 1e-3 * n_o + 1e-14


def test_brill_lindquist_is_exactly_zero(gpu):
    """Zero momentum and spin: beta = 0, so u = v = 0 for all time."""
    desc = W.grid_desc("sinhsymtp", (32, 16, 4), 4)
    g = nrr.Grid(desc)
    g.set_punctures(W.brill_lindquist_pair())
    res = g.relax(mode="fp64", tol=1e-10)
    assert res["iters"] == 0 and res["norm"] == 0.0
    dt, eta = g.timestep(0.5)
    g.step(50, dt, eta)
    u = np.ones(g.shape)
    g.get_state(u)
    assert not u.any()


@pytest.mark.parametrize("mode", ["fp64", "fp32_dc"])
def test_relax_outcomes_other_than_convergence(gpu, mode):
    """nrr_relax stops with a status instead of running on: exactly
    max_iters steps -> NOT_CONVERGED; CFL 2, beyond RK4's stability for this
    operator (the oracle's relaxation blows up there too) -> DIVERGED; a
    1 ms wall-clock limit on a solve of ~0.1 s -> TIMEOUT; and with
    raise_on_error the binding raises."""
    desc, punc, og, alpha, beta, g = _setup("sinh_44x26x6_o8")
    r = g.relax(mode=mode, tol=1e-10, max_iters=100, check_every=50,
                raise_on_error=False)
    assert r["status"] == nrr.ERR_NOT_CONVERGED and r["iters"] == 100, r
    r = g.relax(mode=mode, tol=1e-10, cfl=2.0, max_iters=20000, check_every=50,
                raise_on_error=False)
    assert r["status"] == nrr.ERR_DIVERGED, r
    u, v = og.zeros(), og.zeros()
    dt, eta = default_dt_eta(og)
    _, _, st = og.relax(alpha, beta, u, v, eta=eta, dt=2.0 * og.dsmin, tol=1e-10,
                        max_iters=20000, check_every=50)
    assert st == 2  # the oracle's diverged status
    with pytest.raises(nrr.NrrError):
        g.relax(mode=mode, tol=1e-10, max_iters=100, check_every=50)
    g.close()
    desc, punc, og, alpha, beta, g = _setup("sinh_128x128x16_o8")
    r = g.relax(mode=mode, tol=1e-10, timeout_ms=1, check_every=50,
                raise_on_error=False)
    assert r["status"] == nrr.ERR_TIMEOUT and r["iters"] < 6400, r
    g.close()


def test_relax_initial_data_modes(gpu):
    """Warm starts: a converged u handed back from host memory, from device
    memory, or left in place (INIT_CURRENT) meets the tolerance at the first
    norm check; INIT_ZERO starts over."""
    desc, punc, og, alpha, beta, g = _setup("sinh_44x26x6_o8")
    r0 = g.relax(mode="fp64", tol=1e-10, check_every=50)
    u = np.zeros(og.shape)
    g.get_state(u)
    for u0 in (u, _dev(u)):
        g.relax(mode="fp64", tol=1e-10, max_iters=100, check_every=50,
                raise_on_error=False)  # move the state away first
        r = g.relax(mode="fp64", tol=1e-10, u0=u0, check_every=50)
        assert r["status"] == 0 and r["iters"] <= 50, r
    r = g.relax(mode="fp64", tol=1e-10, initial=nrr.INIT_CURRENT, check_every=50)
    assert r["status"] == 0 and r["iters"] <= 50, r
    r = g.relax(mode="fp64", tol=1e-10, initial=nrr.INIT_ZERO, check_every=50)
    assert r["iters"] == r0["iters"]
    g.close()


# ------------------------------------------------ FP32 and defect correction
FP32_RHS_TOL = 2e-5  # see test docstring


@pytest.mark.parametrize("name", ["sinh_32x16x2_o4", "sinh_44x26x6_o8",
                                  "sph_40x22x8_o8", "cart_26x20x22_o4",
                                  "sinhcyl_40x26x8_o8", "sinh_128x128x16_o8"])
def test_rhs_parity_fp32(gpu, name):
    """Single-precision RHS against the FP64 oracle.  Tolerance from the
    arithmetic: inputs and the ~5*ng+1 folded weights are rounded to FP32
    (unit roundoff 6e-8) and summed over 25-31 terms whose magnitudes exceed
    the result by at most ~10 for these smooth-plus-noise states, so the
    norm-relative error stays below 31 x 10 x 6e-8 ~ 2e-5."""
    desc, punc, og, alpha, beta, g = _setup(name)
    u = W.smooth_random_field(desc, seed=11, amplitude=0.2, noise=0.01)
    v = W.smooth_random_field(desc, seed=12, amplitude=0.1, noise=0.01)
    dt, eta = default_dt_eta(og)
    ku_o, kv_o = og.rhs(alpha, beta, eta, og.fill_inner_ghosts(u),
                        og.fill_inner_ghosts(v))
    ku, kv = torch.empty_like(_dev(u)), torch.empty_like(_dev(u))
    g.rhs(_dev(u), _dev(v), ku, kv, eta, mode="fp32")
    ku, kv = ku.cpu().numpy(), kv.cpu().numpy()
    for region, m in region_masks(og).items():
        assert rel_err(ku, ku_o, m) <= FP32_RHS_TOL, (region, rel_err(ku, ku_o, m))
        assert rel_err(kv, kv_o, m) <= FP32_RHS_TOL, (region, rel_err(kv, kv_o, m))


@pytest.mark.parametrize("name", ["sinh_32x16x2_o4", "sinh_44x26x6_o8",
                                  "sph_40x22x8_o8", "cart_26x20x22_o4",
                                  "sinhcyl_22x18x6_o4"])
def test_defect_correction_reaches_fp64_solution(gpu, name):
    """FP32 relaxation inside the FP64 defect-correction loop reaches the
    1e-10 residual (confirmed by the oracle) in about as many steps as the
    FP64 relaxation.  A residual of 1e-10 fixes u only up to the conditioning
    of the discrete operator, and the two paths round differently, so u is
    compared after both have been driven to 1e-12: agreement to 1e-10."""
    desc, punc, og, alpha, beta, g = _setup(name)
    dt, eta = default_dt_eta(og)
    res = g.relax(mode="fp32_dc", tol=1e-10, check_every=50)
    assert res["status"] == 0 and res["norm"] < 1e-10
    u = np.zeros(og.shape)
    g.get_state(u)
    assert og.norm(og.residual(alpha, beta, u)) < 1.02e-10
    uo, vo = og.zeros(), og.zeros()
    it, _, st = og.relax(alpha, beta, uo, vo, eta=eta, dt=dt, tol=1e-10,
                         check_every=50)
    assert st == 0
    assert abs(res["iters"] - it) <= 100, (res, it)
    # (the SinhCylindrical grid's operator is less well conditioned: its two
    # solutions are compared at residual 3e-13)
    tight = 3e-13 if name.startswith("sinhcyl") else 1e-12
    res = g.relax(mode="fp32_dc", tol=tight, check_every=50)
    assert res["status"] == 0
    g.get_state(u)
    _, _, st = og.relax(alpha, beta, uo, vo, eta=eta, dt=dt, tol=tight,
                        check_every=50)
    assert st == 0
    assert rel_err(u, uo) <= 1e-10, rel_err(u, uo)


def test_defect_correction_full_size_matches_fp64(gpu):
    """128x128x16: the defect-correction solve and the FP64 solve agree to
    1e-9 and the oracle re-evaluates the residual of both."""
    desc, punc, og, alpha, beta, g = _setup("sinh_128x128x16_o8")
    r64 = g.relax(mode="fp64", tol=1e-10, check_every=50)
    u64 = np.zeros(og.shape)
    g.get_state(u64)
    rdc = g.relax(mode="fp32_dc", tol=1e-10, check_every=50)
    udc = np.zeros(og.shape)
    g.get_state(udc)
    assert rdc["status"] == 0 and abs(rdc["iters"] - r64["iters"]) <= 100
    assert og.norm(og.residual(alpha, beta, udc)) < 1.02e-10
    assert rel_err(udc, u64) <= 1e-9


def test_multi_stage_tensor_copy_full_size_solves(gpu):
    """128x128x16 with the multi-stage tensor-copy launch in both precisions:
    the FP64 and the defect-correction solves reach the tolerance, confirmed
    by the oracle's residual, in the FP64 solve's number of steps."""
    desc, punc, og, alpha, beta, g = _setup("sinh_128x128x16_o8")
    g.set_launch(2, "fp64", 5)
    g.set_launch(4, "fp32", 5)
    u = np.zeros(og.shape)
    r64 = g.relax(mode="fp64", tol=1e-10, check_every=50)
    g.get_state(u)
    assert r64["status"] == 0 and og.norm(og.residual(alpha, beta, u)) < 1.02e-10
    rdc = g.relax(mode="fp32_dc", tol=1e-10, check_every=50)
    g.get_state(u)
    assert rdc["status"] == 0 and abs(rdc["iters"] - r64["iters"]) <= 100
    assert og.norm(og.residual(alpha, beta, u)) < 1.02e-10


# ------------------------------- stage-kernel variants against the oracle
# Every launch shape must reproduce the oracle; the parity tests above run
# the default shape.  Cartesian variant 1 is the tensor-copy kernel (order 8,
# n0 % 32 == 0, n1 % 4 == 0, even n2); curvilinear variants 1 and 2 are the
# tiled and persistent kernels, variant 3 the tensor-copy tiled kernel and
# variant 4 the multi-stage cooperative kernel and variant 5 its
# tensor-copy tiled form (RK4 steps only; single RHS evaluations use the
# column and the tensor-copy kernels).
VARIANT_CASES = {
    "cart_64x20x24_o8": (W.grid_desc("cartesian", (64, 20, 24), 8, xmax=32.0), Q4),
    "sinh_64x20x8_o8": (W.grid_desc("sinhsymtp", (64, 20, 8), 8), Q4),
    "sph_64x20x8_o8": (W.grid_desc("spherical", (64, 20, 8), 8, rmax=64.0), Q4),
    "sinhsph_64x20x8_o8": (W.grid_desc("sinhspherical", (64, 20, 8), 8), Q4),
    # fewer phi planes than the stencil radius: the phi stencil and the
    # phi + pi images wrap around the whole circle more than once
    "sinh_32x8x2_o8": (W.grid_desc("sinhsymtp", (32, 8, 2), 8), Q4),
    "sph_64x12x4_o8": (W.grid_desc("spherical", (64, 12, 4), 8, rmax=64.0), Q4),
}


@pytest.mark.parametrize("name", list(VARIANT_CASES))
@pytest.mark.parametrize("variant,zc", [(0, 1), (1, 2), (1, 4), (1, 16), (2, 1),
                                        (3, 2), (3, 4), (3, 16), (4, 1), (5, 2),
                                        (5, 16)])
def test_stage_variants_rhs_and_trajectory(gpu, name, variant, zc):
    desc, punc = VARIANT_CASES[name]
    if desc["coord"] == "cartesian" and variant in (2, 4, 5):
        pytest.skip("Cartesian grids have variants 0 and 1")
    og = oracle_grid(desc)
    alpha, beta = og.source(punc)
    g = nrr.Grid(desc)
    g.set_punctures(punc)
    g.set_launch(zc, "fp64", variant)
    g.set_launch(zc, "fp32", variant)
    dt, eta = default_dt_eta(og)
    u = W.smooth_random_field(desc, seed=41, amplitude=0.2, noise=0.01)
    v = W.smooth_random_field(desc, seed=42, amplitude=0.1, noise=0.01)
    ku_o, kv_o = og.rhs(alpha, beta, eta, og.fill_inner_ghosts(u),
                        og.fill_inner_ghosts(v))
    for mode, tol in (("fp64", 1e-12), ("fp32", FP32_RHS_TOL)):
        ku, kv = torch.empty_like(_dev(u)), torch.empty_like(_dev(u))
        g.rhs(_dev(u), _dev(v), ku, kv, eta, mode=mode)
        ku, kv = ku.cpu().numpy(), kv.cpu().numpy()
        for region, m in region_masks(og).items():
            assert rel_err(ku, ku_o, m) <= tol, (mode, region, rel_err(ku, ku_o, m))
            assert rel_err(kv, kv_o, m) <= tol, (mode, region, rel_err(kv, kv_o, m))
    # 30 RK4 steps from a smooth state (all four stage kinds, both fields)
    u = og.fill_inner_ghosts(W.smooth_random_field(desc, seed=43, amplitude=0.1))
    v = og.zeros()
    g.set_state(_dev(u), _dev(v))
    g.step(30, dt, eta, mode="fp64")
    for _ in range(30):
        og.rk4_step(alpha, beta, eta, dt, u, v)
    ug, vg = torch.empty_like(_dev(u)), torch.empty_like(_dev(u))
    g.get_state(ug, vg)
    assert rel_err(ug.cpu().numpy(), u) <= 1e-12
    assert rel_err(vg.cpu().numpy(), v) <= 1e-12
    g.close()


def test_column_kernel_block_sizes_agree(gpu):
    """The column kernel's block size only regroups threads: 32-, 64-,
    128- and 256-thread blocks give bit-identical trajectories in both
    precisions on a grid with ragged tiles."""
    desc = W.grid_desc("sinhsymtp", (44, 26, 6), 8)
    og = oracle_grid(desc)
    dt, eta = default_dt_eta(og)
    u0 = og.fill_inner_ghosts(W.smooth_random_field(desc, seed=61, amplitude=0.1))
    v0 = W.smooth_random_field(desc, seed=62, amplitude=0.05)
    out = {}
    for block in (32, 64, 128, 256):
        g = nrr.Grid(desc)
        g.set_punctures(Q4)
        for mode in ("fp64", "fp32"):
            g.set_launch(1, mode, 0, block)
            g.set_state(_dev(u0), _dev(v0))
            g.step(11, dt, eta, mode=mode)
            ug, vg = torch.empty_like(_dev(u0)), torch.empty_like(_dev(u0))
            g.get_state(ug, vg)
            out[block, mode] = (ug.cpu(), vg.cpu())
        g.close()
    for block in (32, 64, 256):
        for mode in ("fp64", "fp32"):
            assert torch.equal(out[block, mode][0], out[128, mode][0]), (block, mode)
            assert torch.equal(out[block, mode][1], out[128, mode][1]), (block, mode)


@pytest.mark.parametrize("coord,n,zc", [("sinhsymtp", (64, 24, 8), 4),
                                         ("spherical", (64, 32, 8), 2),
                                         ("sinhspherical", (64, 40, 8), 16)])
def test_tensor_copy_tiles_of_8_rows(gpu, coord, n, zc):
    """FP32 tensor-copy stage with 32 x 8 tiles (256-thread blocks): the RHS
    against the oracle, and trajectories bit for bit equal to the 32 x 4
    tiles (the same arithmetic per point; only the tiling differs)."""
    extra = {"rmax": 64.0} if coord == "spherical" else {}
    desc = W.grid_desc(coord, n, 8, **extra)
    og = oracle_grid(desc)
    alpha, beta = og.source(Q4)
    dt, eta = default_dt_eta(og)
    u = W.smooth_random_field(desc, seed=51, amplitude=0.2, noise=0.01)
    v = W.smooth_random_field(desc, seed=52, amplitude=0.1, noise=0.01)
    ku_o, kv_o = og.rhs(alpha, beta, eta, og.fill_inner_ghosts(u),
                        og.fill_inner_ghosts(v))
    out = {}
    for block in (128, 256):
        g = nrr.Grid(desc)
        g.set_punctures(Q4)
        g.set_launch(zc, "fp32", 3, block)
        assert g.get_launch("fp32") == (3, zc, block)
        ku, kv = torch.empty_like(_dev(u)), torch.empty_like(_dev(u))
        g.rhs(_dev(u), _dev(v), ku, kv, eta, mode="fp32")
        ku, kv = ku.cpu().numpy(), kv.cpu().numpy()
        for region, m in region_masks(og).items():
            assert rel_err(ku, ku_o, m) <= FP32_RHS_TOL, (block, region)
            assert rel_err(kv, kv_o, m) <= FP32_RHS_TOL, (block, region)
        g.set_state(_dev(og.fill_inner_ghosts(u)), _dev(v))
        g.step(17, dt, eta, mode="fp32")
        ug, vg = torch.empty_like(_dev(u)), torch.empty_like(_dev(u))
        g.get_state(ug, vg)
        out[block] = (ug.cpu(), vg.cpu(), ku, kv)
        g.close()
    for k in range(4):
        a, b = out[128][k], out[256][k]
        assert (torch.equal(a, b) if isinstance(a, torch.Tensor)
                else np.array_equal(a, b)), k


@pytest.mark.parametrize("n,zc", [((64, 20, 8), 2), ((128, 64, 16), 2),
                                  ((128, 64, 16), 16)])
def test_multi_stage_tensor_copy_equals_single_stage_launches(gpu, n, zc):
    """Variant 5 runs the tensor-copy tile code of variant 3 inside one
    cooperative launch per chunk of steps: the same arithmetic per point, so
    trajectories agree bit for bit in both precisions (the 128 x 64 x 16
    grid at zc = 2 has more tiles than resident blocks, so blocks run
    several tiles per stage)."""
    desc = W.grid_desc("sinhsymtp", n, 8)
    og = oracle_grid(desc)
    dt, eta = default_dt_eta(og)
    u0 = og.fill_inner_ghosts(W.smooth_random_field(desc, seed=44, amplitude=0.1))
    v0 = W.smooth_random_field(desc, seed=45, amplitude=0.05)
    out = {}
    for variant in (3, 5):
        g = nrr.Grid(desc)
        g.set_punctures(Q4)
        for mode in ("fp64", "fp32"):
            g.set_launch(zc, mode, variant)
            g.set_state(_dev(u0), _dev(v0))
            g.step(23, dt, eta, mode=mode)
            ug, vg = torch.empty_like(_dev(u0)), torch.empty_like(_dev(u0))
            g.get_state(ug, vg)
            out[variant, mode] = (ug.cpu(), vg.cpu())
        g.close()
    for mode in ("fp64", "fp32"):
        assert torch.equal(out[3, mode][0], out[5, mode][0]), mode
        assert torch.equal(out[3, mode][1], out[5, mode][1]), mode
    assert torch.isfinite(out[5, "fp32"][0]).all()


def test_cartesian_tensor_copy_variant_full_size(gpu):
    """Cartesian 256^3 (order 8) with the tensor-copy stage: FP64 RHS at every
    point against the oracle."""
    desc, punc = FULL["cart_256x256x256_o8"]
    og = oracle_grid(desc)
    alpha, beta = og.source(punc)
    g = nrr.Grid(desc)
    g.set_punctures(punc)
    g.set_launch(16, "fp64", 1)
    u = W.smooth_random_field(desc, seed=11, amplitude=0.2, noise=0.01)
    v = W.smooth_random_field(desc, seed=12, amplitude=0.1, noise=0.01)
    dt, eta = default_dt_eta(og)
    ku_o, kv_o = og.rhs(alpha, beta, eta, u, v)
    ku, kv = torch.empty_like(_dev(u)), torch.empty_like(_dev(u))
    g.rhs(_dev(u), _dev(v), ku, kv, eta, mode="fp64")
    ku, kv = ku.cpu().numpy(), kv.cpu().numpy()
    for region, m in region_masks(og).items():
        assert rel_err(ku, ku_o, m) <= 1e-12, (region, rel_err(ku, ku_o, m))
        assert rel_err(kv, kv_o, m) <= 1e-12, (region, rel_err(kv, kv_o, m))
    g.close()


def test_loaded_autotune_entry_sets_new_grids_shape(gpu, tmp_path):
    """A grid created after loading a cache entry for its key starts with
    that shape; grids of other keys keep the default."""
    import json
    nrr.autotune_clear()
    (tmp_path / "t.json").write_text(json.dumps({"nrr_autotune": 1, "entries": [
        {"coord": 0, "n": [32, 16, 2], "ng": 2, "fp32": 0, "variant": 1, "zc": 2,
         "block": 128, "pdl": 1}]}))
    nrr.autotune_load(str(tmp_path / "t.json"))
    desc, punc = W.small_equal_mass()
    g = nrr.Grid(desc)
    assert g.get_launch("fp64") == (1, 2, 128)
    g.close()
    g2 = nrr.Grid(W.grid_desc("sinhsymtp", (36, 16, 2), 4))
    assert g2.get_launch("fp64")[0] == 0
    g2.close()
    nrr.autotune_clear()


def test_autotune_picks_caches_and_restores(gpu, tmp_path):
    """nrr_autotune times the candidate launch shapes on the grid, applies
    the fastest, caches it for later grids of the same key (and in a saved
    cache file) and leaves the state it started from; a solve with the tuned
    shapes takes the default shapes' steps to the same u."""
    import json
    import math
    nrr.autotune_clear()
    desc, punc = W.grid_desc("sinhsymtp", (64, 32, 8), 8), Q4
    g0 = nrr.Grid(desc)
    g0.set_punctures(punc)
    r0 = g0.relax(mode="fp64", tol=1e-10)
    u_ref = torch.empty(g0.shape, dtype=torch.float64, device="cuda")
    g0.get_state(u_ref)
    g0.close()

    g = nrr.Grid(desc)
    g.set_punctures(punc)
    u = W.smooth_random_field(desc, seed=5, amplitude=0.1, noise=0.01)
    v = W.smooth_random_field(desc, seed=6, amplitude=0.1, noise=0.01)
    g.set_state(_dev(u), _dev(v))
    before = [torch.empty(g.shape, dtype=torch.float64, device="cuda") for _ in range(2)]
    g.get_state(*before)
    tuned = {}
    for mode in ("fp64", "fp32"):
        var, zc, ms = g.autotune(mode, 3)
        assert ms > 0 and math.isfinite(ms), (mode, ms)
        tuned[mode] = g.get_launch(mode)
        assert tuned[mode][:2] == (var, zc), (mode, tuned[mode], var, zc)
    after = [torch.empty_like(before[0]) for _ in range(2)]
    g.get_state(*after)
    assert torch.equal(before[0], after[0]) and torch.equal(before[1], after[1])

    g2 = nrr.Grid(desc)
    for mode in ("fp64", "fp32"):
        assert g2.get_launch(mode) == tuned[mode], mode
    g2.close()
    nrr.autotune_save(str(tmp_path / "tuned.json"))
    entries = json.loads((tmp_path / "tuned.json").read_text())["entries"]
    for mode, prec in (("fp64", 0), ("fp32", 1)):
        assert any(e["n"] == [64, 32, 8] and e["fp32"] == prec and
                   (e["variant"], e["zc"], e["block"]) == tuned[mode]
                   for e in entries), (mode, entries)

    r = g.relax(mode="fp64", tol=1e-10)
    assert r["iters"] == r0["iters"]
    u_t = torch.empty_like(u_ref)
    g.get_state(u_t)
    assert (u_t - u_ref).abs().max().item() <= 1e-12 * u_ref.abs().max().item()
    g.close()
    nrr.autotune_clear()


TWO_STAGE_CASES = {
    "sinh_32x16x2_o8": (W.grid_desc("sinhsymtp", (32, 16, 2), 8), Q4),
    "sinh_64x32x8_o8": (W.grid_desc("sinhsymtp", (64, 32, 8), 8), Q4),
    "sinh_96x20x16_o8": (W.grid_desc("sinhsymtp", (96, 20, 16), 8),
                         W.equal_mass_pair()),
    "sinh_128x128x16_o8": W.q4_sinhsymtp_128(),
}


@pytest.mark.parametrize("name", list(TWO_STAGE_CASES))
def test_two_stage_kernel_equals_column_kernel(gpu, name):
    """Variant 6 evaluates two RK4 stages per launch (the first on the tile
    with a halo, from shared memory) with the per-stage kernels' arithmetic:
    FP32 trajectories of an odd and an even number of steps, a plain FP32
    solve and a defect-correction solve give the column kernel's states
    bit for bit."""
    desc, punc = TWO_STAGE_CASES[name]
    out = {}
    for variant in (0, 6):
        g = nrr.Grid(desc)
        g.set_punctures(punc)
        g.set_launch(1, "fp32", variant)
        dt, eta = g.timestep(0.5)
        u0 = torch.from_numpy(W.smooth_random_field(desc, seed=51, amplitude=0.1)).cuda()
        res = []
        for steps in (7, 30):
            g.set_state(u0.clone(), torch.zeros_like(u0))
            g.step(steps, dt, eta, mode="fp32")
            u, v = torch.empty_like(u0), torch.empty_like(u0)
            g.get_state(u, v)
            res.append((u, v))
        r32 = g.relax(mode="fp32", tol=1e-5, check_every=50, max_iters=2000,
                      raise_on_error=False)
        u32 = torch.empty_like(u0)
        g.get_state(u32)
        rdc = g.relax(mode="fp32_dc", tol=1e-10, check_every=50)
        udc = torch.empty_like(u0)
        g.get_state(udc)
        out[variant] = (res, r32, u32, rdc, udc)
        g.close()
    (res0, r0, u0_, d0, ud0), (res6, r6, u6, d6, ud6) = out[0], out[6]
    for (a, b), (c, d) in zip(res0, res6):
        assert torch.equal(a, c) and torch.equal(b, d)
    assert r0["iters"] == r6["iters"] and torch.equal(u0_, u6)
    assert d0["status"] == d6["status"] == 0 and d0["iters"] == d6["iters"]
    assert torch.equal(ud0, ud6)


def test_two_stage_kernel_eligibility(gpu):
    g = nrr.Grid(W.grid_desc("sinhsymtp", (64, 32, 8), 8))
    with pytest.raises(nrr.NrrError):
        g.set_launch(1, "fp64", 6)            # FP32 stages only
    g.close()
    for desc in (W.grid_desc("sinhsymtp", (48, 32, 8), 8),     # n0 % 32
                 W.grid_desc("sinhsymtp", (64, 32, 32), 8),    # n2 > 16
                 W.grid_desc("sinhsymtp", (64, 32, 8), 4),     # order
                 W.grid_desc("spherical", (64, 32, 8), 8)):    # family
        g = nrr.Grid(desc)
        with pytest.raises(nrr.NrrError):
            g.set_launch(1, "fp32", 6)
        g.close()
