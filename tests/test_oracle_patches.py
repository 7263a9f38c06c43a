"""Pins of the oracle's two-patch coupling (CPU only).

Two overlapping patches (the paper's Sec. 5 multiple patches and Sec. 6
multipatch grids): an inner Cartesian box whose ghost points are
interpolated from an outer patch, and a hole of outer interior points
inside the box interpolated from the box.  Interpolation is the
tensor-product Lagrange polynomial of q points per direction in the donor's
coordinates.  Pinned to:

- polynomial exactness: q-point Lagrange interpolation reproduces every
  polynomial of degree < q in each donor coordinate (Cartesian donor), and
  r^2 = xx0^2 on Spherical, SinhSpherical and SinhSymTP donors (a function
  that is even under the inner-boundary images);
- the weights sum to one;
- when the box's nodes coincide with the outer Cartesian patch's nodes,
  interpolation is injection and the two-patch system is the single-grid
  system: equal trajectories and equal converged solutions;
- the coupled solve of the q=4 pair on a Spherical patch with a Cartesian
  box converges, and its solution agrees with the single Spherical grid's to
  the discretisation error.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_2501_14030_gb300 import workloads as W
from tests.helpers import default_dt_eta, oracle_grid

pytestmark = pytest.mark.usefixtures("oracle_mod")


def _poly(x, y, z):
    """Degree 3 in each coordinate (exact for q = 4)."""
    return (1.0 + 0.3 * x - 0.2 * y ** 2 + 0.05 * z ** 3 + 0.01 * x * y * z
            - 0.002 * x ** 3 * y ** 2 + 0.001 * y ** 3 * z ** 3)


@pytest.mark.parametrize("q", [2, 4, 6])
def test_cartesian_donor_reproduces_polynomials(oracle_mod, q):
    O = oracle_mod
    inner = oracle_grid(W.grid_desc("cartesian", (12, 10, 14), 6, xmax=3.0))
    outer = oracle_grid(W.grid_desc("cartesian", (22, 26, 20), 6, xmax=7.0))
    link = O.Link(inner, outer, 0, q=q)
    assert link.n == inner.npts - 12 * 10 * 14
    recv, donor, w = link.arrays()
    np.testing.assert_allclose(w.sum(axis=1), 1.0, atol=1e-13)
    deg = q - 1
    f = lambda x, y, z: sum(c * x ** i * y ** j * z ** k for (i, j, k), c in {
        (deg, 0, 0): 0.01, (0, deg, 1 if deg else 0): -0.02,
        (1 if deg else 0, 1 if deg else 0, deg): 0.003, (0, 0, 0): 1.0}.items())
    fo = f(outer.field("x"), outer.field("y"), outer.field("z"))
    got = np.zeros(inner.shape)
    link.apply(fo, got)
    expect = f(inner.field("x"), inner.field("y"), inner.field("z")).ravel()[recv]
    np.testing.assert_allclose(got.ravel()[recv], expect, rtol=1e-12, atol=1e-12)
    # a polynomial of degree q in one coordinate is not reproduced
    fo = outer.field("x") ** q
    link.apply(fo, got)
    assert np.abs(got.ravel()[recv] - inner.field("x").ravel()[recv] ** q).max() > 1e-8


@pytest.mark.parametrize("desc", [
    W.grid_desc("spherical", (48, 24, 16), 8, rmax=24.0),
    W.grid_desc("sinhspherical", (48, 24, 16), 8, amax=40.0, sinhwaa=0.4),
    W.grid_desc("sinhsymtp", (48, 24, 16), 8, amax=40.0, bscale=2.0,
                sinhwaa=0.4),
])
def test_curvilinear_donor_reproduces_even_quadratic(oracle_mod, desc):
    """f = xx0^2 is unchanged by the xx0 -> -xx0 image, so stencils that
    reach inner ghosts read their images and still see the polynomial; a
    q = 4 stencil reproduces it exactly, including receivers whose donor
    stencils cross the axis (theta images) and the phi seam."""
    O = oracle_mod
    outer = oracle_grid(desc)
    inner = oracle_grid(W.grid_desc("cartesian", (10, 10, 12), 4, xmax=5.0))
    link = O.Link(inner, outer, 0, q=4)
    recv, donor, w = link.arrays()
    f = outer.field("xx0") ** 2
    got = np.zeros(inner.shape)
    link.apply(f, got)
    xx = np.array([_to_xx(desc, *p) for p in zip(
        inner.field("x").ravel()[recv], inner.field("y").ravel()[recv],
        inner.field("z").ravel()[recv])])
    np.testing.assert_allclose(got.ravel()[recv], xx[:, 0] ** 2, rtol=1e-11,
                               atol=1e-12)
    # the stencils do cross the theta = 0 / pi axis and the phi seam
    kind = outer.field("kind").ravel()
    i1 = (np.arange(outer.npts) // outer.s[0]) % outer.s[1]
    assert np.isin(i1[donor], [outer.ng, outer.ng + outer.n[1] - 1]).any()
    assert (kind[donor] != O.INNER).all()


def _to_xx(desc, x, y, z):
    """xx0 of a Cartesian point, written out per family for the test."""
    rho2 = x * x + y * y
    if desc["coord"] == "spherical":
        return (math.sqrt(rho2 + z * z),)
    if desc["coord"] == "sinhspherical":
        w = desc["sinhwaa"]
        return (w * math.asinh(math.sqrt(rho2 + z * z) * math.sinh(1 / w)
                               / desc["amax"]),)
    b, w = desc["bscale"], desc["sinhwaa"]
    # A^2 is the root of X^2 - (rho^2 + z^2 - b^2) X - rho^2 b^2 = 0
    qq = rho2 + z * z - b * b
    A2 = 0.5 * (qq + math.sqrt(qq * qq + 4 * rho2 * b * b))
    return (w * math.asinh(math.sqrt(A2) * math.sinh(1 / w) / desc["amax"]),)


def _aligned():
    outer = W.grid_desc("cartesian", (32, 32, 32), 4, xmax=16.0)
    inner = W.grid_desc("cartesian", (16, 16, 16), 4, xmax=8.0)
    return outer, inner


def test_aligned_boxes_reduce_to_the_single_grid(oracle_mod):
    """Box nodes on the outer Cartesian nodes (spacing 1 in both): every
    weight is 0 or 1, the box's ghosts copy the outer values and the hole
    copies the box.  The two-patch system is then the single-grid system, so
    30 RK4 steps from the same state give the single grid's trajectory in
    both patches, to rounding."""
    O = oracle_mod
    do, di = _aligned()
    a, b = oracle_grid(do), oracle_grid(di)
    punc = W.spinning_q4_pair()
    sa, sb = a.source(punc), b.source(punc)
    la = O.Link(a, b, 1, hole=5.0, q=4)
    lb = O.Link(b, a, 0, q=4)
    assert la.n == 10 ** 3 and lb.n == 20 ** 3 - 16 ** 3
    assert not la.conflicts_with(lb) and not lb.conflicts_with(la)
    for link in (la, lb):
        w = link.arrays()[2]
        assert set(np.unique(w)) <= {0.0, 1.0}
    dt, eta = default_dt_eta(a)
    u0 = a.fill_inner_ghosts(W.smooth_random_field(do, seed=3, amplitude=0.1))
    ua, va = u0.copy(), a.zeros()
    ub, vb = np.zeros(b.shape), b.zeros()
    sl = (slice(8, 28), slice(8, 28), slice(8, 28))  # box incl. ghosts in a
    ub[...] = u0[sl]
    us, vs = u0.copy(), a.zeros()
    for _ in range(30):
        O.patch_rk4_step(a, sa, b, sb, la, lb, eta, dt, ua, va, ub, vb)
        a.rk4_step(*sa, eta, dt, us, vs)
    scale = np.abs(us).max()
    assert np.abs(ua - us).max() <= 1e-14 * scale
    assert np.abs(ub - us[sl]).max() <= 1e-14 * scale
    assert np.abs(vb - vs[sl]).max() <= 1e-14 * np.abs(vs).max()


def test_aligned_boxes_converge_to_the_single_grid_solution(oracle_mod):
    O = oracle_mod
    do, di = _aligned()
    a, b = oracle_grid(do), oracle_grid(di)
    punc = W.spinning_q4_pair()
    sa, sb = a.source(punc), b.source(punc)
    la, lb = O.Link(a, b, 1, hole=5.0, q=4), O.Link(b, a, 0, q=4)
    dt, eta = default_dt_eta(a)
    ua, va, ub, vb = a.zeros(), a.zeros(), b.zeros(), b.zeros()
    it, nrm, st = O.patch_relax(a, sa, b, sb, la, lb, ua, va, ub, vb, eta=eta,
                                dt=dt, tol=1e-10, check_every=50)
    us, vs = a.zeros(), a.zeros()
    it1, nrm1, st1 = a.relax(*sa, us, vs, eta=eta, dt=dt, tol=1e-10,
                             check_every=50)
    assert st == st1 == 0 and it == it1, (it, it1)
    sl = (slice(8, 28), slice(8, 28), slice(8, 28))
    assert np.abs(ua - us).max() <= 1e-13 * np.abs(us).max()
    assert np.abs(ub - us[sl]).max() <= 1e-13 * np.abs(us).max()


def test_spherical_patch_with_cartesian_box_converges(oracle_mod):
    """The q=4 pair on a Spherical patch with a finer Cartesian box around
    both punctures.  One time step for both patches, the wave speed in each
    the local spacing over the smallest spacing of the two (Sec. 2: c
    proportional to the local spacing), so both run at the same Courant
    number.  The coupled relaxation reaches the 1e-10 residual, no receiver
    is a donor of the other link, and in the overlap the two patches carry
    the same solution up to the interpolation and truncation errors."""
    O = oracle_mod
    a = oracle_grid(W.grid_desc("spherical", (32, 16, 16), 4, rmax=48.0))
    b = oracle_grid(W.grid_desc("cartesian", (24, 24, 24), 4, xmax=8.0))
    ds = min(a.dsmin, b.dsmin)
    assert ds == a.dsmin
    a.set_speed_reference(ds)
    b.set_speed_reference(ds)
    c = b.field("c")
    np.testing.assert_allclose(c, b.dxx[0] / ds, rtol=1e-14)
    punc = W.spinning_q4_pair()
    sa, sb = a.source(punc), b.source(punc)
    la, lb = O.Link(a, b, 1, hole=3.0, q=4), O.Link(b, a, 0, q=4)
    assert not la.conflicts_with(lb) and not lb.conflicts_with(la)
    # a larger hole reaches the outer patch's donor stencils of the box's
    # boundary: the conflict check sees it
    assert O.Link(a, b, 1, hole=5.0, q=4).conflicts_with(lb)
    dt, eta = default_dt_eta(a)
    ua, va, ub, vb = a.zeros(), a.zeros(), b.zeros(), b.zeros()
    it, nrm, st = O.patch_relax(a, sa, b, sb, la, lb, ua, va, ub, vb, eta=eta,
                                dt=dt, tol=1e-10, check_every=50,
                                max_iters=10000)
    assert st == 0 and nrm < 1e-10, (it, nrm, st)
    # overlap (a plausibility check; the exact pins are above): box interior
    # points outside the hole against the sphere patch's values interpolated
    # to them.  The coarse sphere patch (dr = 1.5) does not resolve u near
    # the punctures at z = +-5, so the two differ most there, and far less
    # away from them.
    lk = O.Link(b, a, 1, hole=7.0, q=4)
    back = np.zeros(b.shape)
    lk.apply(ua, back)
    recv = lk.arrays()[0]
    x, y, z = (b.field(c).ravel()[recv] for c in "xyz")
    dist = np.minimum(np.sqrt(x * x + y * y + (z - 5) ** 2),
                      np.sqrt(x * x + y * y + (z + 5) ** 2))
    ring = np.maximum(np.abs(x), np.maximum(np.abs(y), np.abs(z))) > 4.0
    diff = np.abs(back.ravel()[recv] - ub.ravel()[recv])
    near, far = diff[ring & (dist > 1.5)].max(), diff[ring & (dist > 3.5)].max()
    assert far < 5e-3 and far < near / 4, (near, far, np.abs(ub).max())


def test_receivers_stay_interpolated_from_their_donors(oracle_mod):
    """The coupling sets each receiver's right-hand side (u and v) from its
    donor at every RK stage, and RK4 combines stages linearly, so a state
    that starts interpolated stays interpolated: after any number of steps,
    at every receiver of both links, u and v equal the interpolation of the
    donor patch's u and v (to rounding)."""
    O = oracle_mod
    a = oracle_grid(W.grid_desc("spherical", (32, 16, 16), 4, rmax=48.0))
    b = oracle_grid(W.grid_desc("cartesian", (24, 24, 24), 4, xmax=8.0))
    ds = min(a.dsmin, b.dsmin)
    a.set_speed_reference(ds)
    b.set_speed_reference(ds)
    punc = W.spinning_q4_pair()
    sa, sb = a.source(punc), b.source(punc)
    la, lb = O.Link(a, b, 1, hole=3.0, q=4), O.Link(b, a, 0, q=4)
    dt, eta = default_dt_eta(a)
    ua, va, ub, vb = a.zeros(), a.zeros(), b.zeros(), b.zeros()
    for _ in range(20):
        O.patch_rk4_step(a, sa, b, sb, la, lb, eta, dt, ua, va, ub, vb)
    assert np.abs(va).max() > 0 and np.abs(vb).max() > 0
    for link, donor_fields, recv_fields in ((la, (ub, vb), (ua, va)),
                                            (lb, (ua, va), (ub, vb))):
        recv = link.arrays()[0]
        for fd, fr in zip(donor_fields, recv_fields):
            got = np.zeros_like(fr)
            link.apply(fd, got)
            scale = np.abs(fr).max()
            assert np.abs(got.ravel()[recv] - fr.ravel()[recv]).max() <= 1e-13 * scale
