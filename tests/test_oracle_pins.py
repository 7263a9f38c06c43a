"""Pins of the CPU oracle to facts outside itself (CPU only).

Each test ties one part of the oracle to mathematics the paper's method fixes:
textbook FD weights and polynomial exactness, the FD convergence order on an
analytic function, scale factors against the coordinate map, closed forms of
the Bowen-York contraction, the Cartesian round trip of the inner-boundary
images, symmetries of the physical configuration, the RK4 update on a linear
ODE, the radiation condition on exact profiles, and a brute-force Newton
solve of the discrete steady state.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

from paper_2501_14030_gb300 import workloads as W
from tests.helpers import default_dt_eta, oracle_grid

pytestmark = pytest.mark.usefixtures("oracle_mod")


# ------------------------------------------------------------ FD weights
def _golden_fd_weights():
    """Full stencils (offsets -m..m) from tests/golden/fd_weights_centred.txt
    (Fornberg's table)."""
    from fractions import Fraction
    rows = {}
    path = os.path.join(os.path.dirname(__file__), "golden", "fd_weights_centred.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            order, d, k, w = line.split()
            rows.setdefault((int(order), int(d)), {})[int(k)] = float(Fraction(w))
    out = {}
    for (order, d), wk in rows.items():
        m = order // 2
        sign = -1.0 if d == 1 else 1.0
        out[order, d] = [sign * wk[-k] if k < 0 else wk.get(k, 0.0)
                         for k in range(-m, m + 1)]
    return out


def test_fd_weights_textbook_values(oracle_mod):
    exp = _golden_fd_weights()
    assert len(exp) == 10
    for (order, d), w in exp.items():
        np.testing.assert_allclose(oracle_mod.fd_weights(order, d), w, rtol=0,
                                   atol=1e-14)


@pytest.mark.parametrize("order", [2, 4, 6, 8, 10, 12])
@pytest.mark.parametrize("deriv", [1, 2])
def test_fd_weights_exact_on_polynomials(oracle_mod, order, deriv):
    """sum_k w_k k^j = j! delta_{j,deriv} for every degree the stencil can
    represent (2m+1 nodes: degrees 0..2m)."""
    w = oracle_mod.fd_weights(order, deriv)
    m = order // 2
    k = np.arange(-m, m + 1, dtype=float)
    for j in range(0, order + 1):
        expect = math.factorial(j) if j == deriv else 0.0
        assert abs(np.dot(w, k ** j) - expect) <= 1e-9 * max(1.0, m ** j)


# ------------------------------------------------ FD convergence order
def _gauss(x, y, z, x0=(0.7, -0.4, 1.3), s=2.0):
    d2 = (x - x0[0]) ** 2 + (y - x0[1]) ** 2 + (z - x0[2]) ** 2
    f = np.exp(-d2 / s ** 2)
    return f, f * (4 * d2 / s ** 4 - 6 / s ** 2)


@pytest.mark.parametrize("coord,kw", [
    ("sinhsymtp", dict(amax=40.0, bscale=2.0, sinhwaa=0.4)),
    ("spherical", dict(rmax=12.0)),
    ("cartesian", dict(xmax=8.0)),
    ("sinhspherical", dict(amax=40.0, sinhwaa=0.4)),
    ("sinhcylindrical", dict(amax=20.0, sinhwaa=0.4, zmax=20.0, sinhwz=0.4)),
])
@pytest.mark.parametrize("order", [4, 8])
def test_laplacian_converges_at_fd_order(oracle_mod, coord, kw, order):
    """Discrete flat Laplacian of a Gaussian (ghosts filled analytically)
    against its closed form; error slope between the two finest grids within
    0.4 of the FD order, away from the coordinate axis and origin."""
    errs = []
    for f in (4, 8):
        desc = W.grid_desc(coord, (16 * f, 16 * f, 16 * f), order, **kw)
        g = oracle_grid(desc)
        x, y, z = g.field("x"), g.field("y"), g.field("z")
        u, lap = _gauss(x, y, z)
        L = g.laplacian(u)
        r, rho = g.field("r"), np.hypot(x, y)
        m = (g.field("kind") == 0) & (r < 5) & (r > 1) & (rho > 0.5)
        errs.append(np.abs(L - lap)[m].max())
    slope = math.log2(errs[0] / errs[1])
    assert abs(slope - order) <= 0.4, (errs, slope)


# -------------------------------------- reference metric vs coordinate map
def _d_dxx(f, axis, h):
    """Fourth-order centred derivative along a padded-array axis."""
    return (-np.roll(f, -2, axis) + 8 * np.roll(f, -1, axis)
            - 8 * np.roll(f, 1, axis) + np.roll(f, 2, axis)) / (12 * h)


@pytest.mark.parametrize("desc", [
    W.grid_desc("sinhsymtp", (96, 64, 64), 4),
    W.grid_desc("sinhsymtp", (96, 64, 64), 4, amax=40.0, bscale=2.0,
                sinhwaa=0.4),
    W.grid_desc("spherical", (96, 64, 64), 4, rmax=20.0),
    W.grid_desc("sinhspherical", (96, 64, 64), 4, amax=40.0, sinhwaa=0.4),
    # the strong stretch of SINHWAA 0.07 needs finer xx0 sampling for the
    # fourth-order numerical derivative to resolve J / h0^2
    W.grid_desc("sinhspherical", (192, 64, 64), 4),
    W.grid_desc("sinhcylindrical", (96, 64, 64), 4, amax=20.0, sinhwaa=0.4,
                zmax=20.0, sinhwz=0.4),
])
def test_scale_factors_match_coordinate_map(oracle_mod, desc):
    """h_i = |d(x,y,z)/d xx_i| and g_i = (1/J) d_i (J / h_i^2), by
    differentiating the oracle's own Cartesian positions and J numerically."""
    g = oracle_grid(desc)
    X = [g.field("x"), g.field("y"), g.field("z")]
    h = [g.field("h0"), g.field("h1"), g.field("h2")]
    gl = [g.field("g0"), g.field("g1")]
    J = g.field("jac")
    sl = (slice(3, -3), slice(3, -3), slice(3, -3))
    axes = {0: 2, 1: 1, 2: 0}  # xx_i -> numpy axis of (s2, s1, s0) arrays
    for i in range(3):
        d = [_d_dxx(c, axes[i], g.dxx[i]) for c in X]
        hnum = np.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
        err = np.abs(hnum - np.abs(h[i]))[sl] / np.abs(h[i])[sl]
        assert err.max() < 2e-4, (i, err.max())
    for i in range(2):
        q = J / h[i] ** 2
        gnum = _d_dxx(q, axes[i], g.dxx[i]) / J
        scale = np.abs(gl[i])[sl] + 1.0 / np.abs(h[i] ** 2 * g.dxx[i])[sl]
        err = np.abs(gnum - gl[i])[sl] / scale
        assert err.max() < 2e-4, (i, err.max())


def test_sinhspherical_reduces_to_spherical(oracle_mod):
    """As SINHWAA grows, sinh(xx0/w)/sinh(1/w) -> xx0: SinhSpherical with
    amax = R tends to Spherical with rmax = R, at the rate 1/w^2.  Its xx0 is
    r / R, so h0 and g0 carry the factors R and 1/R of that change of
    variable; r, h1, h2 and g1 agree directly."""
    R = 30.0
    sph = oracle_grid(W.grid_desc("spherical", (12, 10, 4), 4, rmax=R))
    scale = {"r": 1.0, "h0": 1.0 / R, "h1": 1.0, "h2": 1.0, "g0": R, "g1": 1.0}
    diffs = []
    for w in (50.0, 100.0):
        sh = oracle_grid(W.grid_desc("sinhspherical", (12, 10, 4), 4,
                                     amax=R, sinhwaa=w))
        m = sh.field("kind") == 0
        d = max(np.abs(sh.field(f) * k - sph.field(f))[m].max() /
                np.abs(sph.field(f))[m].max() for f, k in scale.items())
        diffs.append(d)
    assert diffs[1] < 1e-4 and 3.5 < diffs[0] / diffs[1] < 4.5, diffs


def test_sinhcylindrical_reduces_to_cylindrical(oracle_mod):
    """As both sinh widths grow, rho -> R xx0 and z -> Z xx1: the scale
    factors tend to the textbook cylindrical ones (R, Z, rho) and the
    Laplacian's first-derivative terms to (1/(rho R), 0), the cylindrical
    d_rho (1/rho) term in the coordinates xx0 = rho/R, at the rate 1/w^2."""
    R, Z = 30.0, 20.0
    diffs = []
    for w in (50.0, 100.0):
        g = oracle_grid(W.grid_desc("sinhcylindrical", (12, 10, 4), 4, amax=R,
                                    sinhwaa=w, zmax=Z, sinhwz=w))
        m = g.field("kind") == 0
        rho, z = R * g.field("xx0"), Z * g.field("xx1")
        expect = {"h0": np.full(g.shape, R), "h1": np.full(g.shape, Z),
                  "h2": rho, "g0": 1.0 / (rho * R),
                  "r": np.hypot(rho, z)}
        d = max(np.abs(g.field(f) - e)[m].max() / np.abs(e)[m].max()
                for f, e in expect.items())
        d = max(d, np.abs(g.field("g1"))[m].max() * Z * Z)
        diffs.append(d)
    assert diffs[1] < 1e-4 and 3.5 < diffs[0] / diffs[1] < 4.5, diffs


def test_sinhsymtp_geometry_closed_forms(oracle_mod):
    """Foci at z = +-bscale (A = 0 segment); b -> 0 reduces to spherical
    geometry with r = A(xx0)."""
    desc = W.grid_desc("sinhsymtp", (16, 16, 4), 4)
    g = oracle_grid(desc)
    # at xx0 -> 0 the coordinate surface collapses onto the focal segment
    xx0, z, x = g.field("xx0"), g.field("z"), g.field("x")
    first = g.ng
    assert np.abs(x[:, :, first]).max() < 1e-2
    assert np.abs(z[:, :, first]).max() <= 5.0 + 1e-2
    gs = oracle_grid(W.grid_desc("sinhsymtp", (16, 16, 4), 4, bscale=0.0))
    r = gs.field("r")
    A = 1e4 * np.sinh(gs.field("xx0") / 0.07) / np.sinh(1 / 0.07)
    kind = gs.field("kind")
    np.testing.assert_allclose(r[kind == 0], np.abs(A)[kind == 0], rtol=1e-13)
    th = gs.field("xx1")
    Ap = 1e4 * np.cosh(gs.field("xx0") / 0.07) / (0.07 * np.sinh(1 / 0.07))
    App = A / 0.07 ** 2
    m = kind == 0
    np.testing.assert_allclose(gs.field("g0")[m],
                               (2 / (A * Ap) - App / Ap ** 3)[m], rtol=1e-10)
    np.testing.assert_allclose(gs.field("g1")[m],
                               (np.cos(th) / (np.sin(th) * A * A))[m],
                               rtol=1e-10)


# ------------------------------------------------------ Bowen-York source
def _single(P=(0, 0, 0), S=(0, 0, 0), m=0.7, x=(0.3, -0.2, 0.5)):
    return [{"m": m, "x": x, "P": P, "S": S}]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bowen_york_closed_forms(oracle_mod, seed):
    """Single puncture: A~A~ = 9P^2(1 + 2 cos^2)/(2 r^4) for momentum,
    18 |S x n|^2 / r^6 for spin, and the cross term 18 P.(S x n)/r^5;
    psi_s = 1 + m/(2r)."""
    rng = np.random.default_rng(seed)
    P = rng.normal(size=3) * 0.2
    S = rng.normal(size=3) * 0.3
    c = np.array([0.3, -0.2, 0.5])
    for _ in range(5):
        X = c + rng.normal(size=3) * 2.0
        d = X - c
        r = np.linalg.norm(d)
        n = d / r
        aa_p, psi = oracle_mod.bowen_york(_single(P=P, x=c), X)
        assert abs(psi - (1 + 0.7 / (2 * r))) < 1e-14
        cos2 = (P @ n) ** 2 / (P @ P)
        assert abs(aa_p - 9 * (P @ P) * (1 + 2 * cos2) / (2 * r ** 4)) <= 1e-12 * aa_p
        aa_s, _ = oracle_mod.bowen_york(_single(S=S, x=c), X)
        sxn = np.cross(S, n)
        assert abs(aa_s - 18 * (sxn @ sxn) / r ** 6) <= 1e-12 * aa_s
        aa_ps, _ = oracle_mod.bowen_york(_single(P=P, S=S, x=c), X)
        cross = 18 * (P @ sxn) / r ** 5
        assert abs(aa_ps - (aa_p + aa_s + cross)) <= 1e-12 * (aa_p + aa_s)


def test_two_punctures_superpose_and_psi(oracle_mod):
    p = W.spinning_q4_pair()
    X = np.array([1.0, 2.0, 0.5])
    _, psi = oracle_mod.bowen_york(p, X)
    r1 = np.linalg.norm(X - np.array(p[0]["x"]))
    r2 = np.linalg.norm(X - np.array(p[1]["x"]))
    assert abs(psi - (1 + 0.8 / (2 * r1) + 0.2 / (2 * r2))) < 1e-14


def test_source_alpha_beta_definition(oracle_mod):
    desc, punc = W.small_equal_mass()
    g = oracle_grid(desc)
    alpha, beta = g.source(punc)
    x, y, z = g.field("x"), g.field("y"), g.field("z")
    idx = [(1, 5, 7), (3, 10, 20), (4, 18, 35)]
    for (a, b, c) in idx:
        aa, psi = oracle_mod.bowen_york(punc, (x[a, b, c], y[a, b, c], z[a, b, c]))
        assert abs(alpha[a, b, c] - 1 / psi) < 1e-15
        assert abs(beta[a, b, c] - aa / (8 * psi ** 7)) <= 1e-14 * abs(beta[a, b, c])


# ----------------------------------------------- inner-boundary images
@pytest.mark.parametrize("desc", [
    W.grid_desc("sinhsymtp", (32, 16, 2), 4),
    W.grid_desc("sinhsymtp", (20, 12, 8), 8),
    W.grid_desc("spherical", (20, 12, 8), 10, rmax=30.0),
    W.grid_desc("sinhspherical", (20, 12, 8), 8),
    W.grid_desc("sinhcylindrical", (20, 12, 8), 8, amax=50.0, sinhwaa=0.3,
                zmax=40.0, sinhwz=0.3),
])
def test_inner_ghost_images_round_trip(oracle_mod, desc):
    O = oracle_mod
    g = oracle_grid(desc)
    kind, img = g.field("kind").ravel(), g.field("image").ravel()
    X = np.stack([g.field(c).ravel() for c in "xyz"])
    inner = np.nonzero(kind == O.INNER)[0]
    assert inner.size > 0
    assert np.all(kind[img[inner]] != O.INNER)
    d = np.abs(X[:, inner] - X[:, img[inner]]).max(axis=0)
    scale = 1 + np.abs(X[:, inner]).max(axis=0)
    assert np.all(d <= 1e-12 * scale)
    ev = np.nonzero(kind != O.INNER)[0]
    assert np.all(img[ev] == ev)


# ---------------------------------------------------------------- RK4
def test_rk4_update_on_linear_ode(oracle_mod):
    """u = u0, v = v0 constant: far from the boundary du/dt = v - eta u,
    dv/dt = 0 (Laplacian of a constant vanishes), so one step must give the
    fourth-degree Taylor polynomial of the exact solution."""
    desc = W.grid_desc("sinhsymtp", (48, 48, 16), 4)
    g = oracle_grid(desc)
    alpha, beta = g.zeros(), g.zeros()
    u0, v0 = 0.3, 0.05
    u, v = np.full(g.shape, u0), np.full(g.shape, v0)
    dt = 0.5 * g.dsmin
    eta = 0.2 / dt
    g.rk4_step(alpha, beta, eta, dt, u, v)
    x = eta * dt
    poly = 1 - x + x ** 2 / 2 - x ** 3 / 6 + x ** 4 / 24
    expect = v0 / eta + (u0 - v0 / eta) * poly
    far = (slice(g.ng + 12, -g.ng - 12), slice(g.ng + 12, -g.ng - 12),
           slice(g.ng + 12, -g.ng - 12))
    sl = (slice(g.ng, -g.ng),) + far[1:]
    assert np.abs(u[sl] - expect).max() < 1e-13
    # the FD Laplacian of a constant is zero up to rounding of its weights
    assert np.abs(v[sl] - v0).max() < 1e-10


# ------------------------------------------------ wave speed and time step
def test_wave_speed_makes_the_local_courant_number_uniform(oracle_mod):
    """Sec. 2: the wave speed is proportional to the local grid spacing, so
    with dt = CFL x (smallest spacing) every interior point runs at the same
    Courant number c dt / ds = CFL.  The spacing is the smallest of
    h_i dxx_i with the textbook spherical scale factors (1, r, r sin theta);
    c is 1 where it is smallest and above 1 elsewhere."""
    O = oracle_mod
    g = oracle_grid(W.grid_desc("spherical", (40, 22, 8), 8, rmax=64.0))
    inner = g.field("kind") == O.INTERIOR
    r, th = g.field("xx0"), g.field("xx1")
    d0, d1, d2 = g.dxx
    ds = np.minimum(np.minimum(d0 * np.ones_like(r), d1 * np.abs(r)),
                    d2 * np.abs(r * np.sin(th)))
    np.testing.assert_allclose(g.field("dsmin")[inner], ds[inner], rtol=1e-13)
    assert g.dsmin == pytest.approx(ds[inner].min(), rel=1e-13)
    # the smallest cell: first radial point next to the axis, h2 dphi
    assert g.dsmin == pytest.approx((d0 / 2) * np.sin(d1 / 2) * d2, rel=1e-12)
    c = g.field("c")[inner]
    assert c.min() == pytest.approx(1.0, rel=1e-14) and (c >= 1.0 - 1e-14).all()
    cfl = 0.5
    np.testing.assert_allclose(c * (cfl * g.dsmin) / ds[inner], cfl, rtol=1e-13)


# ------------------------------------------------ radiation condition
def test_radiation_condition_on_exact_profiles(oracle_mod):
    """Outer ghosts: for f = const the backward difference vanishes and
    df/dt = -c f / r; for f = xx0 it is exactly 1, giving
    -c (1/(dr/dxx0) + xx0/r)."""
    O = oracle_mod
    desc = W.grid_desc("sinhsymtp", (24, 12, 4), 4)
    g = oracle_grid(desc)
    alpha, beta = g.zeros(), g.zeros()
    outer = g.field("kind") == O.OUTER
    c, r, dr, xx0 = g.field("c"), g.field("r"), g.field("drdxx0"), g.field("xx0")
    ku, _ = g.rhs(alpha, beta, 0.0, np.full(g.shape, 0.5), g.zeros())
    np.testing.assert_allclose(ku[outer], (-c * 0.5 / r)[outer], rtol=1e-13)
    ku, _ = g.rhs(alpha, beta, 0.0, xx0.copy(), g.zeros())
    np.testing.assert_allclose(ku[outer], (-c * (1 / dr + xx0 / r))[outer],
                               rtol=1e-11)
    # dr/dxx0 itself against a numerical derivative of r along xx0 (the
    # same formula serves interior and ghost points)
    big = oracle_grid(W.grid_desc("sinhsymtp", (400, 12, 4), 4))
    rb, drb = big.field("r"), big.field("drdxx0")
    inner = (slice(None), slice(big.ng, -big.ng), slice(4, -4))
    dnum = _d_dxx(rb, 2, big.dxx[0])[inner]
    np.testing.assert_allclose(drb[inner], dnum, rtol=1e-4)


def test_cartesian_radiation_condition_on_polynomials(oracle_mod):
    """Cartesian outer ghosts (every ghost of a Cartesian grid):
    d_r f = sum_i (x^i/r) D_i f with D_i one-sided inward (second order)
    along the directions in which the point lies outside, centred otherwise.
    Both second-order differences are exact on polynomials of degree <= 2,
    so for f = const, f = x^i and f = x^2 the condition is exact:
    k = -c f/r, -c (x^i/r + x^i/r), -c (2 x^2/r + x^2/r).  On f = x^3 the
    two stencils differ by known amounts -- one-sided 3x^2 - 2h^2, centred
    3x^2 + h^2 (Taylor expansion) -- which pins which one is used where,
    including edge and corner ghosts that lie outside in y or z only."""
    O = oracle_mod
    g = oracle_grid(W.grid_desc("cartesian", (10, 8, 6), 4, xmax=4.0))
    alpha, beta = g.zeros(), g.zeros()
    outer = g.field("kind") == O.OUTER
    assert outer.sum() == g.npts - 10 * 8 * 6
    c, r = g.field("c"), g.field("r")
    pos = [g.field("x"), g.field("y"), g.field("z")]
    ku, _ = g.rhs(alpha, beta, 0.0, np.full(g.shape, 0.75), g.zeros())
    np.testing.assert_allclose(ku[outer], (-c * 0.75 / r)[outer], rtol=1e-13)
    for i in range(3):
        f = pos[i].copy()
        ku, kv = g.rhs(alpha, beta, 0.0, f, f.copy())
        expect = -c * 2.0 * f / r
        np.testing.assert_allclose(ku[outer], expect[outer], rtol=1e-12,
                                   atol=1e-14)
        np.testing.assert_allclose(kv[outer], expect[outer], rtol=1e-12,
                                   atol=1e-14)
        f = pos[i] ** 2
        ku, _ = g.rhs(alpha, beta, 0.0, f, g.zeros())
        np.testing.assert_allclose(ku[outer], (-c * 3.0 * f / r)[outer],
                                   rtol=1e-12, atol=1e-13)
    # f = x^3: which stencil along x depends on whether the point lies
    # outside the interior range in x (one-sided) or not (centred)
    x, h = pos[0], g.dxx[0]
    i0 = np.broadcast_to(np.arange(g.s[0])[None, None, :], g.shape)
    out_x = (i0 < g.ng) | (i0 >= g.ng + g.n[0])
    Dx = np.where(out_x, 3 * x ** 2 - 2 * h ** 2, 3 * x ** 2 + h ** 2)
    ku, _ = g.rhs(alpha, beta, 0.0, x ** 3, g.zeros())
    expect = -c * (x / r * Dx + x ** 3 / r)
    np.testing.assert_allclose(ku[outer], expect[outer], rtol=1e-11,
                               atol=1e-12)
    # some outer ghosts lie outside only in y or z: their x difference is the
    # centred one
    assert (outer & ~out_x).sum() > 0


def test_sinhcylindrical_radiation_condition(oracle_mod):
    """SinhCylindrical outer ghosts lie beyond the side (rho > amax) or the
    ends (|z| > zmax): d_r f = (rho/r) (1/rho') D_xx0 f + (z/r) (1/z') D_xx1 f,
    each difference one-sided inward where the point lies beyond that
    direction's boundary and centred otherwise.  Exact on profiles linear in
    xx0 or xx1; f = xx1^3 separates the one-sided (3x^2 - 2h^2) from the
    centred (3x^2 + h^2) difference; the classification puts rho < 0 and the
    periodic phi ghosts among the images and everything else beyond the
    boundary among the evolved outer points."""
    O = oracle_mod
    g = oracle_grid(W.grid_desc("sinhcylindrical", (12, 10, 4), 4, amax=20.0,
                                sinhwaa=0.3, zmax=15.0, sinhwz=0.3))
    kind = g.field("kind")
    i0 = np.broadcast_to(np.arange(g.s[0])[None, None, :], g.shape)
    i1 = np.broadcast_to(np.arange(g.s[1])[None, :, None], g.shape)
    i2 = np.broadcast_to(np.arange(g.s[2])[:, None, None], g.shape)
    ng = g.ng
    in1 = (i1 >= ng) & (i1 < ng + g.n[1])
    in2 = (i2 >= ng) & (i2 < ng + g.n[2])
    assert (kind[(i0 < ng) | ~in2] == O.INNER).all()
    outer = kind == O.OUTER
    np.testing.assert_array_equal(
        outer, (i0 >= ng) & in2 & ((i0 >= ng + g.n[0]) | ~in1))
    alpha, beta = g.zeros(), g.zeros()
    c, r, z = g.field("c"), g.field("r"), g.field("z")
    rho = np.hypot(g.field("x"), g.field("y"))
    h0, h1 = g.field("h0"), g.field("h1")
    xx0, xx1 = g.field("xx0"), g.field("xx1")
    ku, _ = g.rhs(alpha, beta, 0.0, np.full(g.shape, 0.5), g.zeros())
    np.testing.assert_allclose(ku[outer], (-c * 0.5 / r)[outer], rtol=1e-13)
    # f = xx1: exact in both stencils along xx1; constant along xx0
    ku, _ = g.rhs(alpha, beta, 0.0, xx1.copy(), g.zeros())
    expect = -c * (z / r / h1 + xx1 / r)
    np.testing.assert_allclose(ku[outer], expect[outer], rtol=1e-12, atol=1e-14)
    # f = xx0 where the xx0 stencil stays at rho > 0 (i0 > ng)
    ku, _ = g.rhs(alpha, beta, 0.0, xx0.copy(), g.zeros())
    expect = -c * (rho / r / h0 + xx0 / r)
    m = outer & (i0 > ng)
    np.testing.assert_allclose(ku[m], expect[m], rtol=1e-12, atol=1e-14)
    # f = xx1^3: one-sided beyond the ends, centred on the side face
    h = g.dxx[1]
    D1 = np.where(in1, 3 * xx1 ** 2 + h ** 2, 3 * xx1 ** 2 - 2 * h ** 2)
    ku, _ = g.rhs(alpha, beta, 0.0, xx1 ** 3, g.zeros())
    expect = -c * (z / r / h1 * D1 + xx1 ** 3 / r)
    np.testing.assert_allclose(ku[outer], expect[outer], rtol=1e-11, atol=1e-13)
    assert (outer & in1).sum() > 0 and (outer & ~in1).sum() > 0


# ------------------------------------------------------------ norm
def test_norm_of_unit_residual_is_one(oracle_mod):
    g = oracle_grid(W.grid_desc("sinhsymtp", (32, 16, 4), 4))
    assert abs(g.norm(np.ones(g.shape)) - 1.0) < 1e-14
    H = np.zeros(g.shape)
    H[g.field("r") >= 100.0] = 7.0
    assert g.norm(H) == 0.0


def test_norm_weights_cells_by_their_volume(oracle_mod):
    """The norm is a volume average: sqrt(sum H^2 J / sum J) over r < r_int
    with J = h0 h1 h2, the reference-metric volume factor.  On a Spherical
    grid (J = r^2 sin(theta)) with H = 1 inside r < R1 and 0 elsewhere it is
    the square root of the volume fraction (R1/R)^3 up to the midpoint rule.
    With unit radial cells and R1 = K1, R = K on cell faces the midpoint sum
    of r^2 over the first K cells is K^3/3 - K/12 exactly, and the theta and
    phi sums cancel in the ratio, so the norm squared is
    (K1^3 - K1/4) / (K^3 - K/4).  An unweighted mean would give K1/K; a
    1/J weight something larger still."""
    K1, K = 10, 40
    g = oracle_grid(W.grid_desc("spherical", (64, 16, 4), 4, rmax=64.0))
    assert g.dxx[0] == 1.0
    r = g.field("r")
    H = np.where(r < K1, 1.0, 0.0)
    nrm = g.norm(H, r_int=float(K))
    exact = math.sqrt((K1 ** 3 - K1 / 4) / (K ** 3 - K / 4))
    assert nrm == pytest.approx(exact, rel=1e-13)
    assert nrm == pytest.approx((K1 / K) ** 1.5, rel=2e-3)
    assert abs(nrm - math.sqrt(K1 / K)) > 0.3
    # the same volume fraction on a SinhSymTP grid (J from its own scale
    # factors), where the cell faces do not fall on r = R1: within the
    # resolution of the shell r = R1
    gs = oracle_grid(W.grid_desc("sinhsymtp", (128, 64, 4), 4, amax=64.0,
                                 bscale=1.0, sinhwaa=0.4))
    rs = gs.field("r")
    nrm = gs.norm(np.where(rs < 8.0, 1.0, 0.0), r_int=24.0)
    assert nrm == pytest.approx((8.0 / 24.0) ** 1.5, rel=0.03)


# ------------------------------------------------- special solutions
def test_brill_lindquist_is_trivial(oracle_mod):
    desc = W.grid_desc("sinhsymtp", (32, 16, 2), 4)
    g = oracle_grid(desc)
    alpha, beta = g.source(W.brill_lindquist_pair())
    assert not beta.any()
    dt, eta = default_dt_eta(g)
    u, v = g.zeros(), g.zeros()
    it, nrm, st = g.relax(alpha, beta, u, v, eta=eta, dt=dt)
    assert (it, nrm, st) == (0, 0.0, 0)
    for _ in range(20):
        g.rk4_step(alpha, beta, eta, dt, u, v)
    assert not u.any() and not v.any()


@pytest.fixture(scope="module")
def equal_mass_solution(oracle_mod):
    desc, punc = W.small_equal_mass()
    g = oracle_grid(desc)
    alpha, beta = g.source(punc)
    dt, eta = default_dt_eta(g)
    u, v = g.zeros(), g.zeros()
    it, nrm, st = g.relax(alpha, beta, u, v, eta=eta, dt=dt, tol=1e-12,
                          check_every=50)
    assert st == 0
    return g, u


def test_equal_mass_mirror_symmetry(equal_mass_solution):
    """The equal-mass configuration is invariant under the rotation by pi
    about y, (x, z) -> (-x, -z), i.e. th -> pi - th, ph -> pi - ph, and under
    y -> -y (ph -> -ph)."""
    g, u = equal_mass_solution
    ng, (n0, n1, n2) = g.ng, g.n
    ui = u[ng:ng + n2, ng:ng + n1, ng:ng + n0]
    j = np.arange(n2)
    rot = ui[(n2 // 2 - 1 - j) % n2][:, ::-1, :]
    scale = np.abs(ui).max()
    assert np.abs(rot - ui).max() <= 1e-13 * scale
    refl = ui[(n2 - 1 - j) % n2]
    assert np.abs(refl - ui).max() <= 1e-13 * scale


def test_axisymmetric_data_gives_phi_independent_u(oracle_mod):
    desc = W.grid_desc("sinhsymtp", (32, 16, 8), 4)
    g = oracle_grid(desc)
    punc = [{"m": 0.6, "x": (0, 0, 5), "P": (0, 0, 0.1), "S": (0, 0, 0.2)},
            {"m": 0.4, "x": (0, 0, -5), "P": (0, 0, -0.1), "S": (0, 0, 0.05)}]
    alpha, beta = g.source(punc)
    dt, eta = default_dt_eta(g)
    u, v = g.zeros(), g.zeros()
    g.relax(alpha, beta, u, v, eta=eta, dt=dt, tol=1e-11, check_every=50)
    ng = g.ng
    ui = u[ng:-ng, ng:-ng, ng:-ng]
    assert np.abs(ui - ui[:1]).max() <= 1e-13 * np.abs(ui).max()


def test_momentum_flip_gives_identical_u(oracle_mod):
    desc, punc = W.small_equal_mass()
    flipped = [dict(p, P=tuple(-c for c in p["P"])) for p in punc]
    g = oracle_grid(desc)
    out = []
    for pp in (punc, flipped):
        alpha, beta = g.source(pp)
        dt, eta = default_dt_eta(g)
        u, v = g.zeros(), g.zeros()
        g.relax(alpha, beta, u, v, eta=eta, dt=dt, tol=1e-10, check_every=50)
        out.append((beta, u))
    assert np.array_equal(out[0][0], out[1][0])
    assert np.array_equal(out[0][1], out[1][1])


# --------------------------------------------------- brute-force Newton
@pytest.mark.parametrize("desc", [
    W.grid_desc("sinhsymtp", (8, 4, 2), 4),
    W.grid_desc("sinhsymtp", (8, 8, 2), 8, amax=20.0, sinhwaa=0.3),
    W.grid_desc("cartesian", (8, 8, 8), 4, xmax=16.0),
    W.grid_desc("sinhspherical", (8, 4, 2), 4, amax=20.0, sinhwaa=0.3),
    W.grid_desc("sinhcylindrical", (6, 8, 2), 4, amax=20.0, sinhwaa=0.3,
                zmax=20.0, sinhwz=0.3),
])
def test_relaxation_agrees_with_dense_newton(oracle_mod, desc):
    """The relaxation's steady state is the solution of the discrete
    nonlinear system that Newton's method finds with a dense LU: after 4000
    RK4 steps (norm at the rounding floor) the two agree to 1e-13."""
    g = oracle_grid(desc)
    punc = W.spinning_q4_pair()
    alpha, beta = g.source(punc)
    un = g.zeros()
    it, step = g.newton(alpha, beta, un, max_it=30, step_tol=1e-15)
    assert it < 30 and step < 1e-15
    dt, eta = default_dt_eta(g)
    u, v = g.zeros(), g.zeros()
    _, nrm, st = g.relax(alpha, beta, u, v, eta=eta, dt=dt, tol=1e-30,
                         r_int=1e30, check_every=1000, max_iters=4000)
    assert nrm < 1e-16, nrm
    assert np.abs(u - un).max() <= 1e-13 * np.abs(un).max()


# -------------------------------------------- defect-correction operator
def test_linearisation_is_the_derivative_of_the_residual(oracle_mod):
    """H(u + e d) - H(u - e d) = 2 e (lap d - a d) + O(e^3): the correction
    equation's coefficient a is minus the derivative of the source term."""
    desc, punc = W.small_equal_mass()
    g = oracle_grid(desc)
    alpha, beta = g.source(punc)
    u = g.fill_inner_ghosts(W.smooth_random_field(desc, seed=5, amplitude=0.1))
    d = g.fill_inner_ghosts(W.smooth_random_field(desc, seed=6, amplitude=0.1))
    a = g.linear_coefficient(alpha, beta, u)
    eps = 1e-4
    fd = (g.residual(alpha, beta, u + eps * d)
          - g.residual(alpha, beta, u - eps * d)) / (2 * eps)
    lin = g.laplacian(d) - a * d
    m = g.field("kind") == 0
    assert np.abs(fd - lin)[m].max() <= 1e-7 * np.abs(lin)[m].max()


def test_linear_rhs_matches_relaxation_rhs_structure(oracle_mod):
    """With a = 0 and rhat = beta (1 + alpha u)^-7 evaluated at u = 0 the
    correction system's RHS at d = 0 equals the nonlinear RHS at u = 0."""
    desc, punc = W.small_equal_mass()
    g = oracle_grid(desc)
    alpha, beta = g.source(punc)
    z = g.zeros()
    ku, kv = g.rhs(alpha, beta, 0.3, z, z)
    kd, kw = g.linear_rhs(z, beta, 0.3, z, z)
    assert np.array_equal(ku, kd)
    np.testing.assert_allclose(kw, kv, rtol=1e-15, atol=0)


# ------------------------------------------------ recorded reference
def test_oracle_matches_its_recorded_reference(oracle_mod):
    """Regression record (not an independent pin): the oracle's relaxation
    of the small equal-mass workload as tests/golden/make_oracle_reference.py
    wrote it.  A change of the oracle's arithmetic must regenerate the file
    and name, in its commit, the passage that justifies it."""
    import importlib.util
    here = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location(
        "make_oracle_reference", os.path.join(here, "make_oracle_reference.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    rec = {}
    samples = {}
    for line in open(os.path.join(here, "oracle_small_equal_mass.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "u":
            samples[tuple(int(x) for x in f[1:4])] = float(f[4])
        else:
            rec[f[0]] = float(f[1])
    iters, norm, status, got = mod.compute()
    assert status == 0 and iters == int(rec["steps"])
    assert norm == pytest.approx(rec["norm"], rel=1e-9)
    assert set(got) == set(samples)
    for k, val in samples.items():
        assert got[k] == pytest.approx(val, rel=1e-11, abs=1e-20), k
