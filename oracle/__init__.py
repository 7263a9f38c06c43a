"""Plain FP64 CPU oracle for the hyperbolic-relaxation puncture solve.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the
CUDA path: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline leg may import it.  The product library never loads it, and it
shares no code, header, table or constant generator with the CUDA sources.

The arithmetic lives in ``nrr_oracle.c`` (straight loops, FP64, no blocking or
fusion); this module compiles it with gcc and marshals numpy arrays through
ctypes.  Grid functions are numpy arrays of shape ``(s2, s1, s0)`` so that the
flat index is ``i0 + s0*(i1 + s1*i2)``, with ``s_d = n_d + 2*ng``.

Citations refer to arXiv 2501.14030: Sec. 2 (the Hamiltonian constraint for
u, the relaxation system, wave speed proportional to local spacing), Alg. 1
(the RHS -> BC -> RK driver with the residual and its L2 norm), Sec. 4 (centred
finite differences).  Readings of what the paper leaves to its predecessor
(coordinate map, Bowen-York curvature, boundary conditions, eta, c, the norm)
are stated in ``nrr_oracle.c`` beside the code that implements them.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nrr_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

SINHSYMTP, SPHERICAL, CARTESIAN, SINHSPHERICAL, SINHCYLINDRICAL = 0, 1, 2, 3, 4
INTERIOR, OUTER, INNER = 0, 1, 2
CONVERGED, NOT_CONVERGED, DIVERGED = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` with gcc.

    ``-ffp-contract=off`` keeps every multiply and add separately rounded, as
    written; OpenMP only parallelises independent per-point loops.
    """
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
             or os.path.getmtime(_LIB_PATH)
             < os.path.getmtime(os.path.join(_HERE, "nrr_oracle.h")))
    if force or stale:
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
               "-ffp-contract=off", "-Wall", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Desc(C.Structure):
    _fields_ = [("coord", C.c_int), ("n", C.c_int * 3), ("order", C.c_int),
                ("amax", C.c_double), ("bscale", C.c_double),
                ("sinhwaa", C.c_double), ("rmax", C.c_double),
                ("xmax", C.c_double), ("zmax", C.c_double),
                ("sinhwz", C.c_double)]


class Puncture(C.Structure):
    _fields_ = [("m", C.c_double), ("x", C.c_double * 3),
                ("P", C.c_double * 3), ("S", C.c_double * 3)]


class _RelaxParams(C.Structure):
    _fields_ = [("eta", C.c_double), ("dt", C.c_double), ("tol", C.c_double),
                ("r_int", C.c_double), ("max_iters", C.c_long),
                ("check_every", C.c_int)]


class _RelaxResult(C.Structure):
    _fields_ = [("iters", C.c_long), ("norm", C.c_double),
                ("status", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        D = C.POINTER(C.c_double)
        _lib.or_grid_new.restype = C.c_void_p
        _lib.or_grid_new.argtypes = [C.POINTER(_Desc), C.c_char_p, C.c_int]
        _lib.or_grid_free.argtypes = [C.c_void_p]
        _lib.or_grid_info.argtypes = [C.c_void_p, C.POINTER(C.c_int), D]
        _lib.or_grid_field.restype = C.c_void_p
        _lib.or_grid_field.argtypes = [C.c_void_p, C.c_char_p]
        _lib.or_fd_weights.argtypes = [C.c_int, C.c_int, D]
        _lib.or_bowen_york.argtypes = [C.c_int, C.POINTER(Puncture), D, D, D]
        _lib.or_source.argtypes = [C.c_void_p, C.c_int, C.POINTER(Puncture),
                                   D, D]
        _lib.or_fill_inner_ghosts.argtypes = [C.c_void_p, D]
        _lib.or_laplacian.argtypes = [C.c_void_p, D, D]
        _lib.or_rhs.argtypes = [C.c_void_p, D, D, C.c_double, D, D, D, D]
        _lib.or_rk4_step.argtypes = [C.c_void_p, D, D, C.c_double,
                                     C.c_double, D, D]
        _lib.or_residual.argtypes = [C.c_void_p, D, D, D, D]
        _lib.or_residual_norm.restype = C.c_double
        _lib.or_residual_norm.argtypes = [C.c_void_p, D, C.c_double]
        _lib.or_relax.argtypes = [C.c_void_p, D, D, C.POINTER(_RelaxParams),
                                  D, D, C.POINTER(_RelaxResult)]
        _lib.or_linear_coefficient.argtypes = [C.c_void_p, D, D, D, D]
        _lib.or_linear_rhs.argtypes = [C.c_void_p, D, D, C.c_double, D, D,
                                       D, D]
        _lib.or_newton.argtypes = [C.c_void_p, D, D, D, C.c_int, C.c_double,
                                   D]
        _lib.or_grid_set_speed_reference.argtypes = [C.c_void_p, C.c_double]
        L = C.POINTER(C.c_long)
        _lib.or_link_new.restype = C.c_void_p
        _lib.or_link_new.argtypes = [C.c_void_p, C.c_void_p, C.c_int,
                                     C.c_double, C.c_int, C.c_char_p, C.c_int]
        _lib.or_link_free.argtypes = [C.c_void_p]
        _lib.or_link_count.restype = C.c_long
        _lib.or_link_count.argtypes = [C.c_void_p]
        _lib.or_link_get.argtypes = [C.c_void_p, L, L, D]
        _lib.or_link_apply.argtypes = [C.c_void_p, D, D]
        _lib.or_link_conflict.argtypes = [C.c_void_p, C.c_void_p]
        _lib.or_patch_rk4_step.argtypes = [C.c_void_p, D, D, C.c_void_p, D, D,
                                           C.c_void_p, C.c_void_p, C.c_double,
                                           C.c_double, D, D, D, D]
        _lib.or_patch_norm.restype = C.c_double
        _lib.or_patch_norm.argtypes = [C.c_void_p, D, C.c_void_p, C.c_void_p,
                                       D, C.c_void_p, C.c_double]
        _lib.or_patch_relax.argtypes = [C.c_void_p, D, D, C.c_void_p, D, D,
                                        C.c_void_p, C.c_void_p,
                                        C.POINTER(_RelaxParams), D, D, D, D,
                                        C.POINTER(_RelaxResult)]
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(C.POINTER(C.c_double))


def fd_weights(order: int, deriv: int) -> np.ndarray:
    """Centred weights at offsets -order/2..order/2 (Fornberg's recursion)."""
    w = np.zeros(order + 1)
    if lib().or_fd_weights(order, deriv, _dp(w)) != 0:
        raise ValueError("unsupported order/derivative")
    return w


def punctures_to_c(punctures) -> C.Array:
    """``punctures``: sequence of dicts with keys m, x, P, S."""
    arr = (Puncture * max(1, len(punctures)))()
    for i, p in enumerate(punctures):
        arr[i].m = float(p["m"])
        for k in range(3):
            arr[i].x[k] = float(p["x"][k])
            arr[i].P[k] = float(p["P"][k])
            arr[i].S[k] = float(p["S"][k])
    return arr


def bowen_york(punctures, x) -> tuple[float, float]:
    """(A~_ij A~^ij, psi_singular) at Cartesian point x."""
    arr = punctures_to_c(punctures)
    xa = np.ascontiguousarray(x, dtype=np.float64)
    aa = C.c_double()
    ps = C.c_double()
    lib().or_bowen_york(len(punctures), arr, _dp(xa), C.byref(aa),
                        C.byref(ps))
    return aa.value, ps.value


class Grid:
    """One padded grid with its geometry, built by the oracle."""

    def __init__(self, coord: int, n, order: int, amax: float = 1.0e4,
                 bscale: float = 5.0, sinhwaa: float = 0.07,
                 rmax: float = 64.0, xmax: float = 32.0, zmax: float = 1.0e4,
                 sinhwz: float = 0.07):
        d = _Desc(coord, (C.c_int * 3)(*[int(v) for v in n]), int(order),
                  amax, bscale, sinhwaa, rmax, xmax, zmax, sinhwz)
        err = C.create_string_buffer(256)
        h = lib().or_grid_new(C.byref(d), err, 256)
        if not h:
            raise ValueError("oracle grid: " + err.value.decode())
        self._h = h
        self.coord, self.n, self.order = coord, tuple(int(v) for v in n), order
        ints = (C.c_int * 5)()
        dbls = (C.c_double * 7)()
        lib().or_grid_info(h, ints, dbls)
        self.ng = ints[0]
        self.s = (ints[1], ints[2], ints[3])
        self.npts = self.s[0] * self.s[1] * self.s[2]
        self.xxmin = tuple(dbls[0:3])
        self.dxx = tuple(dbls[3:6])
        self.dsmin = dbls[6]
        self.shape = (self.s[2], self.s[1], self.s[0])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_grid_free(h)
            self._h = None

    def field(self, name: str) -> np.ndarray:
        ptr = lib().or_grid_field(self._h, name.encode())
        if not ptr:
            raise KeyError(name)
        if name in ("kind", "image"):
            arr = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(C.c_int)),
                                        (self.npts,))
        else:
            arr = np.ctypeslib.as_array(C.cast(ptr, C.POINTER(C.c_double)),
                                        (self.npts,))
        return arr.reshape(self.shape).copy()

    def zeros(self) -> np.ndarray:
        return np.zeros(self.shape)

    def set_speed_reference(self, ds_ref: float) -> None:
        """c = local spacing / ds_ref (a patch of a multi-patch system)."""
        lib().or_grid_set_speed_reference(self._h, float(ds_ref))
        self.dsmin = float(ds_ref)

    def source(self, punctures):
        alpha, beta = self.zeros(), self.zeros()
        arr = punctures_to_c(punctures)
        lib().or_source(self._h, len(punctures), arr, _dp(alpha), _dp(beta))
        return alpha, beta

    def fill_inner_ghosts(self, f: np.ndarray) -> np.ndarray:
        f = np.ascontiguousarray(f, dtype=np.float64).copy()
        lib().or_fill_inner_ghosts(self._h, _dp(f))
        return f

    def laplacian(self, u):
        out = self.zeros()
        lib().or_laplacian(self._h, _dp(np.ascontiguousarray(u)), _dp(out))
        return out

    def rhs(self, alpha, beta, eta, u, v):
        ku, kv = self.zeros(), self.zeros()
        lib().or_rhs(self._h, _dp(alpha), _dp(beta), float(eta),
                     _dp(np.ascontiguousarray(u)),
                     _dp(np.ascontiguousarray(v)), _dp(ku), _dp(kv))
        return ku, kv

    def linear_coefficient(self, alpha, beta, u):
        a = self.zeros()
        lib().or_linear_coefficient(self._h, _dp(alpha), _dp(beta),
                                    _dp(np.ascontiguousarray(u)), _dp(a))
        return a

    def linear_rhs(self, a, rhat, eta, d, w):
        kd, kw = self.zeros(), self.zeros()
        lib().or_linear_rhs(self._h, _dp(a), _dp(np.ascontiguousarray(rhat)),
                            float(eta), _dp(np.ascontiguousarray(d)),
                            _dp(np.ascontiguousarray(w)), _dp(kd), _dp(kw))
        return kd, kw

    def rk4_step(self, alpha, beta, eta, dt, u, v):
        """One RK4 step in place on (u, v)."""
        lib().or_rk4_step(self._h, _dp(alpha), _dp(beta), float(eta),
                          float(dt), _dp(u), _dp(v))

    def residual(self, alpha, beta, u):
        H = self.zeros()
        lib().or_residual(self._h, _dp(alpha), _dp(beta),
                          _dp(np.ascontiguousarray(u)), _dp(H))
        return H

    def norm(self, H, r_int: float = 100.0) -> float:
        return lib().or_residual_norm(self._h, _dp(np.ascontiguousarray(H)),
                                      float(r_int))

    def relax(self, alpha, beta, u, v, *, eta, dt, tol=1e-10, r_int=100.0,
              max_iters=100000, check_every=1):
        """Relax (u, v) in place; returns (iters, norm, status)."""
        prm = _RelaxParams(float(eta), float(dt), float(tol), float(r_int),
                           int(max_iters), int(check_every))
        res = _RelaxResult()
        lib().or_relax(self._h, _dp(alpha), _dp(beta), C.byref(prm), _dp(u),
                       _dp(v), C.byref(res))
        return res.iters, res.norm, res.status

    def newton(self, alpha, beta, u, max_it=30, step_tol=1e-15):
        """Newton's method in place on u; returns (iterations, last step)."""
        step = C.c_double()
        it = lib().or_newton(self._h, _dp(alpha), _dp(beta), _dp(u),
                             int(max_it), float(step_tol), C.byref(step))
        if it < 0:
            raise RuntimeError("oracle newton failed (%d)" % it)
        return it, step.value


_COORD_NAMES = {"sinhsymtp": SINHSYMTP, "spherical": SPHERICAL,
                "cartesian": CARTESIAN, "sinhspherical": SINHSPHERICAL,
                "sinhcylindrical": SINHCYLINDRICAL}


def grid_from_desc(desc: dict) -> Grid:
    """Oracle grid for a descriptor dict: coord name, n, order and the map
    parameters amax, bscale, sinhwaa, rmax, xmax (and zmax, sinhwz)."""
    return Grid(_COORD_NAMES[desc["coord"]], desc["n"], desc["order"],
                amax=desc["amax"], bscale=desc["bscale"],
                sinhwaa=desc["sinhwaa"], rmax=desc["rmax"], xmax=desc["xmax"],
                zmax=desc.get("zmax", 1.0e4), sinhwz=desc.get("sinhwz", 0.07))


def default_dt_eta(og: Grid, cfl: float = 0.5) -> tuple[float, float]:
    """Time step and damping of the relaxation: dt = cfl * (smallest local
    spacing), so that one step satisfies the CFL limit at every point once
    the wave speed follows the local spacing (Sec. 2); eta dt =
    2 pi cfl / n0, the damping reading (critical damping of the longest
    mode along xx0)."""
    dt = cfl * og.dsmin
    return dt, 2.0 * math.pi * cfl / (og.n[0] * dt)


class Link:
    """Receivers of patch `recv` interpolated from patch `donor` (q-point
    Lagrange interpolation per direction in the donor's coordinates).
    kind 0: every ghost of a Cartesian patch; kind 1: interior points with
    max(|x|, |y|, |z|) < hole."""

    def __init__(self, recv: Grid, donor: Grid, kind: int, hole: float = 0.0,
                 q: int = 4):
        err = C.create_string_buffer(256)
        h = lib().or_link_new(recv._h, donor._h, int(kind), float(hole), int(q),
                              err, 256)
        if not h:
            raise ValueError("oracle link: " + err.value.decode())
        self._h, self.q = h, q
        self.recv_grid, self.donor_grid = recv, donor
        self.n = lib().or_link_count(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_link_free(h)
            self._h = None

    def arrays(self):
        """(receiver flat indices, donor flat indices [n, q^3], weights)."""
        m = self.q ** 3
        recv = np.zeros(self.n, dtype=np.int64)
        donor = np.zeros((self.n, m), dtype=np.int64)
        w = np.zeros((self.n, m))
        lib().or_link_get(self._h, recv.ctypes.data_as(C.POINTER(C.c_long)),
                          donor.ctypes.data_as(C.POINTER(C.c_long)), _dp(w))
        return recv, donor, w

    def apply(self, f_donor: np.ndarray, f_recv: np.ndarray) -> None:
        lib().or_link_apply(self._h, _dp(np.ascontiguousarray(f_donor)),
                            _dp(f_recv))

    def conflicts_with(self, other: "Link") -> bool:
        return bool(lib().or_link_conflict(self._h, other._h))


def patch_rk4_step(a: Grid, src_a, b: Grid, src_b, la: Link, lb: Link, eta,
                   dt, ua, va, ub, vb) -> None:
    """One RK4 step of the two-patch system in place (src_* = (alpha, beta))."""
    lib().or_patch_rk4_step(a._h, _dp(src_a[0]), _dp(src_a[1]), b._h,
                            _dp(src_b[0]), _dp(src_b[1]), la._h, lb._h,
                            float(eta), float(dt), _dp(ua), _dp(va), _dp(ub),
                            _dp(vb))


def patch_norm(a: Grid, Ha, la: Link, b: Grid, Hb, lb: Link,
               r_int: float = 100.0) -> float:
    return lib().or_patch_norm(a._h, _dp(np.ascontiguousarray(Ha)), la._h,
                               b._h, _dp(np.ascontiguousarray(Hb)), lb._h,
                               float(r_int))


def patch_relax(a: Grid, src_a, b: Grid, src_b, la: Link, lb: Link, ua, va,
                ub, vb, *, eta, dt, tol=1e-10, r_int=100.0, max_iters=100000,
                check_every=1):
    """Relax the two-patch system in place; returns (iters, norm, status)."""
    prm = _RelaxParams(float(eta), float(dt), float(tol), float(r_int),
                       int(max_iters), int(check_every))
    res = _RelaxResult()
    lib().or_patch_relax(a._h, _dp(src_a[0]), _dp(src_a[1]), b._h,
                         _dp(src_b[0]), _dp(src_b[1]), la._h, lb._h,
                         C.byref(prm), _dp(ua), _dp(va), _dp(ub), _dp(vb),
                         C.byref(res))
    return res.iters, res.norm, res.status
