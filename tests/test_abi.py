"""The C ABI without a GPU: the library loads, exports every entry point that
include/*.h declares, validates arguments on the host, and its host-side
inner-boundary map agrees with the oracle's Cartesian matching."""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2501_14030_gb300 import nrr, workloads as W
from tests.helpers import oracle_grid

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2501_14030_gb300 import build
    build.build()
    return nrr.lib()


def declared_functions() -> set[str]:
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"\b(nrr_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = declared_functions()
    assert declared, "no declarations found"
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert set(nrr.EXPORTS) <= declared


def test_version_and_defaults(lib):
    assert b"sm_103a" in lib.nrr_version()
    o = nrr.RelaxOpts()
    assert lib.nrr_default_opts(C.byref(o)) == nrr.OK
    assert (o.mode, o.tol, o.check_every, o.cfl, o.r_int) == (
        nrr.FP64, 1e-10, 50, 0.5, 100.0)
    assert lib.nrr_default_opts(None) == nrr.ERR_INVALID_ARG


@pytest.mark.parametrize("bad", [
    dict(coord="sinhsymtp", n=(32, 16, 3), order=4),   # odd n2
    dict(coord="sinhsymtp", n=(32, 16, 2), order=6),   # unsupported order
    dict(coord="sinhsymtp", n=(32, 3, 2), order=8),    # n1 < ng
    dict(coord="spherical", n=(0, 16, 2), order=4),    # empty
    dict(coord="cartesian", n=(1, 16, 16), order=4),   # too small
])
def test_create_grid_rejects_bad_descriptors_on_host(lib, bad):
    desc = W.grid_desc(bad["coord"], bad["n"], bad["order"])
    d = nrr.make_desc(desc)
    h = C.c_void_p()
    st = lib.nrr_create_grid(C.byref(d), None, C.byref(h))
    assert st == nrr.ERR_INVALID_ARG
    assert not h.value
    assert lib.nrr_last_error()


def test_create_grid_rejects_more_than_2_31_points_on_host(lib):
    """The stage kernels index a grid's arrays with 32-bit offsets: a
    padded grid of more than 2^31 points (here 1284^2 x 1404 = 2.31e9, each
    plane well inside 32 bits) is refused before any device call, so this
    runs without a GPU."""
    d = nrr.make_desc(W.grid_desc("cartesian", (1280, 1280, 1400), 4))
    h = C.c_void_p()
    assert lib.nrr_create_grid(C.byref(d), None, C.byref(h)) == nrr.ERR_INVALID_ARG
    assert not h.value
    assert b"2^31" in lib.nrr_last_error()


def test_null_handles_are_rejected(lib):
    assert lib.nrr_relax(None, None, None) == nrr.ERR_INVALID_ARG
    assert lib.nrr_residual(None, 100.0, None, None, 0) == nrr.ERR_INVALID_ARG
    assert lib.nrr_destroy_grid(None) == nrr.OK


@pytest.mark.parametrize("desc", [
    W.grid_desc("sinhsymtp", (32, 16, 2), 4),
    W.grid_desc("sinhsymtp", (44, 26, 6), 8),
    W.grid_desc("sinhsymtp", (20, 5, 4), 10),
    W.grid_desc("spherical", (40, 22, 8), 8, rmax=64.0),
    W.grid_desc("spherical", (12, 6, 2), 10, rmax=9.0),
    W.grid_desc("cartesian", (10, 12, 14), 4),
    W.grid_desc("sinhcylindrical", (20, 12, 8), 8, amax=50.0, sinhwaa=0.3,
                zmax=40.0, sinhwz=0.3),
    W.grid_desc("sinhcylindrical", (9, 7, 4), 4, amax=20.0, sinhwaa=0.5,
                zmax=10.0, sinhwz=0.5),
])
def test_host_image_map_matches_oracle_cartesian_matching(lib, oracle_mod,
                                                          desc):
    og = oracle_grid(desc)
    assert np.array_equal(nrr.image_map(desc), og.field("image"))


def test_bench_names_every_documented_stage_variant():
    """bench.py reports the autotuner's launch shape by name: every
    curvilinear stage variant that nrr_set_launch documents has one."""
    text = open(os.path.join(ROOT, "include", "nrr.h")).read()
    doc = text[text.index("Launch shape of the fused stage kernels"):
               text.index("nrr_status nrr_set_launch(")]
    doc = re.sub(r"\s*\n\s*\*\s*", " ", doc)  # comment lines joined
    documented = {int(v) for v in re.findall(r"variant (\d)", doc)}
    import bench
    assert documented == set(range(7))
    assert documented <= set(bench.STAGE_VARIANTS)


@pytest.mark.parametrize("coord", ["cartesian", "sinhsymtp"])
def test_descriptor_sizes_are_checked_in_64_bits(lib, coord):
    """n0 = n1 = 65536 are each within range, but the padded plane s0*s1
    overflows 32-bit integers.  The descriptor check shared by every entry
    point computes it in 64 bits and rejects the grid on the host, before any
    pointer is used or any device work is queued (the pointers below are
    never dereferenced; this test runs without a GPU)."""
    d = nrr.make_desc(W.grid_desc(coord, (65536, 65536, 2), 4))
    out = (C.c_int32 * 1)()
    assert lib.nrr_image_map(C.byref(d), out) == nrr.ERR_INVALID_ARG
    assert b"s0*s1" in lib.nrr_last_error()
    punc = nrr.make_punctures(W.spinning_q4_pair())
    st = lib.nrr_residual_noalloc(C.byref(d), 2, punc, C.c_void_p(256), 100.0,
                                  C.c_void_p(256), None, None)
    assert st == nrr.ERR_INVALID_ARG
    assert b"s0*s1" in lib.nrr_last_error()


@pytest.mark.parametrize("bad", [
    dict(coord="sinhsymtp", sinhwaa=0.0),
    dict(coord="sinhsymtp", amax=0.0),
    dict(coord="spherical", rmax=0.0),
    dict(coord="cartesian", xmax=0.0),
    dict(coord="sinhspherical"),
])
def test_noalloc_residual_rejects_bad_descriptors_on_host(lib, bad):
    """The allocation-free residual applies the same descriptor check as
    nrr_create_grid (map parameters included) and takes no SinhSpherical
    grid; all of it on the host, before any device call."""
    kw = {k: v for k, v in bad.items() if k != "coord"}
    d = nrr.make_desc(W.grid_desc(bad["coord"], (16, 8, 4), 4, **kw))
    punc = nrr.make_punctures(W.spinning_q4_pair())
    st = lib.nrr_residual_noalloc(C.byref(d), 2, punc, C.c_void_p(256), 100.0,
                                  C.c_void_p(256), None, None)
    assert st == nrr.ERR_INVALID_ARG, lib.nrr_last_error()


def test_noalloc_binding_checks_tensors_before_the_call(lib):
    """The C side gets bare pointers and cannot see the buffers' sizes, so
    the binding refuses a u or h_out that is not a contiguous float64 CUDA
    tensor of exactly s0*s1*s2 elements, and a norm_out that is not float64,
    before anything is passed to the library."""
    import torch
    desc = W.grid_desc("sinhsymtp", (16, 8, 4), 4)
    shape = W.padded_shape(desc)
    good = torch.zeros(shape, dtype=torch.float64)
    norm = torch.zeros(1, dtype=torch.float64)
    cases = [
        (torch.zeros(shape, dtype=torch.float32), norm, None, "float64"),
        (torch.zeros(good.numel() - 1, dtype=torch.float64), norm, None, "elements"),
        (torch.zeros(shape[::-1], dtype=torch.float64).transpose(0, 2), norm,
         None, "contiguous"),
        (good, norm, None, "CUDA"),
        (good, torch.zeros(1, dtype=torch.float32), None, "float64"),
        (good, torch.zeros(0, dtype=torch.float64), None, "elements"),
        (good, norm, torch.zeros(7, dtype=torch.float64), "elements"),
    ]
    for u, n, h, msg in cases:
        with pytest.raises(ValueError, match=msg):
            nrr.residual_noalloc(desc, W.spinning_q4_pair(), u, n, h)


def test_binding_checks_buffers_before_the_call(lib):
    """Every binding call that hands the library a caller's buffer checks
    its type, size, layout and side (host or device) first: the C side gets
    bare pointers.  Objects are built without a GPU (no handle); each call
    below must raise before the library is reached."""
    import types
    import torch
    desc = W.grid_desc("sinhsymtp", (16, 8, 4), 4)
    npts = int(np.prod(W.padded_shape(desc)))
    g = nrr.Grid.__new__(nrr.Grid)
    g._h, g.npts = None, npts
    bad_padded = [
        (np.zeros(npts - 1), "float64 array"),
        (np.zeros(npts, dtype=np.float32), "float64 array"),
        (np.zeros((npts, 2))[:, 0], "float64 array"),
        (torch.zeros(npts, dtype=torch.float32), "float64"),
        (torch.zeros(npts + 1, dtype=torch.float64), "elements"),
    ]
    for a, msg in bad_padded:
        for call in (lambda: g.get_state(a), lambda: g.set_state(a),
                     lambda: g.residual(100.0, a), lambda: g.relax(u0=a)):
            with pytest.raises(ValueError, match=msg):
                call()
    ok = np.zeros(npts)
    frozen = np.zeros(npts)
    frozen.flags.writeable = False
    with pytest.raises(ValueError, match="read-only"):
        g.get_state(frozen)
    # an input may be read-only: the binding passes it on, and the library
    # refuses the stub's null handle
    with pytest.raises(nrr.NrrError, match="null grid"):
        g.set_state(frozen)
    assert nrr._ptr(ok, npts, "u")[1] == 0
    assert nrr._ptr(torch.zeros(npts, dtype=torch.float64), npts, "u")[1] == 0
    with pytest.raises(ValueError, match="CUDA"):
        g.rhs(ok, ok, ok, ok, 1.0)  # the right-hand side takes device arrays

    b = nrr.Batch.__new__(nrr.Batch)
    b._h, b.n = None, 2
    b.shapes = [W.padded_shape(desc)] * 2
    b.interior_points = 2 * 16 * 8 * 4
    with pytest.raises(ValueError, match="solve index"):
        b.get_u(2, ok)
    with pytest.raises(ValueError, match="float64 array"):
        b.set_u(1, np.zeros(npts - 1))
    with pytest.raises(ValueError, match="elements"):
        b.get_interior(torch.zeros(b.interior_points - 1, dtype=torch.float32))

    s = nrr.Surrogate.__new__(nrr.Surrogate)
    s._h, s.dims, s.batch = None, [12, 128, 256], 128
    X, Y = torch.zeros((300, 12)), torch.zeros((300, 256))
    order = torch.zeros(128 * 4, dtype=torch.int32)
    cases = [
        (lambda: s.fit_scaling(torch.zeros((300, 255))), "elements"),
        (lambda: s.fit_scaling(Y.double()), "float32"),
        (lambda: s.train(X, torch.zeros((299, 256)), order, 4), "elements"),
        (lambda: s.train(X, Y, order.long(), 4), "int32"),
        (lambda: s.train(X, Y, order, 5), "elements"),
        (lambda: s.predict(X, torch.zeros((300, 128))), "elements"),
        (lambda: s.gradients(torch.zeros((100, 12)), Y), "elements"),
        (lambda: s.predict(X, torch.zeros((300, 256))), "CUDA"),
    ]
    for call, msg in cases:
        with pytest.raises(ValueError, match=msg):
            call()

    coarse = W.grid_desc("sinhsymtp", (8, 4, 2), 4)
    stream = types.SimpleNamespace(cuda_stream=0)
    uf = torch.zeros(W.padded_shape(desc), dtype=torch.float64)
    with pytest.raises(ValueError, match="elements"):
        nrr.prolong(coarse, torch.zeros(63), desc, uf, stream=stream)
    with pytest.raises(ValueError, match="float64"):
        nrr.prolong(coarse, torch.zeros(64), desc, uf.float(), stream=stream)


@pytest.mark.parametrize("M,N,K,bn,splits", [
    (128, 128, 512, 32, 1),      # tile width not offered
    (128, 128, 512, 256, 1),     # 256 does not divide N
    (128, 192, 512, 128, 0),     # 128 does not divide N
    (128, 128, 512, 128, 9),     # more splits than k-blocks (8)
    (128, 128, 512, 128, -1),
    (100, 128, 512, 0, 0),       # M not a multiple of 128
    (128, 96, 512, 0, 0),        # N not a multiple of 64
    (128, 128, 500, 0, 0),       # K not a multiple of 64
])
def test_gemm_async_rejects_bad_shapes_and_tiles_on_host(lib, M, N, K, bn, splits):
    """Shape, tile-width and split checks happen on the host, before any
    device call (the pointers are never dereferenced)."""
    p = C.c_void_p(1 << 20)
    st = lib.nrr_gemm_bf16_tn_async(p, p, p, M, N, K, bn, splits, -1, None)
    assert st == nrr.ERR_INVALID_ARG, lib.nrr_last_error()


@pytest.mark.parametrize("M,persistent,splits", [(256, 3, 1), (256, -2, 1),
                                                 (256, 1, 4), (256, 2, 4),
                                                 (384, 2, 1)])
def test_gemm_async_rejects_bad_kernel_choice_on_host(lib, M, persistent, splits):
    """persistent -1, 0, 1 or 2; no K split with the persistent kernels; the
    2-CTA clusters take pairs of 128-row tiles (M % 256 == 0)."""
    p = C.c_void_p(1 << 20)
    st = lib.nrr_gemm_bf16_tn_async(p, p, p, M, 256, 4096, 128, splits,
                                    persistent, None)
    assert st == nrr.ERR_INVALID_ARG, lib.nrr_last_error()


def test_release_build_reports_no_address_checks(lib):
    """nrr_debug_check on the release build: checks disabled, nothing
    recorded, no device call needed."""
    en = C.c_int(-1)
    bad = C.c_ulonglong(7)
    cnt = C.c_ulonglong(7)
    assert lib.nrr_debug_check(C.byref(en), C.byref(bad), C.byref(cnt)) == nrr.OK
    assert (en.value, bad.value, cnt.value) == (0, 0, 0)
    assert lib.nrr_debug_check(None, None, None) == nrr.OK
    assert b"NRR_DEBUG" not in lib.nrr_version()
