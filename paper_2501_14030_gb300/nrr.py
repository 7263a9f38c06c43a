"""Python binding of libnrr (include/nrr.h): argument marshalling only.

Every step of the solve runs in the CUDA library; this module converts Python
values to the C structs, passes torch tensor pointers (device memory and the
current CUDA stream come from PyTorch) or numpy buffers, and turns status codes
into exceptions.  The library must have been built (``__graft_entry__.build()``
or ``python -m paper_2501_14030_gb300.build``); there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
# NRR_DEBUG=1 in the environment selects the address-checking debug build
# (build.build(debug=True) makes it).
DEBUG = os.environ.get("NRR_DEBUG", "0") not in ("", "0")
LIB_PATH = os.path.join(_HERE, "_build_debug" if DEBUG else "_build",
                        "libnrr_debug.so" if DEBUG else "libnrr.so")

OK, ERR_INVALID_ARG, ERR_OOM, ERR_CUDA = 0, 1, 2, 3
ERR_NOT_CONVERGED, ERR_DIVERGED, ERR_TIMEOUT, ERR_STATE = 4, 5, 6, 7
FP64, FP32, FP32_DC = 0, 1, 2
INIT_ZERO, INIT_CURRENT, INIT_HOST, INIT_DEVICE = 0, 1, 2, 3
MODES = {"fp64": FP64, "fp32": FP32, "fp32_dc": FP32_DC}

# Every entry point declared in include/nrr.h.
EXPORTS = ("nrr_default_opts", "nrr_create_grid", "nrr_destroy_grid",
           "nrr_grid_dims", "nrr_set_punctures", "nrr_relax", "nrr_residual",
           "nrr_get_state", "nrr_set_state", "nrr_rhs", "nrr_step",
           "nrr_timestep", "nrr_image_map", "nrr_profile_stages",
           "nrr_kernel_launches", "nrr_residual_noalloc", "nrr_set_launch",
           "nrr_get_launch", "nrr_selftest_wait_expiry", "nrr_autotune_save",
           "nrr_autotune_load", "nrr_autotune_clear",
           "nrr_set_pdl",
           "nrr_autotune", "nrr_batch_create", "nrr_batch_destroy",
           "nrr_batch_info", "nrr_batch_relax", "nrr_batch_get_u",
           "nrr_batch_autotune", "nrr_batch_set_launch", "nrr_gemm_bf16_tn", "nrr_gemm_bf16_tn_async", "nrr_gemm_status", "nrr_surrogate_create",
           "nrr_surrogate_destroy", "nrr_surrogate_num_params",
           "nrr_surrogate_fit_scaling", "nrr_surrogate_train",
           "nrr_surrogate_predict", "nrr_surrogate_gradients",
           "nrr_surrogate_get_params", "nrr_batch_set_u",
           "nrr_batch_get_interior", "nrr_prolong", "nrr_last_error",
           "nrr_version", "nrr_selftest_recip", "nrr_probe_peaks",
           "nrr_debug_check",
           "nrr_set_device_loop", "nrr_set_speed_reference",
           "nrr_patchset_create", "nrr_patchset_destroy", "nrr_patchset_info",
           "nrr_patchset_timestep", "nrr_patchset_step",
           "nrr_patchset_residual", "nrr_patchset_relax")


class NrrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("nrr status %d: %s" % (status, msg))
        self.status = status


class GridDesc(C.Structure):
    _fields_ = [("coord", C.c_int), ("n", C.c_int * 3), ("fd_order", C.c_int),
                ("amax", C.c_double), ("bscale", C.c_double),
                ("sinhwaa", C.c_double), ("rmax", C.c_double),
                ("xmax", C.c_double), ("zmax", C.c_double),
                ("sinhwz", C.c_double)]


class Puncture(C.Structure):
    _fields_ = [("m", C.c_double), ("x", C.c_double * 3),
                ("P", C.c_double * 3), ("S", C.c_double * 3)]


class RelaxOpts(C.Structure):
    _fields_ = [("mode", C.c_int), ("tol", C.c_double),
                ("max_iters", C.c_int64), ("check_every", C.c_int),
                ("cfl", C.c_double), ("eta", C.c_double),
                ("r_int", C.c_double), ("initial", C.c_int),
                ("u0", C.POINTER(C.c_double)), ("timeout_ms", C.c_int64),
                ("inner_steps", C.c_int64), ("max_outer", C.c_int)]


class RelaxResult(C.Structure):
    _fields_ = [("iters", C.c_int64), ("outer_iters", C.c_int64),
                ("final_norm", C.c_double), ("seconds", C.c_double),
                ("status", C.c_int)]


_lib = None


def lib() -> C.CDLL:
    """Load libnrr.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(
            "%s is missing: build it with __graft_entry__.build()%s"
            % (LIB_PATH, " and build.build(debug=True)" if DEBUG else ""))
    L = C.CDLL(LIB_PATH)
    V, D, I = C.c_void_p, C.POINTER(C.c_double), C.c_int
    sig = {
        "nrr_default_opts": [C.POINTER(RelaxOpts)],
        "nrr_create_grid": [C.POINTER(GridDesc), V, C.POINTER(V)],
        "nrr_destroy_grid": [V],
        "nrr_grid_dims": [V, C.POINTER(C.c_int), C.POINTER(C.c_int),
                          C.POINTER(C.c_int64)],
        "nrr_set_punctures": [V, I, C.POINTER(Puncture)],
        "nrr_relax": [V, C.POINTER(RelaxOpts), C.POINTER(RelaxResult)],
        "nrr_residual": [V, C.c_double, D, V, I],
        "nrr_get_state": [V, V, V, I],
        "nrr_set_state": [V, V, V, I],
        "nrr_rhs": [V, I, C.c_double, V, V, V, V],
        "nrr_step": [V, I, C.c_double, C.c_double, C.c_int64],
        "nrr_timestep": [V, C.c_double, D, D],
        "nrr_image_map": [C.POINTER(GridDesc), C.POINTER(C.c_int32)],
        "nrr_profile_stages": [V, I, C.c_double, C.c_double, C.c_int64, D],
        "nrr_set_launch": [V, I, I, I, I],
        "nrr_get_launch": [V, I, C.POINTER(C.c_int), C.POINTER(C.c_int),
                           C.POINTER(C.c_int)],
        "nrr_set_pdl": [V, I],
        "nrr_set_device_loop": [V, I],
        "nrr_set_speed_reference": [V, C.c_double],
        "nrr_patchset_create": [V, V, C.c_double, I, C.POINTER(V)],
        "nrr_patchset_destroy": [V],
        "nrr_patchset_info": [V, C.POINTER(C.c_int64), C.POINTER(C.c_int64), D],
        "nrr_patchset_timestep": [V, C.c_double, D, D],
        "nrr_patchset_step": [V, C.c_double, C.c_double, C.c_int64],
        "nrr_patchset_residual": [V, C.c_double, D],
        "nrr_patchset_relax": [V, C.POINTER(RelaxOpts), C.POINTER(RelaxResult)],
        "nrr_selftest_wait_expiry": [I, V, C.POINTER(C.c_int)],
        "nrr_autotune_save": [C.c_char_p],
        "nrr_autotune_load": [C.c_char_p],
        "nrr_autotune_clear": [],
        "nrr_autotune": [V, I, C.c_int64, C.POINTER(C.c_int),
                         C.POINTER(C.c_int), D],
        "nrr_batch_create": [I, C.POINTER(GridDesc), C.POINTER(C.c_int),
                             C.POINTER(C.POINTER(Puncture)), I, V,
                             C.POINTER(V)],
        "nrr_batch_destroy": [V],
        "nrr_batch_info": [V, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
        "nrr_batch_relax": [V, C.POINTER(RelaxOpts), C.POINTER(RelaxResult),
                            C.POINTER(RelaxResult)],
        "nrr_batch_get_u": [V, I, V, I],
        "nrr_batch_autotune": [V, I, C.c_int64, C.POINTER(C.c_int), D,
                               C.POINTER(C.c_int)],
        "nrr_batch_set_launch": [V, I, I, I],
        "nrr_gemm_bf16_tn": [V, V, V, I, I, I, V],
        "nrr_gemm_bf16_tn_async": [V, V, V, I, I, I, I, I, I, V],
        "nrr_gemm_status": [V],
        "nrr_surrogate_create": [I, I, I, I, I, C.POINTER(C.c_float), V,
                                 C.POINTER(V)],
        "nrr_surrogate_destroy": [V],
        "nrr_surrogate_fit_scaling": [V, V, C.c_int64],
        "nrr_surrogate_train": [V, V, V, C.c_int64, V, C.c_int64, C.c_double,
                                C.c_double, C.POINTER(C.c_float)],
        "nrr_surrogate_predict": [V, V, C.c_int64, V],
        "nrr_surrogate_gradients": [V, V, V, C.POINTER(C.c_float), D],
        "nrr_surrogate_get_params": [V, C.POINTER(C.c_float)],
        "nrr_batch_set_u": [V, I, V, I],
        "nrr_batch_get_interior": [V, V],
        "nrr_prolong": [C.POINTER(GridDesc), V, C.POINTER(GridDesc), V, V],
        "nrr_residual_noalloc": [C.POINTER(GridDesc), I, C.POINTER(Puncture),
                                 V, C.c_double, V, V, V],
        "nrr_selftest_recip": [V, V, C.c_int64, I, V],
        "nrr_probe_peaks": [C.c_int64, V, D, D, D],
        "nrr_debug_check": [C.POINTER(C.c_int), C.POINTER(C.c_ulonglong),
                            C.POINTER(C.c_ulonglong)],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.nrr_last_error.restype = C.c_char_p
    L.nrr_last_error.argtypes = []
    L.nrr_surrogate_num_params.restype = C.c_int64
    L.nrr_surrogate_num_params.argtypes = [V]
    L.nrr_kernel_launches.restype = C.c_int64
    L.nrr_kernel_launches.argtypes = []
    L.nrr_version.restype = C.c_char_p
    L.nrr_version.argtypes = []
    _lib = L
    return L


def _check(status: int) -> None:
    if status != OK:
        raise NrrError(status, lib().nrr_last_error().decode())


def make_desc(desc: dict) -> GridDesc:
    return GridDesc(workloads.COORDS[desc["coord"]],
                    (C.c_int * 3)(*desc["n"]), int(desc["order"]),
                    float(desc["amax"]), float(desc["bscale"]),
                    float(desc["sinhwaa"]), float(desc["rmax"]),
                    float(desc["xmax"]), float(desc.get("zmax", 1.0e4)),
                    float(desc.get("sinhwz", 0.07)))


def make_punctures(punctures) -> C.Array:
    arr = (Puncture * len(punctures))()
    for i, p in enumerate(punctures):
        arr[i].m = p["m"]
        for k in range(3):
            arr[i].x[k] = p["x"][k]
            arr[i].P[k] = p["P"][k]
            arr[i].S[k] = p["S"][k]
    return arr


def image_map(desc: dict) -> np.ndarray:
    """Inner-boundary image index of every padded point (host computation)."""
    shape = workloads.padded_shape(desc)
    out = np.zeros(shape, dtype=np.int32)
    d = make_desc(desc)
    _check(lib().nrr_image_map(C.byref(d),
                               out.ctypes.data_as(C.POINTER(C.c_int32))))
    return out


def _require_tensor(name: str, t, dtype, numel: int, exact: bool = True,
                    cuda: bool = True) -> None:
    """Raises ValueError unless t is a contiguous torch tensor of `dtype`
    with `numel` elements (at least `numel` if not exact), on the current
    CUDA device if `cuda`.  The C side receives bare pointers and cannot
    check any of this."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise ValueError("%s must be a torch tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s (got %s)" % (name, dtype, t.dtype))
    if (t.numel() != numel) if exact else (t.numel() < numel):
        raise ValueError("%s has %d elements, needs %s%d" % (
            name, t.numel(), "" if exact else "at least ", numel))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if cuda:
        _require_current_device(name, t)


def _require_f64(name: str, t, numel: int, exact: bool) -> None:
    import torch
    _require_tensor(name, t, torch.float64, numel, exact, cuda=False)


def _require_current_device(name: str, t) -> None:
    import torch
    if t.device.type != "cuda":
        raise ValueError("%s must be a CUDA tensor (got %s)" % (name, t.device))
    if t.device.index != torch.cuda.current_device():
        raise ValueError("%s is on cuda:%d, the current device is cuda:%d" % (
            name, t.device.index, torch.cuda.current_device()))


def residual_noalloc(desc: dict, punctures, u, norm_out, h_out=None,
                     r_int: float = 100.0, stream=None) -> None:
    """Residual norm of a device u without device allocation (queued on
    `stream`, default the current torch stream); writes norm_out[0] and,
    if given, H into h_out.  u and h_out: float64, contiguous, exactly
    s0*s1*s2 elements (padded layout); norm_out: float64, >= 1 element; all
    on the current CUDA device.  Checked here, before the call."""
    npts = int(np.prod(workloads.padded_shape(desc)))
    tensors = [("u", u, npts, True), ("norm_out", norm_out, 1, False)]
    if h_out is not None:
        tensors.append(("h_out", h_out, npts, True))
    for name, t, n, exact in tensors:
        _require_f64(name, t, n, exact)
    for name, t, _, _ in tensors:
        _require_current_device(name, t)
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    d = make_desc(desc)
    arr = make_punctures(punctures)
    h = C.c_void_p(h_out.data_ptr()) if h_out is not None else None
    _check(lib().nrr_residual_noalloc(
        C.byref(d), len(punctures), arr, C.c_void_p(u.data_ptr()), r_int,
        C.c_void_p(norm_out.data_ptr()), h, C.c_void_p(stream.cuda_stream)))


def selftest_recip(s, out, stream=None) -> None:
    """out = the stage kernels' reciprocal of s (float64 or float32 CUDA
    tensors of one size and type)."""
    import torch
    if s.dtype != out.dtype or s.numel() != out.numel():
        raise ValueError("s and out need one dtype and size")
    if s.dtype not in (torch.float64, torch.float32) or not (
            s.is_cuda and out.is_cuda and s.is_contiguous() and out.is_contiguous()):
        raise ValueError("contiguous float64/float32 CUDA tensors expected")
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().nrr_selftest_recip(C.c_void_p(s.data_ptr()),
                                    C.c_void_p(out.data_ptr()), s.numel(),
                                    int(s.dtype == torch.float32),
                                    C.c_void_p(stream.cuda_stream)))


def probe_peaks(l2_bytes: int = 0, stream=None) -> dict:
    """Measured FP64/FP32 FMA throughput (TFLOP/s) and L2 read bandwidth
    (GB/s) of the current GPU, from this library's probe kernels."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    f64, f32, l2 = C.c_double(), C.c_double(), C.c_double()
    _check(lib().nrr_probe_peaks(int(l2_bytes), C.c_void_p(stream.cuda_stream),
                                 C.byref(f64), C.byref(f32), C.byref(l2)))
    return {"fp64_tflops": f64.value, "fp32_tflops": f32.value,
            "l2_gbs": l2.value}


def _gemm_shape(A, B, D):
    import torch
    for t in (A, B):
        if t.dtype != torch.bfloat16 or t.dim() != 2 or not t.is_contiguous():
            raise NrrError(ERR_INVALID_ARG, "gemm operands: contiguous 2-D bfloat16")
    if D.dtype != torch.float32 or not D.is_contiguous():
        raise NrrError(ERR_INVALID_ARG, "gemm output: contiguous float32")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K or tuple(D.shape) != (M, N):
        raise NrrError(ERR_INVALID_ARG, "gemm: shapes A (M, K), B (N, K), D (M, N)")
    return M, N, K


def gemm_bf16_tn(A, B, D, stream=None) -> None:
    """D (float32, M x N) = A (bf16, M x K) @ B (bf16, N x K)^T on device;
    synchronous, raises on a pipeline timeout."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    M, N, K = _gemm_shape(A, B, D)
    _check(lib().nrr_gemm_bf16_tn(C.c_void_p(A.data_ptr()),
                                  C.c_void_p(B.data_ptr()),
                                  C.c_void_p(D.data_ptr()), M, N, K,
                                  C.c_void_p(stream.cuda_stream)))


def gemm_bf16_tn_async(A, B, D, bn=0, splits=0, persistent=-1, stream=None) -> None:
    """The same product only enqueued; bn / splits 0 and persistent -1 =
    chosen from the shape.  Check with gemm_status()."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    M, N, K = _gemm_shape(A, B, D)
    _check(lib().nrr_gemm_bf16_tn_async(C.c_void_p(A.data_ptr()),
                                        C.c_void_p(B.data_ptr()),
                                        C.c_void_p(D.data_ptr()), M, N, K,
                                        int(bn), int(splits), int(persistent),
                                        C.c_void_p(stream.cuda_stream)))


def debug_check() -> dict:
    """Address-check record of the debug build since the previous call:
    {"enabled", "first_bad", "refused"} (enabled False for the release
    build)."""
    en = C.c_int(0)
    bad = C.c_ulonglong(0)
    cnt = C.c_ulonglong(0)
    _check(lib().nrr_debug_check(C.byref(en), C.byref(bad), C.byref(cnt)))
    return {"enabled": bool(en.value), "first_bad": bad.value, "refused": cnt.value}


def gemm_status(stream=None) -> None:
    """Wait for the stream and raise if a GEMM pipeline wait expired."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().nrr_gemm_status(C.c_void_p(stream.cuda_stream)))


def prolong(coarse: dict, uc, fine: dict, uf, stream=None) -> None:
    """Trilinear prolongation of coarse interior u (float32 tensor) onto the
    padded fine grid (float64 tensor)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    dc, df = make_desc(coarse), make_desc(fine)
    _require_tensor("uc", uc, torch.float32, int(np.prod(coarse["n"])), cuda=False)
    _require_tensor("uf", uf, torch.float64,
                    int(np.prod(workloads.padded_shape(fine))), cuda=False)
    _require_current_device("uc", uc)
    _require_current_device("uf", uf)
    _check(lib().nrr_prolong(C.byref(dc), C.c_void_p(uc.data_ptr()), C.byref(df),
                             C.c_void_p(uf.data_ptr()),
                             C.c_void_p(stream.cuda_stream)))


def kernel_launches() -> int:
    """Kernels launched by libnrr so far in this process."""
    return int(lib().nrr_kernel_launches())


def _ptr(x, numel: int, name: str = "array", out: bool = False):
    """(pointer, on_device) of a padded FP64 array: a C-contiguous float64
    numpy array (writable if `out`), or a contiguous float64 torch tensor
    (on the current device if on a GPU), with exactly `numel` elements.
    Checked here: the C side receives the bare pointer."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags["C_CONTIGUOUS"] or x.size != numel:
            raise ValueError("%s must be a C-contiguous float64 array of %d "
                             "elements (got %s, %d)" % (name, numel, x.dtype, x.size))
        if out and not x.flags["WRITEABLE"]:
            raise ValueError("%s is read-only" % name)
        return C.c_void_p(x.ctypes.data), 0
    import torch
    _require_tensor(name, x, torch.float64, numel, cuda=False)
    if x.is_cuda:
        _require_current_device(name, x)
    return C.c_void_p(x.data_ptr()), int(x.is_cuda)


class Grid:
    """One grid on the current CUDA device, driven through the C ABI."""

    def __init__(self, desc: dict, stream=None):
        import torch
        self.desc = dict(desc)
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        handle = C.c_void_p()
        d = make_desc(desc)
        _check(lib().nrr_create_grid(C.byref(d), C.c_void_p(stream.cuda_stream),
                                     C.byref(handle)))
        self._h = handle
        s = (C.c_int * 3)()
        ng = C.c_int()
        ni = C.c_int64()
        _check(lib().nrr_grid_dims(handle, s, C.byref(ng), C.byref(ni)))
        self.s = (s[0], s[1], s[2])
        self.ng = ng.value
        self.interior_points = ni.value
        self.shape = (s[2], s[1], s[0])
        self.npts = s[0] * s[1] * s[2]

    def close(self):
        if getattr(self, "_h", None):
            lib().nrr_destroy_grid(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_punctures(self, punctures):
        arr = make_punctures(punctures)
        _check(lib().nrr_set_punctures(self._h, len(punctures), arr))

    def timestep(self, cfl: float = 0.5):
        dt, eta = C.c_double(), C.c_double()
        _check(lib().nrr_timestep(self._h, cfl, C.byref(dt), C.byref(eta)))
        return dt.value, eta.value

    def relax(self, mode="fp64", tol=1e-10, max_iters=1_000_000,
              check_every=50, cfl=0.5, eta=0.0, r_int=100.0, initial=None,
              u0=None, timeout_ms=0, inner_steps=0, max_outer=0,
              raise_on_error=True) -> dict:
        o = RelaxOpts()
        _check(lib().nrr_default_opts(C.byref(o)))
        o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        o.tol, o.max_iters, o.check_every = tol, max_iters, check_every
        o.cfl, o.eta, o.r_int = cfl, eta, r_int
        o.timeout_ms, o.inner_steps, o.max_outer = timeout_ms, inner_steps, max_outer
        if u0 is not None:
            p, on_dev = _ptr(u0, self.npts, "u0")
            o.initial = INIT_DEVICE if on_dev else INIT_HOST
            o.u0 = C.cast(p, C.POINTER(C.c_double))
        else:
            o.initial = INIT_ZERO if initial is None else int(initial)
        r = RelaxResult()
        st = lib().nrr_relax(self._h, C.byref(o), C.byref(r))
        if raise_on_error:
            _check(st)
        return {"iters": r.iters, "outer_iters": r.outer_iters,
                "norm": r.final_norm, "seconds": r.seconds, "status": st}

    def residual(self, r_int: float = 100.0, h_out=None) -> float:
        nrm = C.c_double()
        if h_out is None:
            _check(lib().nrr_residual(self._h, r_int, C.byref(nrm), None, 0))
        else:
            p, on_dev = _ptr(h_out, self.npts, "h_out", out=True)
            _check(lib().nrr_residual(self._h, r_int, C.byref(nrm), p, on_dev))
        return nrm.value

    def _pair(self, u, v, names, out=False):
        """Pointers of u and (nullable) v, both padded FP64 arrays of this
        grid on the same side (host or device)."""
        pu, on_dev = _ptr(u, self.npts, names[0], out)
        if v is None:
            return pu, None, on_dev
        pv, on_dev_v = _ptr(v, self.npts, names[1], out)
        if on_dev_v != on_dev:
            raise ValueError("%s and %s must both be on the host or both on "
                             "the device" % names)
        return pu, pv, on_dev

    def get_state(self, u_out, v_out=None):
        pu, pv, on_dev = self._pair(u_out, v_out, ("u_out", "v_out"), out=True)
        _check(lib().nrr_get_state(self._h, pu, pv, on_dev))

    def set_state(self, u, v=None):
        pu, pv, on_dev = self._pair(u, v, ("u", "v"))
        _check(lib().nrr_set_state(self._h, pu, pv, on_dev))

    def rhs(self, u, v, ku, kv, eta: float, mode="fp64"):
        """ku, kv = the relaxation right-hand side at (u, v): padded FP64
        device tensors."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        ptrs = []
        for name, t in (("u", u), ("v", v), ("ku", ku), ("kv", kv)):
            p, on_dev = _ptr(t, self.npts, name)
            if not on_dev:
                raise ValueError("%s must be a CUDA tensor" % name)
            ptrs.append(p)
        _check(lib().nrr_rhs(self._h, m, eta, *ptrs))

    def profile_stages(self, steps: int, dt: float, eta: float,
                       mode="fp64") -> float:
        """Average ms of one fused stage launch over `steps` RK4 steps,
        timed with CUDA events on the library's work stream."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        ms = C.c_double()
        _check(lib().nrr_profile_stages(self._h, m, dt, eta, int(steps),
                                        C.byref(ms)))
        return ms.value

    def set_launch(self, zc: int, mode="fp64", variant: int = 0, block: int = 0):
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        _check(lib().nrr_set_launch(self._h, m, int(variant), int(zc), int(block)))

    def get_launch(self, mode="fp64"):
        """(variant, zc, block) of the stage kernels for `mode`."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        v, z, bl = C.c_int(), C.c_int(), C.c_int()
        _check(lib().nrr_get_launch(self._h, m, C.byref(v), C.byref(z), C.byref(bl)))
        return v.value, z.value, bl.value

    def set_pdl(self, on: bool):
        """Programmatic dependent launch of the stage kernels (default on)."""
        _check(lib().nrr_set_pdl(self._h, int(bool(on))))

    def set_speed_reference(self, ds_ref: float):
        """Wave speed = local spacing / ds_ref (a patch of a multi-patch
        system)."""
        _check(lib().nrr_set_speed_reference(self._h, float(ds_ref)))

    def set_device_loop(self, on: bool):
        """Stop test on the device, one graph launch per solve (default on),
        or one host read of the norm per chunk (off)."""
        _check(lib().nrr_set_device_loop(self._h, int(bool(on))))

    def autotune(self, mode="fp64", trial_steps: int = 20):
        """Pick the fastest stage kernel and launch shape; returns
        (variant, zc, ms/launch)."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        var, zc, ms = C.c_int(), C.c_int(), C.c_double()
        _check(lib().nrr_autotune(self._h, m, int(trial_steps), C.byref(var),
                                  C.byref(zc), C.byref(ms)))
        return var.value, zc.value, ms.value

    def step(self, steps: int, dt: float, eta: float, mode="fp64"):
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        _check(lib().nrr_step(self._h, m, dt, eta, int(steps)))


class PatchSet:
    """An outer grid and an inner Cartesian box relaxed as one system
    (receivers interpolated from the other patch).  The grids stay owned by
    the caller and must outlive the patch set."""

    def __init__(self, outer: "Grid", inner: "Grid", hole: float, q: int = 4):
        h = C.c_void_p()
        _check(lib().nrr_patchset_create(outer._h, inner._h, float(hole), int(q),
                                         C.byref(h)))
        self._h = h
        self.outer, self.inner = outer, inner
        no, ni, ds = C.c_int64(), C.c_int64(), C.c_double()
        _check(lib().nrr_patchset_info(h, C.byref(no), C.byref(ni), C.byref(ds)))
        self.outer_receivers, self.inner_receivers = no.value, ni.value
        self.ds_ref = ds.value

    def close(self):
        if getattr(self, "_h", None):
            lib().nrr_patchset_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def timestep(self, cfl: float = 0.5):
        dt, eta = C.c_double(), C.c_double()
        _check(lib().nrr_patchset_timestep(self._h, cfl, C.byref(dt), C.byref(eta)))
        return dt.value, eta.value

    def step(self, steps: int, dt: float, eta: float):
        _check(lib().nrr_patchset_step(self._h, dt, eta, int(steps)))

    def residual(self, r_int: float = 100.0) -> float:
        n = C.c_double()
        _check(lib().nrr_patchset_residual(self._h, r_int, C.byref(n)))
        return n.value

    def relax(self, tol=1e-10, max_iters=1_000_000, check_every=50, cfl=0.5,
              eta=0.0, r_int=100.0, initial=None, timeout_ms=0, mode="fp64",
              inner_steps=0, max_outer=0, raise_on_error=True) -> dict:
        """mode "fp64", or "fp32_dc" (FP32 increments of both patches inside
        the FP64 defect correction, one outer iteration per inner_steps
        steps, default check_every)."""
        o = RelaxOpts()
        _check(lib().nrr_default_opts(C.byref(o)))
        o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        o.tol, o.max_iters, o.check_every = tol, max_iters, check_every
        o.cfl, o.eta, o.r_int, o.timeout_ms = cfl, eta, r_int, timeout_ms
        o.inner_steps, o.max_outer = inner_steps, max_outer
        o.initial = INIT_ZERO if initial is None else int(initial)
        r = RelaxResult()
        st = lib().nrr_patchset_relax(self._h, C.byref(o), C.byref(r))
        if raise_on_error:
            _check(st)
        return _result(r, st)


def _result(r: RelaxResult, st: int | None = None) -> dict:
    return {"iters": r.iters, "outer_iters": r.outer_iters,
            "norm": r.final_norm, "seconds": r.seconds,
            "status": r.status if st is None else st}


class Batch:
    """Independent solves of uneven sizes relaxed together on the current
    CUDA device (one graph launch per relaxation)."""

    def __init__(self, descs, punctures, with_fp64: bool = False,
                 stream=None):
        import torch
        n = len(descs)
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        self.descs = [dict(d) for d in descs]
        self.n = n
        self.shapes = [workloads.padded_shape(d) for d in descs]
        d_arr = (GridDesc * n)(*[make_desc(d) for d in descs])
        self._punc = [make_punctures(p) for p in punctures]
        np_arr = (C.c_int * n)(*[len(p) for p in punctures])
        pp = (C.POINTER(Puncture) * n)(*[C.cast(a, C.POINTER(Puncture))
                                         for a in self._punc])
        h = C.c_void_p()
        _check(lib().nrr_batch_create(n, d_arr, np_arr, pp, int(with_fp64),
                                      C.c_void_p(stream.cuda_stream),
                                      C.byref(h)))
        self._h = h
        tp, ip = C.c_int64(), C.c_int64()
        _check(lib().nrr_batch_info(h, C.byref(tp), C.byref(ip)))
        self.total_points, self.interior_points = tp.value, ip.value

    def close(self):
        if getattr(self, "_h", None):
            lib().nrr_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def relax(self, mode="fp32_dc", tol=1e-10, max_iters=1_000_000,
              check_every=50, cfl=0.5, eta=0.0, r_int=100.0, initial=None,
              timeout_ms=0, inner_steps=0, raise_on_error=True):
        """Returns (per-solve result dicts, total result dict)."""
        o = RelaxOpts()
        _check(lib().nrr_default_opts(C.byref(o)))
        o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
        o.tol, o.max_iters, o.check_every = tol, max_iters, check_every
        o.cfl, o.eta, o.r_int = cfl, eta, r_int
        o.initial = INIT_ZERO if initial is None else int(initial)
        o.timeout_ms, o.inner_steps = timeout_ms, inner_steps
        per = (RelaxResult * self.n)()
        tot = RelaxResult()
        st = lib().nrr_batch_relax(self._h, C.byref(o), per, C.byref(tot))
        if raise_on_error:
            _check(st)
        return [_result(r) for r in per], _result(tot, st)

    def _solve_npts(self, i: int) -> int:
        if not 0 <= int(i) < self.n:
            raise ValueError("solve index %d outside [0, %d)" % (i, self.n))
        return int(np.prod(self.shapes[int(i)]))

    def get_u(self, i: int, out):
        p, on_dev = _ptr(out, self._solve_npts(i), "out", out=True)
        _check(lib().nrr_batch_get_u(self._h, int(i), p, on_dev))

    def set_u(self, i: int, u):
        p, on_dev = _ptr(u, self._solve_npts(i), "u")
        _check(lib().nrr_batch_set_u(self._h, int(i), p, on_dev))

    def get_interior(self, out):
        """Interior u of every solve (equal sizes) into a float32 CUDA
        tensor of all the solves' interior points."""
        import torch
        _require_tensor("out", out, torch.float32, self.interior_points)
        _check(lib().nrr_batch_get_interior(self._h, C.c_void_p(out.data_ptr())))

    def set_launch(self, variant: int, zc: int, mode="fp32_dc"):
        """Stage kernel of the batch: variant 0 (register-staged planes) or
        1 (bulk-copy plane ring), zc phi planes per block chunk."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        _check(lib().nrr_batch_set_launch(self._h, m, int(variant), int(zc)))

    def autotune(self, mode="fp32_dc", trial_steps: int = 5):
        """Pick the fastest stage kernel; returns (zc, ms/launch, variant)."""
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        zc, ms, var = C.c_int(), C.c_double(), C.c_int()
        _check(lib().nrr_batch_autotune(self._h, m, int(trial_steps),
                                        C.byref(zc), C.byref(ms), C.byref(var)))
        return zc.value, ms.value, var.value


class Surrogate:
    """The warm-start network on the current CUDA device."""

    def __init__(self, dims, init_params: np.ndarray, batch: int = 256,
                 stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self._stream = stream
        self.dims = list(dims)
        n_in, hidden, depth, n_out = dims[0], dims[1], len(dims) - 2, dims[-1]
        self.batch = batch
        p = np.ascontiguousarray(init_params, dtype=np.float32)
        h = C.c_void_p()
        _check(lib().nrr_surrogate_create(
            n_in, hidden, depth, n_out, batch,
            p.ctypes.data_as(C.POINTER(C.c_float)),
            C.c_void_p(stream.cuda_stream), C.byref(h)))
        self._h = h
        self.num_params = int(lib().nrr_surrogate_num_params(h))
        assert self.num_params == p.size

    def close(self):
        if getattr(self, "_h", None):
            lib().nrr_surrogate_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _rows(self, name, t, width, rows=None, exact=True):
        """Rows of a contiguous float32 tensor [rows][width] (rows from t);
        the device is checked by _on_device once every shape has been."""
        import torch
        n = int(t.shape[0]) if rows is None and getattr(t, "ndim", 0) >= 1 else rows
        _require_tensor(name, t, torch.float32, (n or 0) * width, exact, cuda=False)
        return n

    @staticmethod
    def _on_device(**tensors):
        for name, t in tensors.items():
            _require_current_device(name, t)

    def fit_scaling(self, Y):
        n = self._rows("Y", Y, self.dims[-1])
        self._on_device(Y=Y)
        _check(lib().nrr_surrogate_fit_scaling(self._h, C.c_void_p(Y.data_ptr()), n))

    def train(self, X, Y, order, steps: int, lr: float = 1e-3,
              weight_decay: float = 0.0) -> np.ndarray:
        import torch
        n = self._rows("X", X, self.dims[0])
        self._rows("Y", Y, self.dims[-1], rows=n)
        _require_tensor("order", order, torch.int32, int(steps) * self.batch,
                        exact=False, cuda=False)
        self._on_device(X=X, Y=Y, order=order)
        losses = np.zeros(steps, dtype=np.float32)
        _check(lib().nrr_surrogate_train(
            self._h, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
            n, C.c_void_p(order.data_ptr()), steps, lr, weight_decay,
            losses.ctypes.data_as(C.POINTER(C.c_float))))
        return losses

    def predict(self, X, out):
        n = self._rows("X", X, self.dims[0])
        self._rows("out", out, self.dims[-1], rows=n)
        self._on_device(X=X, out=out)
        _check(lib().nrr_surrogate_predict(self._h, C.c_void_p(X.data_ptr()),
                                           n, C.c_void_p(out.data_ptr())))

    def gradients(self, X, Y):
        self._rows("X", X, self.dims[0], rows=self.batch, exact=False)
        self._rows("Y", Y, self.dims[-1], rows=self.batch, exact=False)
        self._on_device(X=X, Y=Y)
        g = np.zeros(self.num_params, dtype=np.float32)
        loss = C.c_double()
        _check(lib().nrr_surrogate_gradients(
            self._h, C.c_void_p(X.data_ptr()), C.c_void_p(Y.data_ptr()),
            g.ctypes.data_as(C.POINTER(C.c_float)), C.byref(loss)))
        return loss.value, g

    def params(self) -> np.ndarray:
        p = np.zeros(self.num_params, dtype=np.float32)
        _check(lib().nrr_surrogate_get_params(
            self._h, p.ctypes.data_as(C.POINTER(C.c_float))))
        return p


def selftest_wait_expiry(which: int) -> bool:
    """Run one bounded wait on something that never happens (0: an mbarrier
    phase, 1: a grid barrier); True if it expired and recorded its error."""
    import torch
    out = C.c_int()
    _check(lib().nrr_selftest_wait_expiry(int(which),
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          C.byref(out)))
    return bool(out.value)


def autotune_save(path: str) -> None:
    """Write the autotuner's cache (launch shapes by grid key) to a JSON file."""
    _check(lib().nrr_autotune_save(str(path).encode()))


def autotune_load(path: str) -> None:
    """Add a saved autotuner cache; later grids with matching keys use it."""
    _check(lib().nrr_autotune_load(str(path).encode()))


def autotune_clear() -> None:
    _check(lib().nrr_autotune_clear())
