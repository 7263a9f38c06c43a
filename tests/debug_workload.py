"""A small workload that touches every stencil, boundary and residual kernel
of the library: each coordinate family and FD order, each stage-kernel
variant that applies, plain FP64, plain FP32 and defect-correction
relaxation, the residual, batches with each stage variant, and a two-patch
system.  It returns a digest of every final state.

`tests/test_gpu_debug_build.py` runs it twice: in a subprocess against the
NRR_DEBUG build (`python -m tests.debug_workload`, with NRR_DEBUG=1), where
no access may be refused, and in the test process against the release
build.  The address checks change no arithmetic, so the digests must be
equal.
"""
from __future__ import annotations

import hashlib
import json

import numpy as np

PUNC = None


def _digest(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:24]


def _state(nrr, torch, g):
    u = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    v = torch.empty_like(u)
    g.get_state(u, v)
    return u.cpu().numpy(), v.cpu().numpy()


# (family, interior size, FD order, map parameters, stage variants per mode;
# a variant given as (variant, zc) runs with that plane chunk)
GRIDS = [
    ("sinhsymtp", (32, 16, 4), 8, {}, {"fp64": [0, 1, 2, 3, 4, 5], "fp32": [0, 1, 2, 3, 4, 5, 6]}),
    ("sinhsymtp", (24, 10, 6), 4, {}, {"fp64": [0, 1, 2, 4], "fp32": [0, 1, 2, 4]}),
    ("spherical", (16, 8, 4), 10, {"rmax": 40.0}, {"fp64": [0, 1, 2], "fp32": [0, 1]}),
    ("sinhspherical", (16, 8, 4), 8, {}, {"fp64": [0, 2], "fp32": [0]}),
    ("sinhcylindrical", (16, 12, 4), 8, {}, {"fp64": [0], "fp32": [0]}),
    # Cartesian variant 1 is the tensor-copy kernel; 16 planes per chunk run
    # its ring through more slots than it holds
    ("cartesian", (32, 32, 32), 8, {"xmax": 20.0}, {"fp64": [0, (1, 16)], "fp32": [0, (1, 16)]}),
]


def run() -> dict:
    import torch
    from paper_2501_14030_gb300 import nrr, workloads as W
    torch.cuda.set_device(0)
    punc = W.spinning_q4_pair()
    out = {}
    for coord, n, order, kw, variants in GRIDS:
        desc = W.grid_desc(coord, n, order, **kw)
        name = "%s_%dx%dx%d_o%d" % (coord, *n, order)
        g = nrr.Grid(desc)
        g.set_punctures(punc)
        dt, eta = g.timestep(0.5)
        for mode, vs in variants.items():
            for var in vs:
                if isinstance(var, tuple):
                    var, zc = var
                else:
                    zc = 2 if var in (1, 3, 5) else 1
                try:
                    g.set_launch(zc, mode, var)
                except nrr.NrrError:
                    continue  # not eligible for this grid: nothing launched
                g.set_punctures(punc)
                g.step(6, dt, eta, mode)
                u, v = _state(nrr, torch, g)
                out["%s_%s_v%d" % (name, mode, var)] = _digest(u, v)
        g.set_launch(1, "fp64", 0)
        g.set_launch(1, "fp32", 0)
        for mode in ("fp64", "fp32", "fp32_dc"):
            r = g.relax(mode=mode, tol=1e-6, max_iters=200, raise_on_error=False)
            u, v = _state(nrr, torch, g)
            out["%s_relax_%s" % (name, mode)] = _digest(u, v, np.array([r["iters"]]))
        h = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        nrm = g.residual(100.0, h)
        out["%s_residual" % name] = _digest(h.cpu().numpy(), np.array([nrm]))
        g.close()
    # batches: each stage variant, FP64 and defect correction
    descs = [W.grid_desc("sinhsymtp", s, 8) for s in ((32, 16, 4), (64, 8, 4), (32, 32, 8))]
    for mode in ("fp64", "fp32_dc"):
        for var, zc in ((0, 4), (1, 2), (1, 8), (2, 1), (2, 2)):
            b = nrr.Batch(descs, [punc] * 3, with_fp64=(mode == "fp64"))
            try:
                b.set_launch(var, zc, mode)
            except nrr.NrrError:
                b.close()
                continue
            b.relax(mode=mode, tol=1e-30, max_iters=100, check_every=50,
                    raise_on_error=False)
            us = []
            for i in range(3):
                ub = np.zeros(b.shapes[i])
                b.get_u(i, ub)
                us.append(ub)
            out["batch_%s_v%d_zc%d" % (mode, var, zc)] = _digest(*us)
            b.close()
    # two patches: a Spherical grid and a Cartesian box
    go = nrr.Grid(W.grid_desc("spherical", (32, 16, 16), 4, rmax=48.0))
    gi = nrr.Grid(W.grid_desc("cartesian", (24, 24, 24), 4, xmax=8.0))
    go.set_punctures(punc)
    gi.set_punctures(punc)
    ps = nrr.PatchSet(go, gi, 3.0, 4)
    dt, eta = ps.timestep(0.5)
    ps.step(20, dt, eta)
    out["patches"] = _digest(*_state(nrr, torch, go), *_state(nrr, torch, gi),
                             np.array([ps.residual(100.0)]))
    ps.close()
    go.close()
    gi.close()
    torch.cuda.synchronize()
    return {"digests": out, "check": nrr.debug_check()}


if __name__ == "__main__":
    print(json.dumps(run()), flush=True)
