"""GPU tests of the solve's state handling and of the library's measurement
hooks, through the C ABI:

- the device footprint is checked before any allocation (NRR_ERR_OOM);
- checkpoint and resume (nrr_get_state -> a new grid -> nrr_set_state) give
  a trajectory and a converged solve bitwise identical to an uninterrupted
  one (Alg. 1's state is (u, v) and nothing else);
- the source term's reciprocal is within one ulp of correctly rounded
  division;
- independent grids relaxed concurrently on their own streams from several
  host threads (the paper's Sec. 5 multiple-patches experiment runs them on
  separate streams) equal their solo solves bit for bit and the oracle to
  1e-10;
- the peak probes return plausible rates.
"""
from __future__ import annotations

import threading

import numpy as np
import pytest
import torch

from paper_2501_14030_gb300 import nrr, workloads as W
from tests.helpers import default_dt_eta, oracle_grid, rel_err

pytestmark = pytest.mark.gpu


def test_footprint_checked_before_allocation(gpu):
    """A Cartesian 1280^3 grid (1288^3 padded points, just under 2^31) needs
    about 148 bytes per point, 316 GB, more than the device has: the call
    returns NRR_ERR_OOM after cudaMemGetInfo, having allocated nothing."""
    free0, _ = torch.cuda.mem_get_info()
    desc = W.grid_desc("cartesian", (1280, 1280, 1280), 4)
    with pytest.raises(nrr.NrrError) as e:
        nrr.Grid(desc)
    assert e.value.status == nrr.ERR_OOM, str(e.value)
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)
    # the library still works afterwards
    d2, p2 = W.small_equal_mass()
    g = nrr.Grid(d2)
    g.set_punctures(p2)
    assert g.relax(mode="fp64", tol=1e-10)["status"] == 0
    g.close()


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_checkpoint_resume_trajectory_is_bitwise(gpu, mode):
    """K1 steps, checkpoint (u, v) out, a fresh grid takes the checkpoint
    and runs K2 more: equal bit for bit to K1 + K2 uninterrupted steps."""
    desc, punc = W.grid_desc("sinhsymtp", (44, 26, 6), 8), W.spinning_q4_pair()
    a = nrr.Grid(desc)
    a.set_punctures(punc)
    dt, eta = a.timestep(0.5)
    a.step(37, dt, eta, mode=mode)
    u = torch.empty(a.shape, dtype=torch.float64, device="cuda")
    v = torch.empty_like(u)
    a.get_state(u, v)
    a.step(53, dt, eta, mode=mode)
    b = nrr.Grid(desc)
    b.set_punctures(punc)
    b.set_state(u.clone(), v.clone())
    b.step(53, dt, eta, mode=mode)
    ua, va, ub, vb = (torch.empty_like(u) for _ in range(4))
    a.get_state(ua, va)
    b.get_state(ub, vb)
    assert torch.equal(ua, ub) and torch.equal(va, vb)
    a.close()
    b.close()


def test_checkpoint_resume_relaxation_is_bitwise(gpu):
    """A solve stopped after 200 steps (a multiple of the norm interval),
    checkpointed and continued on a new grid converges after the same total
    number of steps, to the same u bit for bit."""
    desc, punc = W.small_equal_mass()
    ref = nrr.Grid(desc)
    ref.set_punctures(punc)
    r_ref = ref.relax(mode="fp64", tol=1e-10, check_every=50)
    u_ref = torch.empty(ref.shape, dtype=torch.float64, device="cuda")
    ref.get_state(u_ref)
    a = nrr.Grid(desc)
    a.set_punctures(punc)
    assert r_ref["iters"] > 200
    r1 = a.relax(mode="fp64", tol=1e-10, check_every=50, max_iters=200,
                 raise_on_error=False)
    assert r1["status"] == nrr.ERR_NOT_CONVERGED and r1["iters"] == 200
    u = torch.empty_like(u_ref)
    v = torch.empty_like(u_ref)
    a.get_state(u, v)
    b = nrr.Grid(desc)
    b.set_punctures(punc)
    b.set_state(u, v)
    r2 = b.relax(mode="fp64", tol=1e-10, check_every=50,
                 initial=nrr.INIT_CURRENT)
    assert r2["status"] == 0
    assert r1["iters"] + r2["iters"] == r_ref["iters"]
    ub = torch.empty_like(u_ref)
    b.get_state(ub)
    assert torch.equal(ub, u_ref)
    for g in (ref, a, b):
        g.close()


def _ulps(out: np.ndarray, ref: np.ndarray) -> float:
    return float(np.max(np.abs(out - ref) / np.spacing(np.abs(ref))))


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_source_reciprocal_within_one_ulp(gpu, dtype):
    """The stage kernels evaluate (1 + alpha u)^-1 by refining the hardware
    approximation (one third-order step in FP64, one Newton step in FP32).
    Against correctly rounded division (numpy on the host): at most one
    unit in the last place, over the range the source term meets
    (s = 1 + alpha u near 1) and well beyond it."""
    rng = np.random.default_rng(7)
    s = np.concatenate([rng.uniform(0.5, 2.0, 1 << 20),
                        np.exp(rng.uniform(np.log(1e-6), np.log(1e6), 1 << 20)),
                        1.0 + rng.uniform(-1e-6, 1e-6, 1 << 16),
                        [1.0, 2.0, 0.5, 0.75, 1.5]]).astype(dtype)
    ref = (dtype(1.0) / s).astype(dtype)
    sd = torch.from_numpy(s).cuda()
    out = torch.empty_like(sd)
    nrr.selftest_recip(sd, out)
    got = out.cpu().numpy()
    assert _ulps(got, ref) <= 1.0, _ulps(got, ref)
    exact = np.mean(got == ref)
    assert exact > 0.5, exact


STREAM_CASES = [
    (W.grid_desc("sinhsymtp", (44, 26, 6), 8), W.spinning_q4_pair()),
    W.small_equal_mass(),
    (W.grid_desc("spherical", (40, 22, 8), 8, rmax=64.0), W.spinning_q4_pair()),
]


def test_concurrent_grids_on_streams_match_solo_and_oracle(gpu):
    """Three independent solves run at the same time, each grid on its own
    work stream driven by its own host thread: each equals its solo solve
    bit for bit (same step count) and the oracle's converged u to 1e-10."""
    grids, solo = [], []
    for desc, punc in STREAM_CASES:
        g = nrr.Grid(desc)
        g.set_punctures(punc)
        r = g.relax(mode="fp64", tol=1e-10, check_every=50)
        u = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        g.get_state(u)
        grids.append(g)
        solo.append((r, u))
    torch.cuda.synchronize()
    for repeat in range(2):
        res = [None] * len(grids)

        def work(i):
            res[i] = grids[i].relax(mode="fp64", tol=1e-10, check_every=50)

        threads = [threading.Thread(target=work, args=(i,))
                   for i in range(len(grids))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        for i, g in enumerate(grids):
            assert res[i] is not None and res[i]["status"] == 0
            assert res[i]["iters"] == solo[i][0]["iters"]
            u = torch.empty_like(solo[i][1])
            g.get_state(u)
            assert torch.equal(u, solo[i][1]), (repeat, i)
    for (desc, punc), (r, u) in zip(STREAM_CASES, solo):
        og = oracle_grid(desc)
        alpha, beta = og.source(punc)
        dt, eta = default_dt_eta(og)
        uo, vo = og.zeros(), og.zeros()
        it, _, st = og.relax(alpha, beta, uo, vo, eta=eta, dt=dt, tol=1e-10,
                             check_every=50)
        assert st == 0 and it == r["iters"]
        assert rel_err(u.cpu().numpy(), uo) <= 1e-10
    for g in grids:
        g.close()


def test_peak_probes(gpu):
    """The roofline denominators the bench measures: FP64 FMA throughput of
    order 1 TFLOP/s on GB300 (152 SMs x 2 FMA/clk x 2 flop x ~2 GHz =
    1.26 nominal), FP32 far above it, L2 reads above the HBM copy rate."""
    p = nrr.probe_peaks()
    assert 0.5 < p["fp64_tflops"] < 1.6, p
    assert p["fp32_tflops"] > 20 * p["fp64_tflops"], p
    assert 5e3 < p["l2_gbs"] < 1e5, p


LOOP_CASES = [("fp64", 0, 1), ("fp64", 4, 1), ("fp32", 3, 4), ("fp32", 0, 2),
              ("fp32_dc", 0, 2), ("fp32_dc", 4, 1), ("fp32_dc", 3, 4)]


@pytest.mark.parametrize("mode,variant,zc", LOOP_CASES)
def test_device_loop_equals_host_loop(gpu, mode, variant, zc):
    """The stop test on the device (one graph launch per solve, a WHILE node
    over chunks) and on the host (a norm read after every chunk) take the
    same steps and leave identical states, for every mode and for the
    per-stage, tensor-copy and multi-stage (cooperative) stage kernels."""
    desc, punc = W.grid_desc("sinhsymtp", (64, 32, 8), 8), W.spinning_q4_pair()
    launch_mode = "fp64" if mode == "fp64" else "fp32"
    out = []
    for on in (True, False):
        g = nrr.Grid(desc)
        g.set_punctures(punc)
        g.set_launch(zc, launch_mode, variant, 0)
        g.set_device_loop(on)
        # plain FP32 stalls near 1e-7 on this grid: a tolerance it reaches
        r = g.relax(mode=mode, tol=1e-5 if mode == "fp32" else 1e-10,
                    check_every=50)
        u = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        v = torch.empty_like(u)
        g.get_state(u, v)
        out.append((r, u, v))
        g.close()
    (r1, u1, v1), (r0, u0, v0) = out
    assert r1["status"] == r0["status"] == 0
    assert (r1["iters"], r1["outer_iters"]) == (r0["iters"], r0["outer_iters"])
    assert r1["norm"] == r0["norm"]
    assert torch.equal(u1, u0) and torch.equal(v1, v0)


@pytest.mark.parametrize("mode", ["fp64", "fp32_dc"])
def test_device_loop_step_limit_not_a_chunk_multiple(gpu, mode):
    """max_iters = 1234 with 50-step chunks: 24 chunks on the device, the
    last 34 steps by the host; both loops stop at 1234 steps (not converged)
    with identical states."""
    desc, punc = W.grid_desc("sinhsymtp", (64, 32, 8), 8), W.spinning_q4_pair()
    out = []
    for on in (True, False):
        g = nrr.Grid(desc)
        g.set_punctures(punc)
        g.set_device_loop(on)
        r = g.relax(mode=mode, tol=1e-14, check_every=50, max_iters=1234,
                    raise_on_error=False)
        u = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        g.get_state(u)
        out.append((r, u))
        g.close()
    (r1, u1), (r0, u0) = out
    assert r1["status"] == r0["status"] == nrr.ERR_NOT_CONVERGED
    assert r1["iters"] == r0["iters"] == 1234
    assert torch.equal(u1, u0)
