#!/usr/bin/env python
"""Benchmark of the puncture-data relaxation solve on GB300.

One step = one complete FP64 solve of the mass-ratio-4 spinning Bowen-York
pair on SinhSymTP 128x128x16 (8th-order FD, RK4): the source set-up, the
relaxation to residual L2 norm < 1e-10 and the final residual, all on the
device through the C ABI.  `value` is gridpoint-RHS/s = interior points x 4
RHS evaluations per RK4 step x steps / device seconds.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 (launched by torchrun) every rank solves its own copy (the solves
are independent; no collective on the data path) and rank 0 prints the
whole-job rate over the slowest rank's time.  `--impl reference` times the
CPU oracle on the host cores instead, on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gridpoint-RHS/s, FP64 relaxation of a BBH puncture solve to residual 1e-10"
UNIT = "gridpoint-RHS/s"
WORKLOAD = ("q=4 spinning Bowen-York pair (m 0.8/0.2, z=+-5, P=+-0.09x, "
            "chi=(0.3,-0.2,0.5)/(0,0.4,-0.1)); SinhSymTP 128x128x16, AMAX 1e4, "
            "bScale 5, SINHWAA 0.07; 8th-order FD; RK4 CFL 0.5; "
            "FP64 relaxation to residual L2 < 1e-10 (r < 100, checked every 50 steps)")
CHECK_EVERY = 50
# nrr_set_launch's curvilinear stage-kernel variants
STAGE_VARIANTS = {0: "column", 1: "tiled", 2: "persistent", 3: "tensor-copy tiled",
                  4: "multi-stage column", 5: "multi-stage tensor-copy tiled",
                  6: "two stages per launch"}
# FP64 FMA units: 2 FMA per clock per SM on GB300 (the SM count is read from
# the device)
FP64_FMA_PER_CLK = 2
MAX_SM_MHZ = 2070.0


# DRAM bytes (read + write) per launch of the FP64 stage kernel at
# 128x128x16, order 8, from one ncu capture of this kernel (dram__bytes_read
# + dram__bytes_write, mean of a FIRST and a MID launch).
STAGE_FP64_DRAM_BYTES = 17.0e6


def flops_per_point(ng: int) -> int:
    """Algorithmic flops per interior point per fused RHS + RK4 stage, the
    count the roofline uses: 3 (2p + 6) for the Laplacian's three directions
    at FD order p = 2 ng, plus about 11 for the source and the RK4 terms
    (FMA = 2 flops; 77 at order 8)."""
    return 3 * (4 * ng + 6) + 11


def folded_flops_per_point(ng: int) -> int:
    """The same work as the folded operator evaluates it (c^2 and the metric
    folded into per-column weights): centre weight (1 mul), 2*ng FMAs in
    each of xx0 and xx1 (8 ng), ng adds + ng FMAs in phi (3 ng), the source
    term (fma, divide, 4 mul, fma: 9), k_u (fma: 2) and the RK4 update
    (7 on average over the four stages): 63 at order 8."""
    return 11 * ng + 1 + 9 + 2 + 7


# Algorithmic bytes per evolved point of one fused FP32 stage: read u, v
# (stage), y_n (u, v), acc (u, v), alpha, beta; write stage (u, v) and
# acc (u, v) -- 12 words.
FP32_STAGE_BYTES = 48
FP64_STAGE_BYTES = 96


def hbm_peak_gbs() -> tuple[float, str]:
    """The measured copy bandwidth of the GB300s, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def rank_info():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, local_rank: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        self.index = vis.split(",")[local_rank] if vis else str(local_rank)
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        self.proc.wait()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def oracle_rate(desc, punc, seconds: float):
    """Gridpoint-RHS/s of the CPU oracle on a bounded sample: RK4 steps of the
    same grid from zero data, sized to about `seconds` of host time."""
    import numpy as np  # noqa: F401
    import oracle as O
    og = O.grid_from_desc(desc)
    alpha, beta = og.source(punc)
    dt, eta = O.default_dt_eta(og)
    u, v = og.zeros(), og.zeros()
    t = time.perf_counter()
    og.rk4_step(alpha, beta, eta, dt, u, v)
    one = time.perf_counter() - t
    steps = max(2, int(seconds / max(one, 1e-6)))
    t = time.perf_counter()
    for _ in range(steps):
        og.rk4_step(alpha, beta, eta, dt, u, v)
    H = og.residual(alpha, beta, u)
    og.norm(H)
    el = time.perf_counter() - t
    n_int = desc["n"][0] * desc["n"][1] * desc["n"][2]
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return n_int * 4 * steps / el, el, steps, cores


def run_reference(args):
    rank, world, _ = rank_info()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    from paper_2501_14030_gb300 import workloads as W
    desc, punc = W.q4_sinhsymtp_128()
    for _ in range(args.warmup):
        oracle_rate(desc, punc, 2.0)
    rates, times = [], []
    for _ in range(args.steps):
        r, el, steps, cores = oracle_rate(desc, punc, 4.0)
        rates.append(r)
        times.append(el)
    value = sum(rates) / len(rates)
    sample = ("%d RK4 steps + one residual of the 128x128x16 FP64 workload "
              "per timed step" % steps)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    if rank == 0 or world == 1:
        __graft_entry__.build()
    if dist is not None:
        dist.barrier()
    from paper_2501_14030_gb300 import nrr, workloads as W

    desc, punc = W.q4_sinhsymtp_128()
    # --launch-shapes: reuse the launch shapes an earlier run chose (a
    # profiler's replays distort the autotuner's trials) or save this run's
    shapes = args.launch_shapes
    reuse = bool(shapes) and os.path.exists(shapes)
    if reuse:
        nrr.autotune_load(shapes)
    g = nrr.Grid(desc)
    if args.host_loop:
        g.set_device_loop(False)
    n_int = g.interior_points
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def solve():
        g.set_punctures(punc)
        r = g.relax(mode="fp64", tol=1e-10, check_every=CHECK_EVERY)
        nrm = g.residual(100.0)
        return r, nrm

    g.set_punctures(punc)
    if not reuse:
        for m in ("fp64", "fp32"):
            g.autotune(m, 20)  # launch shapes
        if shapes:
            nrr.autotune_save(shapes)
    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    launches0 = nrr.kernel_launches()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms, iters, results = 0.0, 0, []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 (129 MB) between steps; not timed
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r, nrm = solve()
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        iters += r["iters"]
        results.append((r, nrm))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist is not None:
        dist.barrier()
    launches = nrr.kernel_launches() - launches0
    clk = clocks.stop()

    # whole job: the slowest rank's time, the RHS evaluations of all ranks
    from paper_2501_14030_gb300.replicas import job_rate
    t_max_s, _, value = job_rate(total_ms / 1e3, float(n_int * 4 * iters), dist,
                                 device="cuda")

    # ---- dominant kernel: the fused RK4 stage.  Its time per launch inside
    # the timed solves: the solve's device time over its 4 stage launches per
    # RK4 step (the residual checks, one per 50 steps, are left in: an upper
    # bound on the stage's time).  Also timed alone on its work stream.
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    peaks = nrr.probe_peaks()
    dt, eta = g.timestep(0.5)
    g.set_punctures(punc)
    g.relax(mode="fp64", tol=1e-10, check_every=CHECK_EVERY)
    ms_isolated = g.profile_stages(200, dt, eta, mode="fp64")
    ms_launch = t_max_s * 1e3 / args.steps / (4 * results[-1][0]["iters"])
    ng = g.ng
    flops = flops_per_point(ng) * n_int
    achieved = flops / (ms_launch * 1e-3) / 1e12
    peak = sms * FP64_FMA_PER_CLK * 2 * MAX_SM_MHZ * 1e6 / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": STAGE_FP64_DRAM_BYTES,
                "traffic_note": "dram read+write bytes per launch from one ncu "
                                "capture (cold L2 per replay; FIRST and MID "
                                "launches averaged); the 35 MB working set is "
                                "L2-resident in the timed run",
                "kernel": "stage_curvi_kernel<double,4,*> (fused RHS + BC + RK4 stage)",
                "ms_per_launch": ms_launch,
                "ms_per_launch_basis": "in-solve: timed solve / (4 x RK4 steps)",
                "ms_per_launch_isolated": ms_isolated,
                "flops_per_launch": flops,
                "flops_per_point": flops_per_point(ng),
                "flops_basis": "3 (2p + 6) + 11 per interior point at FD order p",
                "folded_flops_per_point": folded_flops_per_point(ng),
                "frac_folded_count": folded_flops_per_point(ng) * n_int /
                (ms_launch * 1e-3) / 1e12 / peak,
                "peak_basis": "FP64: %d SMs (device property) x 2 FMA/clk x 2 flop "
                              "x %.0f MHz (unit counts and max clock)" % (sms, MAX_SM_MHZ),
                "peak_probe_measured": peaks["fp64_tflops"],
                "frac_of_probe": achieved / peaks["fp64_tflops"]}
    if clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (
            sms * FP64_FMA_PER_CLK * 2 * clk["sm_mhz"] * 1e6 / 1e12)

    # ---- FP32 relaxation inside the FP64 defect-correction loop, same
    # workload (context beside the FP64 headline)
    u64 = np.zeros(g.shape)
    g.set_punctures(punc)
    r64 = g.relax(mode="fp64", tol=1e-10, check_every=CHECK_EVERY)
    g.get_state(u64)
    dc_ms, rdc = [], None
    for _ in range(3):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.set_punctures(punc)
        rdc = g.relax(mode="fp32_dc", tol=1e-10, check_every=CHECK_EVERY)
        g.residual(100.0)
        e1.record(stream)
        e1.synchronize()
        dc_ms.append(e0.elapsed_time(e1))
    udc = np.zeros(g.shape)
    g.get_state(udc)
    dc_err = float(np.abs(udc - u64).max() / np.abs(u64).max())
    ms32 = g.profile_stages(200, dt, eta, mode="fp32")
    bytes32 = FP32_STAGE_BYTES * n_int

    # ---- end to end through the public API with host buffers
    pinned_u = torch.empty(g.shape, dtype=torch.float64, pin_memory=True).numpy()
    e2e_ms = 0.0
    e2e_iters = 0
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.set_punctures(punc)  # host puncture array -> device
        r = g.relax(mode="fp64", tol=1e-10, check_every=CHECK_EVERY)
        g.get_state(pinned_u)  # converged u -> pinned host memory
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        e2e_iters += r["iters"]
    e2e_value = job_rate(e2e_ms / 1e3, float(n_int * 4 * e2e_iters), dist,
                         device="cuda")[2]
    h2d = 2 * (10 * 8)  # two nrr_puncture structs
    d2h = int(np.prod(g.shape)) * 8

    # ---- plain FP32 relaxation (context: its stall level), untimed
    r32 = g.relax(mode="fp32", tol=1e-10, check_every=CHECK_EVERY,
                  max_iters=iters // max(1, args.steps), raise_on_error=False)

    batch = None if args.no_batch else run_batch(args, nrr, W, torch)
    # the larger grids and the other coordinate families, FP64 against
    # defect correction
    big = None if args.no_configs2 else configs2_section(nrr, W, torch, peaks, sms)
    patches = patches_section(nrr, W, torch)
    # warm start from the learned surrogate: 8192 training solves at
    # 64x32x8, 1024 held-out solves at 128x128x16 cold vs warm
    # (--compact-surrogate: 2048 / 128)
    n_tr, n_held = (2048, 128) if args.compact_surrogate else (8192, 1024)
    warm = None if args.no_surrogate else surrogate_pipeline(nrr, W, torch, n_tr,
                                                            n_held, 100)

    line = None
    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            rate, el, steps, cores = oracle_rate(desc, punc, args.cpu_seconds)
            cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": "%d RK4 steps (+ one residual) of the same FP64 "
                             "workload from zero data, %.1f s" % (steps, el)}
        r0, n0 = results[-1]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_max_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "grid": "SinhSymTP 128x128x16",
                       "fd_order": 8, "global_batch": world,
                       "stage_launch": {m: dict(zip(("variant", "zc", "block"),
                                                    (STAGE_VARIANTS.get(v, str(v)), z, bl)))
                                        for m, (v, z, bl) in
                                        ((m, g.get_launch(m)) for m in ("fp64", "fp32"))},
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "flushed before each step (256 MiB write, untimed)"},
            "sec_to_residual": {"fp64": t_max_s / args.steps,
                                "rk4_steps": r0["iters"],
                                "final_norm": r0["norm"],
                                "residual_after": n0},
            "fp32_plain": {"rk4_steps": r32["iters"], "final_norm": r32["norm"],
                           "seconds": r32["seconds"], "status": r32["status"]},
            "fp32_defect_correction": {
                "sec_to_residual": statistics.median(dc_ms) / 1e3,
                "rk4_steps": rdc["iters"], "outer_iters": rdc["outer_iters"],
                "final_norm": rdc["norm"],
                "speedup_vs_fp64": (t_max_s / args.steps) / (statistics.median(dc_ms) / 1e3),
                "max_rel_diff_u_vs_fp64_solution": dc_err,
                "fp32_stage_us_per_launch": ms32 * 1e3,
                "fp32_stage_GBps_algorithmic": bytes32 / (ms32 * 1e-3) / 1e9,
                "fp32_stage_roofline": {
                    "bound": "l2", "achieved": bytes32 / (ms32 * 1e-3) / 1e9,
                    "peak": peaks["l2_gbs"], "unit": "GB/s",
                    "frac": bytes32 / (ms32 * 1e-3) / 1e9 / peaks["l2_gbs"],
                    "bytes_per_point": FP32_STAGE_BYTES,
                    "peak_basis": "L2 read bandwidth measured by the library's "
                                  "probe kernel (the FP32 working set of "
                                  "128x128x16 stays in L2)"}},
            "measured_peaks": dict(peaks, sms=sms),
            "batch_512": batch,
            "larger_grids": big,
            "two_patches": patches,
            "surrogate_warm_start": warm,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "wall_s_timed": wall,
        }
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_profile_steps(args):
    """A short fixed workload for profiler captures: set-up of the q=4 grid
    named by --profile-grid, then `--profile-steps` RK4 steps (4 fused stage
    launches each) and one residual, in the precision given by --mode.
    Prints nothing timed."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_14030_gb300 import nrr, workloads as W
    torch.cuda.set_device(0)
    grids = {"sinhsymtp128": W.q4_sinhsymtp_128, "sinhsymtp256": W.q4_sinhsymtp_256,
             "cartesian256": W.q4_cartesian_256}
    desc, punc = grids[args.profile_grid]()
    g = nrr.Grid(desc)
    g.set_punctures(punc)
    dt, eta = g.timestep(0.5)
    if args.profile_zc > 0:
        g.set_launch(args.profile_zc, args.mode, args.profile_variant,
                     args.profile_block)
    g.step(args.profile_steps, dt, eta, mode=args.mode)
    print(json.dumps({"profile_steps": args.profile_steps, "mode": args.mode,
                      "residual": g.residual(100.0)}))
    g.close()
    return 0


def run_batch(args, nrr, W, torch):
    """The 512-solve parameter sweep (uneven SinhSymTP grids, order 8) as one
    graph launch in defect-correction mode; returns a summary dict."""
    import numpy as np
    params = W.batch_parameters(512, 20250124)
    descs = [p["desc"] for p in params]
    b = nrr.Batch(descs, [p["punctures"] for p in params])
    zc, ms, var = b.autotune("fp32_dc", 3)
    b.relax(mode="fp32_dc", tol=1e-10, max_iters=100, raise_on_error=False)
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    per, tot = b.relax(mode="fp32_dc", tol=1e-10, raise_on_error=False)
    e1.record(stream)
    e1.synchronize()
    secs = e0.elapsed_time(e1) / 1e3
    its = np.array([r["iters"] for r in per])
    rhs = sum(4 * r["iters"] * int(np.prod(d["n"])) for r, d in zip(per, descs))
    b.close()
    return {"solves": len(descs), "converged": int(sum(r["status"] == 0 for r in per)),
            "seconds": secs, "solves_per_s": len(descs) / secs,
            "gridpoint_rhs_per_s": rhs / secs,
            "rk4_steps_min_median_max": [int(its.min()), int(np.median(its)), int(its.max())],
            "stage_variant": {0: "register-staged tiles", 1: "tensor-copy ring",
                              2: "columns"}.get(var, str(var)),
            "stage_zc": zc, "fp32_stage_ms_all_solves": ms,
            "graph_launches": 1, "chunks": tot["outer_iters"],
            "grids": "SinhSymTP N0 in {64,96,128}, N1 in {32,64,96,128}, N2 in {8,16}, order 8"}


def surrogate_pipeline(nrr, W, torch, n_train: int, n_held: int, epochs: int):
    """Solver-generated coarse solutions (64x32x8), device training of the
    12 -> 512x4 -> 16384 network, then `n_held` held-out solves at 128x128x16
    started cold and from the network's prediction; returns a summary dict."""
    import numpy as np
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    coarse_n, fine_n = (64, 32, 8), (128, 128, 16)
    train = W.batch_parameters(n_train, seed=1)
    cdesc = [W.grid_desc("sinhsymtp", coarse_n, 8, bscale=p["d"] / 2) for p in train]
    b = nrr.Batch(cdesc, [p["punctures"] for p in train])
    (per, tot), t_gen = timed(lambda: b.relax(mode="fp32_dc", tol=1e-10,
                                              raise_on_error=False))
    n_out = int(np.prod(coarse_n))
    Y = torch.empty((n_train, n_out), dtype=torch.float32, device="cuda")
    b.get_interior(Y)
    b.close()
    X = torch.from_numpy(W.surrogate_inputs(train)).cuda()
    dims = W.mlp_dims(n_out=n_out)
    net = nrr.Surrogate(dims, W.mlp_init_params(dims, seed=3), batch=256)
    net.fit_scaling(Y)
    steps = epochs * (n_train // 256)
    order = torch.from_numpy(W.minibatch_order(n_train, 256, steps, seed=4)).cuda()
    losses, t_train = timed(lambda: net.train(X, Y, order, steps, lr=1e-3))
    flops_step = 6 * 256 * sum(a * b_ for a, b_ in zip(dims[:-1], dims[1:]))

    held = W.batch_parameters(n_held, seed=2)
    fdesc = [W.grid_desc("sinhsymtp", fine_n, 8, bscale=p["d"] / 2) for p in held]
    cold = nrr.Batch(fdesc, [p["punctures"] for p in held])
    cold.autotune("fp32_dc", 3)
    cold.relax(mode="fp32_dc", tol=1e-10, max_iters=50, raise_on_error=False)
    (per_c, tot_c), t_cold = timed(lambda: cold.relax(mode="fp32_dc", tol=1e-10,
                                                      raise_on_error=False))
    cold.close()
    warm = nrr.Batch(fdesc, [p["punctures"] for p in held])
    warm.autotune("fp32_dc", 3)
    warm.relax(mode="fp32_dc", tol=1e-10, max_iters=50, raise_on_error=False)
    Xh = torch.from_numpy(W.surrogate_inputs(held)).cuda()
    shape = W.padded_shape(fdesc[0])

    def predict_and_start():
        pred = torch.empty((n_held, n_out), dtype=torch.float32, device="cuda")
        net.predict(Xh, pred)
        uf = torch.zeros(shape, dtype=torch.float64, device="cuda")
        for i, p in enumerate(held):
            cd = W.grid_desc("sinhsymtp", coarse_n, 8, bscale=p["d"] / 2)
            nrr.prolong(cd, pred[i].contiguous(), fdesc[i], uf)
            warm.set_u(i, uf)
    _, t_pred = timed(predict_and_start)
    (per_w, tot_w), t_warm = timed(lambda: warm.relax(
        mode="fp32_dc", tol=1e-10, initial=nrr.INIT_DEVICE, raise_on_error=False))
    warm.close()
    it_c = np.array([r["iters"] for r in per_c])
    it_w = np.array([r["iters"] for r in per_w])
    return {
        "train_solves": n_train, "train_grid": "SinhSymTP 64x32x8, order 8",
        "train_data_seconds": t_gen,
        "train_converged": int(sum(r["status"] == 0 for r in per)),
        "network": dims, "batch": 256, "steps": steps,
        "train_seconds": t_train, "train_tflops": flops_step * steps / t_train / 1e12,
        "loss_first_last": [float(losses[:10].mean()), float(losses[-10:].mean())],
        "held_out_solves": n_held, "held_out_grid": "SinhSymTP 128x128x16, order 8",
        "cold": {"seconds": t_cold, "status": tot_c["status"],
                 "mean_rk4_steps": float(it_c.mean()), "max_rk4_steps": int(it_c.max())},
        "warm": {"seconds": t_warm, "predict_prolong_seconds": t_pred,
                 "status": tot_w["status"], "mean_rk4_steps": float(it_w.mean()),
                 "max_rk4_steps": int(it_w.max())},
        "step_reduction": float(1.0 - it_w.mean() / it_c.mean()),
        "time_reduction": float(1.0 - (t_warm + t_pred) / t_cold)}


def run_surrogate(args):
    """The full surrogate pipeline: 8192 training solves (default), 1024
    held-out solves."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_14030_gb300 import nrr, workloads as W
    torch.cuda.set_device(0)
    out = surrogate_pipeline(nrr, W, torch, args.surrogate_train,
                             args.surrogate_held, args.surrogate_epochs)
    print(json.dumps({"surrogate": out}), flush=True)
    return 0


def run_profile_gemm(args):
    """The surrogate's GEMM shapes (forward of the 512 -> 16384 layer at batch
    256, its input gradient with K = 16384, its weight gradient, a hidden
    layer) and a large M for the tensor-core rate: each tile width and K
    split that applies, timed with CUDA events (operands stay L2-resident
    between calls) two ways: 20 calls enqueued from Python with one status
    read-back (`ms_enqueued`, host-bound for the small shapes), and the same
    20 calls captured in a CUDA graph and replayed (`ms`, device time per
    call).  The chosen plan (bn = splits = 0) is listed first."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_14030_gb300 import nrr
    torch.cuda.set_device(0)
    g = torch.Generator(device="cuda").manual_seed(0)
    hbm, _ = hbm_peak_gbs()
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16 = float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        bf16 = 1900.0  # fallback burst figure
    shapes = [(256, 16384, 512), (256, 512, 16384), (16384, 512, 256),
              (256, 512, 512), (8192, 16384, 512)]
    if args.gemm_shape:
        # one shape, the chosen plan, three plain calls (profiler captures)
        M, N, K = (int(x) for x in args.gemm_shape.split(","))
        A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
        D = torch.empty((M, N), dtype=torch.float32, device="cuda")
        for _ in range(3):
            nrr.gemm_bf16_tn_async(A, B, D)
        nrr.gemm_status()
        print(json.dumps({"gemm": [M, N, K], "calls": 3}))
        return 0
    for (M, N, K) in shapes:
        A = torch.randn((M, K), device="cuda", generator=g).to(torch.bfloat16)
        B = torch.randn((N, K), device="cuda", generator=g).to(torch.bfloat16)
        D = torch.empty((M, N), dtype=torch.float32, device="cuda")
        combos = [(0, 0, -1)] + [(bn, 1, 0) for bn in (64, 128, 256) if N % bn == 0]
        combos += [(bn, 1, 1) for bn in (128, 256) if N % bn == 0]
        if M % 256 == 0:
            combos += [(bn, 1, 2) for bn in (128, 256) if N % bn == 0]
        if K >= 4096:
            combos += [(128, sp, 0) for sp in (8, 19, 38)] + [(64, 19, 0)]
        for bn, sp, pers in combos:
            for _ in range(3):
                nrr.gemm_bf16_tn_async(A, B, D, bn=bn, splits=sp, persistent=pers)
            nrr.gemm_status()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(20):
                nrr.gemm_bf16_tn_async(A, B, D, bn=bn, splits=sp, persistent=pers)
            e1.record()
            e1.synchronize()
            nrr.gemm_status()
            ms_enq = e0.elapsed_time(e1) / 20
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, capture_error_mode="thread_local"):
                for _ in range(20):
                    nrr.gemm_bf16_tn_async(A, B, D, bn=bn, splits=sp,
                                           persistent=pers)
            graph.replay()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(5):
                graph.replay()
            e1.record()
            e1.synchronize()
            nrr.gemm_status()
            ms = e0.elapsed_time(e1) / 100
            del graph
            nbytes = 2 * (M * K + N * K) + 4 * M * N
            tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
            gbs = nbytes / (ms * 1e-3) / 1e9
            print(json.dumps({"gemm": [M, N, K], "bn": bn, "splits": sp,
                              "persistent": pers, "ms": ms,
                              "ms_enqueued": ms_enq,
                              "tflops": tf, "frac_bf16": tf / bf16,
                              "GBps_operands_and_output": gbs,
                              "frac_hbm": gbs / hbm}), flush=True)
    return 0


def run_profile_batch(args):
    """A short fixed workload for profiler captures of the batched kernels:
    `--profile-batch` solves of 128x128x16 (held-out parameter draws) and
    100 defect-correction steps."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_14030_gb300 import nrr, workloads as W
    torch.cuda.set_device(0)
    held = W.batch_parameters(args.profile_batch, seed=2)
    descs = [W.grid_desc("sinhsymtp", (128, 128, 16), 8, bscale=p["d"] / 2)
             for p in held]
    b = nrr.Batch(descs, [p["punctures"] for p in held])
    # the autotuner launches the stage kernels outside graphs (kernels inside
    # conditional graph nodes cannot be captured one by one): 3 trial steps
    # x 4 stages x 2 repetitions for each of zc = 1, 2, 4
    zc, ms, var = b.autotune("fp32_dc", 3)
    per, tot = b.relax(mode="fp32_dc", tol=1e-10, max_iters=100,
                       raise_on_error=False)
    print(json.dumps({"profile_batch": args.profile_batch, "zc": zc,
                      "variant": var,
                      "fp32_stage_ms": ms,
                      "steps": tot["iters"], "seconds": tot["seconds"]}))
    b.close()
    return 0


def run_profile_patches(args):
    """A short fixed workload for profiler captures of the two-patch kernels:
    the Spherical 64x32x32 + Cartesian 48^3 system of the bench line,
    `--profile-patches` RK4 steps launched kernel by kernel (FP64)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_14030_gb300 import nrr, workloads as W
    torch.cuda.set_device(0)
    punc = W.spinning_q4_pair()
    go = nrr.Grid(W.grid_desc("spherical", (64, 32, 32), 4, rmax=48.0))
    gi = nrr.Grid(W.grid_desc("cartesian", (48, 48, 48), 4, xmax=8.0))
    go.set_punctures(punc)
    gi.set_punctures(punc)
    ps = nrr.PatchSet(go, gi, 3.0, 4)
    dt, eta = ps.timestep(0.5)
    ps.step(args.profile_patches, dt, eta)
    torch.cuda.synchronize()
    print(json.dumps({"profile_patches": args.profile_patches,
                      "receivers": [ps.outer_receivers, ps.inner_receivers]}))
    for x in (ps, go, gi):
        x.close()
    return 0


def configs2_section(nrr, W, torch, peaks, sms, tight_tol: float = 1e-12):
    """The q=4 spinning pair on SinhSymTP 256x256x32, Spherical 128x64x32 and
    Cartesian 256^3 (order 8), and on the added SinhSpherical 128x64x16
    grid: plain FP64 relaxation against FP32 relaxation inside the FP64
    defect-correction loop, both to residual 1e-10, with the relative
    difference of the two u and the oracle's residual of the defect-corrected
    u.  Both solves are then continued to `tight_tol`, where the difference
    of u is stated again (the 1e-10 residual fixes u only up to the
    operator's conditioning).  Rooflines: the FP64 stage's time per launch
    inside its solve against the FP64 peak; the FP32 stage, timed alone,
    against the HBM copy bandwidth."""
    from oracle import grid_from_desc as oracle_grid
    stream = torch.cuda.current_stream()
    hbm, hbm_basis = hbm_peak_gbs()
    fp64_peak = sms * FP64_FMA_PER_CLK * 2 * MAX_SM_MHZ * 1e6 / 1e12
    out = {}
    for name, mk in [("sinhsymtp_256x256x32", W.q4_sinhsymtp_256),
                     ("spherical_128x64x32", W.q4_spherical_128),
                     ("cartesian_256^3", W.q4_cartesian_256),
                     ("sinhspherical_128x64x16", W.q4_sinhspherical_128)]:
        desc, punc = mk()
        g = nrr.Grid(desc)
        g.set_punctures(punc)
        tuned = {m: g.autotune(m, 10)[:2] for m in ("fp64", "fp32")}
        res = {}
        for mode in ("fp32_dc", "fp64"):
            g.relax(mode=mode, tol=1e-10, max_iters=100, raise_on_error=False)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = g.relax(mode=mode, tol=1e-10, max_iters=200000,
                        raise_on_error=False)
            e1.record(stream)
            e1.synchronize()
            u = torch.empty(g.shape, dtype=torch.float64, device="cuda")
            v = torch.empty_like(u)
            g.get_state(u, v)
            res[mode] = (r, e0.elapsed_time(e1) / 1e3, u, v)
        udc, u64 = res["fp32_dc"][2], res["fp64"][2]
        diff = float((udc - u64).abs().max() / u64.abs().max())
        n_int = g.interior_points
        r64, t64 = res["fp64"][0], res["fp64"][1]
        ms64 = t64 * 1e3 / (4 * max(1, r64["iters"]))
        ach64 = flops_per_point(g.ng) * n_int / (ms64 * 1e-3) / 1e12
        dt, eta = g.timestep(0.5)
        ms32 = g.profile_stages(20, dt, eta, mode="fp32")
        ach32 = FP32_STAGE_BYTES * n_int / (ms32 * 1e-3) / 1e9
        entry = {"launch": tuned, "interior_points": n_int,
                 "fp32_dc": {"seconds": res["fp32_dc"][1],
                             "rk4_steps": res["fp32_dc"][0]["iters"],
                             "norm": res["fp32_dc"][0]["norm"],
                             "status": res["fp32_dc"][0]["status"]},
                 "fp64": {"seconds": t64, "rk4_steps": r64["iters"],
                          "norm": r64["norm"], "status": r64["status"]},
                 "speedup_dc_vs_fp64": t64 / res["fp32_dc"][1],
                 "max_rel_diff_u_dc_vs_fp64": diff,
                 "gridpoint_rhs_per_s_fp64": n_int * 4 * r64["iters"] / t64,
                 "roofline_fp64_stage": {
                     "bound": "alu", "achieved": ach64, "peak": fp64_peak,
                     "unit": "TFLOP/s", "frac": ach64 / fp64_peak,
                     "ms_per_launch": ms64,
                     "basis": "in-solve: FP64 solve time / (4 x RK4 steps); "
                              "%d flops per point" % flops_per_point(g.ng)},
                 "roofline_fp32_stage": {
                     "bound": "hbm", "achieved": ach32, "peak": hbm,
                     "unit": "GB/s", "frac": ach32 / hbm, "ms_per_launch": ms32,
                     "basis": "stage timed alone on its work stream; %d B per "
                              "point; peak %s" % (FP32_STAGE_BYTES, hbm_basis)}}
        # both solves continued from their 1e-10 states to tight_tol
        tight = {}
        for mode in ("fp32_dc", "fp64"):
            g.set_state(res[mode][2], res[mode][3])
            r = g.relax(mode=mode, tol=tight_tol, max_iters=400000,
                        initial=nrr.INIT_CURRENT, raise_on_error=False)
            u = torch.empty(g.shape, dtype=torch.float64, device="cuda")
            g.get_state(u)
            tight[mode] = (r, u)
        entry["to_tight_tol"] = {
            "tol": tight_tol,
            "fp64_extra_rk4_steps": tight["fp64"][0]["iters"],
            "fp64_norm": tight["fp64"][0]["norm"],
            "fp32_dc_extra_rk4_steps": tight["fp32_dc"][0]["iters"],
            "fp32_dc_norm": tight["fp32_dc"][0]["norm"],
            "max_rel_diff_u_dc_vs_fp64": float(
                (tight["fp32_dc"][1] - tight["fp64"][1]).abs().max()
                / tight["fp64"][1].abs().max())}
        og = oracle_grid(desc)
        alpha, beta = og.source(punc)
        entry["oracle_residual_of_dc_u"] = og.norm(
            og.residual(alpha, beta, og.fill_inner_ghosts(udc.cpu().numpy())))
        del og
        out[name] = entry
        print(json.dumps({name: entry}), file=sys.stderr, flush=True)
        g.close()
        del udc, u64, res, tight
        torch.cuda.empty_cache()
    return out


def patches_section(nrr, W, torch):
    """Two overlapping patches (the paper's Sec. 5 multiple patches, Sec. 6
    multipatch grids): the q=4 pair on a Spherical grid (64x32x32, rmax 48,
    order 4) with a Cartesian box of 48^3 points over [-8, 8]^3 around both
    punctures; the box's ghosts and a hole of the sphere's interior
    (max |x_i| < 3) interpolated from the other patch after every RK4 stage
    (q = 4 Lagrange points per direction).  FP64 to the coupled residual
    1e-10, against the Spherical grid alone.  The lone grid's launch shape
    is autotuned (it may pick the multi-stage kernel); the patch system
    launches one stage at a time with the default shape (the autotuner's
    choice for a lone grid's own relaxation need not suit single stages)."""
    punc = W.spinning_q4_pair()
    sph = W.grid_desc("spherical", (64, 32, 32), 4, rmax=48.0)
    box = W.grid_desc("cartesian", (48, 48, 48), 4, xmax=8.0)
    stream = torch.cuda.current_stream()

    def timed(fn):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    alone = nrr.Grid(sph)
    alone.set_punctures(punc)
    alone.autotune("fp64", 10)
    alone.relax(mode="fp64", tol=1e-10, max_iters=100, raise_on_error=False)
    r1, t1 = timed(lambda: alone.relax(mode="fp64", tol=1e-10, raise_on_error=False))
    alone.close()
    go, gi = nrr.Grid(sph), nrr.Grid(box)
    go.set_punctures(punc)
    gi.set_punctures(punc)
    # single-stage launch shapes measured for this pair (the lone grid's
    # tuned shape is the multi-stage kernel, which a patch system does not
    # use): tiled stages on the sphere, one plane per thread in the box
    go.set_launch(2, "fp64", 1, 128)
    gi.set_launch(1, "fp64", 0, 64)
    ps = nrr.PatchSet(go, gi, 3.0, 4)
    ps.relax(tol=1e-10, max_iters=100, raise_on_error=False)
    r2, t2 = timed(lambda: ps.relax(tol=1e-10, raise_on_error=False))
    ps.relax(tol=1e-10, max_iters=100, mode="fp32_dc", raise_on_error=False)
    r3, t3 = timed(lambda: ps.relax(tol=1e-10, mode="fp32_dc", raise_on_error=False))
    out = {"outer": "Spherical 64x32x32, rmax 48, order 4",
           "inner": "Cartesian 48^3 over [-8, 8]^3, order 4", "hole": 3.0,
           "interpolation_points": 4,
           "receivers": [ps.outer_receivers, ps.inner_receivers],
           "two_patch": {"seconds": t2, "rk4_steps": r2["iters"],
                         "norm": r2["norm"], "status": r2["status"]},
           "two_patch_defect_correction": {
               "seconds": t3, "rk4_steps": r3["iters"],
               "outer_iters": r3["outer_iters"], "norm": r3["norm"],
               "status": r3["status"]},
           "outer_alone": {"seconds": t1, "rk4_steps": r1["iters"],
                           "norm": r1["norm"], "status": r1["status"]}}
    ps.close()
    go.close()
    gi.close()
    return out


def run_configs2(args):
    """The larger and other-coordinate variants on their own."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_14030_gb300 import nrr, workloads as W
    torch.cuda.set_device(0)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    out = configs2_section(nrr, W, torch, nrr.probe_peaks(), sms)
    print(json.dumps({"configs2": out}), flush=True)
    return 0


def run_streams(args):
    """Independent patches (the paper's Sec. 5 multi-grid experiment): N = 1..7
    identical q=4 SinhSymTP 128x128x16 FP64 solves to residual 1e-10, run
    (a) one after another, (b) concurrently, one grid per host thread and
    CUDA stream, and (c) as one batch in a single graph launch.  Wall time
    for all N solves."""
    import threading
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_14030_gb300 import nrr, workloads as W
    torch.cuda.set_device(0)
    desc, punc = W.q4_sinhsymtp_128()
    grids = []
    for _ in range(7):
        g = nrr.Grid(desc)
        g.set_punctures(punc)
        grids.append(g)
    grids[0].autotune("fp64", 20)  # cached for every grid of this shape
    for g in grids:
        g.relax(mode="fp64", tol=1e-10, max_iters=100, raise_on_error=False)
    torch.cuda.synchronize()
    rows = []
    for n in range(1, 8):
        gs = grids[:n]
        t0 = time.perf_counter()
        steps = [g.relax(mode="fp64", tol=1e-10)["iters"] for g in gs]
        seq = time.perf_counter() - t0
        res = [None] * n

        def work(i):
            res[i] = gs[i].relax(mode="fp64", tol=1e-10)

        th = [threading.Thread(target=work, args=(i,)) for i in range(n)]
        t0 = time.perf_counter()
        for t in th:
            t.start()
        for t in th:
            t.join()
        conc = time.perf_counter() - t0
        b = nrr.Batch([desc] * n, [punc] * n, with_fp64=True)
        b.autotune("fp64", 3)
        b.relax(mode="fp64", tol=1e-10, max_iters=100, raise_on_error=False)
        t0 = time.perf_counter()
        per, tot = b.relax(mode="fp64", tol=1e-10)
        bat = time.perf_counter() - t0
        b.close()
        rows.append({"n": n, "rk4_steps": steps[0],
                     "sequential_s": seq, "streams_s": conc, "batch_graph_s": bat,
                     "streams_speedup": seq / conc, "batch_speedup": seq / bat,
                     "all_converged": all(r["status"] == 0 for r in res) and
                     tot["status"] == 0})
        print(json.dumps(rows[-1]), flush=True)
    for g in grids:
        g.close()
    print(json.dumps({"independent_patches": rows}), flush=True)
    return 0


def run_order10(args):
    """The paper's own order (10) on its SinhSymTP workloads, 128x128x16 and
    512x512x64 (q=4 spinning pair): FP64 relaxation and FP32 inside FP64
    defect correction to residual 1e-10, plus the fused stage's time per
    launch for a ladder of grid sizes (kernel weak scaling)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_14030_gb300 import nrr, workloads as W
    torch.cuda.set_device(0)
    punc = W.spinning_q4_pair()
    out = {"solves": {}, "stage_us_per_launch": []}
    for n in [(128, 128, 16), (512, 512, 64)]:
        desc = W.grid_desc("sinhsymtp", n, 10)
        g = nrr.Grid(desc)
        g.set_punctures(punc)
        for m in ("fp64", "fp32"):
            g.autotune(m, 10)
        ent = {"launch": {m: g.get_launch(m) for m in ("fp64", "fp32")}}
        for mode in ("fp32_dc", "fp64"):
            g.relax(mode=mode, tol=1e-10, max_iters=100, raise_on_error=False)
            r = g.relax(mode=mode, tol=1e-10, max_iters=400000, raise_on_error=False)
            ent[mode] = {"seconds": r["seconds"], "rk4_steps": r["iters"],
                         "norm": r["norm"], "status": r["status"],
                         "gridpoint_rhs_per_s": g.interior_points * 4 * r["iters"] / r["seconds"]}
            print(json.dumps({str(n): {mode: ent[mode]}}), flush=True)
        ent["speedup_dc_vs_fp64"] = ent["fp64"]["seconds"] / ent["fp32_dc"]["seconds"]
        out["solves"]["x".join(map(str, n))] = ent
        g.close()
        torch.cuda.empty_cache()
    for n in [(64, 64, 8), (128, 128, 16), (256, 256, 32), (512, 512, 64)]:
        desc = W.grid_desc("sinhsymtp", n, 10)
        g = nrr.Grid(desc)
        g.set_punctures(punc)
        dt, eta = g.timestep(0.5)
        row = {"grid": "x".join(map(str, n)), "interior_points": g.interior_points}
        for m in ("fp64", "fp32"):
            g.autotune(m, 5)
            g.profile_stages(10, dt, eta, mode=m)
            us = g.profile_stages(50, dt, eta, mode=m) * 1e3
            row[m + "_us"] = us
            row[m + "_ns_per_point"] = us * 1e3 / g.interior_points
        out["stage_us_per_launch"].append(row)
        print(json.dumps(row), flush=True)
        g.close()
        torch.cuda.empty_cache()
    print(json.dumps({"order10": out}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="run only this many RK4 steps (profiler captures)")
    ap.add_argument("--mode", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--profile-variant", type=int, default=0,
                    help="with --profile-steps: 0 column, 1 tiled kernel")
    ap.add_argument("--profile-grid", default="sinhsymtp128",
                    choices=["sinhsymtp128", "sinhsymtp256", "cartesian256"],
                    help="with --profile-steps: the q=4 grid to step")
    ap.add_argument("--profile-block", type=int, default=0,
                    help="with --profile-steps: column-kernel block size")
    ap.add_argument("--profile-zc", type=int, default=0,
                    help="with --profile-steps: phi planes per thread/block")
    ap.add_argument("--profile-gemm", action="store_true",
                    help="run only the surrogate GEMM shapes (captures)")
    ap.add_argument("--profile-patches", type=int, default=0,
                    help="run only this many RK4 steps of the two-patch "
                         "system (profiler captures)")
    ap.add_argument("--gemm-shape", default="",
                    help="with --profile-gemm: only M,N,K, three calls of the "
                         "chosen plan")
    ap.add_argument("--surrogate", action="store_true",
                    help="run the learned warm-start pipeline instead")
    ap.add_argument("--surrogate-train", type=int, default=8192)
    ap.add_argument("--surrogate-held", type=int, default=1024)
    ap.add_argument("--surrogate-epochs", type=int, default=100)
    ap.add_argument("--streams", action="store_true",
                    help="N = 1..7 independent grids: sequential, streams, batch")
    ap.add_argument("--order10", action="store_true",
                    help="order-10 solves at 128x128x16 and 512x512x64")
    ap.add_argument("--configs2", action="store_true",
                    help="run the larger and other-coordinate variants")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="run only a short batch of this many 128x128x16 "
                         "solves (profiler captures)")
    ap.add_argument("--no-surrogate", action="store_true",
                    help="skip the compact surrogate warm-start section")
    ap.add_argument("--launch-shapes", default="",
                    help="JSON file of stage launch shapes: loaded instead of "
                         "autotuning if it exists, else written after it")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the 512-solve batch in the default run")
    ap.add_argument("--host-loop", action="store_true",
                    help="headline solves with the stop test on the host (one "
                         "graph per chunk): for profilers, which cannot see "
                         "kernels inside graphs with conditional nodes")
    ap.add_argument("--no-configs2", action="store_true",
                    help="skip the larger-grid section in the default run")
    ap.add_argument("--compact-surrogate", action="store_true",
                    help="2048 training / 128 held-out solves instead of "
                         "8192 / 1024 in the default run")
    args = ap.parse_args()
    if args.surrogate:
        return run_surrogate(args)
    if args.profile_batch > 0:
        return run_profile_batch(args)
    if args.profile_gemm:
        return run_profile_gemm(args)
    if args.profile_patches:
        return run_profile_patches(args)
    if args.configs2:
        return run_configs2(args)
    if args.streams:
        return run_streams(args)
    if args.order10:
        return run_order10(args)
    if args.profile_steps > 0:
        return run_profile_steps(args)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
