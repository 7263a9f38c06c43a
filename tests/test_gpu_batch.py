"""Batches of independent solves of uneven sizes (one graph launch each):
every member must match its single-grid solve and satisfy the oracle."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2501_14030_gb300 import nrr, workloads as W
from tests.helpers import oracle_grid, rel_err

pytestmark = pytest.mark.gpu


def small_batch(count=5, seed=7):
    """Seeded parameter draws on small uneven SinhSymTP grids (order 4)."""
    rng = np.random.default_rng(seed)
    params = W.batch_parameters(count, seed)
    descs, puncs = [], []
    for p in params:
        n = (int(rng.choice([16, 20, 24])), int(rng.choice([8, 12, 16])),
             int(rng.choice([2, 4])))
        descs.append(W.grid_desc("sinhsymtp", n, 4, bscale=p["d"] / 2))
        puncs.append(p["punctures"])
    return descs, puncs


def _single(desc, punc, mode):
    g = nrr.Grid(desc)
    g.set_punctures(punc)
    r = g.relax(mode=mode, tol=1e-10, check_every=50)
    u = np.zeros(g.shape)
    g.get_state(u)
    g.close()
    return r, u


def test_batch_fp64_equals_single_grid_solves(gpu):
    descs, puncs = small_batch()
    b = nrr.Batch(descs, puncs, with_fp64=True)
    per, tot = b.relax(mode="fp64", tol=1e-10, check_every=50)
    assert tot["status"] == 0
    for i, (d, p) in enumerate(zip(descs, puncs)):
        r, u1 = _single(d, p, "fp64")
        ub = np.zeros(b.shapes[i])
        b.get_u(i, ub)
        assert per[i]["status"] == 0 and per[i]["iters"] == r["iters"]
        assert rel_err(ub, u1) <= 1e-12, (i, rel_err(ub, u1))
        og = oracle_grid(d)
        alpha, beta = og.source(p)
        assert og.norm(og.residual(alpha, beta, ub)) < 1.02e-10


def test_batch_defect_correction_converges_every_solve(gpu):
    descs, puncs = small_batch(count=6, seed=11)
    b = nrr.Batch(descs, puncs)
    b.autotune("fp32_dc", 3)
    per, tot = b.relax(mode="fp32_dc", tol=1e-10, check_every=50)
    assert tot["status"] == 0
    for i, (d, p) in enumerate(zip(descs, puncs)):
        r, u1 = _single(d, p, "fp64")
        ub = np.zeros(b.shapes[i])
        b.get_u(i, ub)
        assert per[i]["status"] == 0 and per[i]["norm"] < 1e-10
        assert abs(per[i]["iters"] - r["iters"]) <= 100, (per[i], r)
        og = oracle_grid(d)
        alpha, beta = og.source(p)
        assert og.norm(og.residual(alpha, beta, ub)) < 1.02e-10


def test_batch_member_already_converged(gpu):
    """A Brill-Lindquist member has zero source: done at step 0 and exactly
    zero, while the others relax."""
    descs, puncs = small_batch(count=3, seed=3)
    descs.append(W.grid_desc("sinhsymtp", (16, 8, 2), 4))
    puncs.append(W.brill_lindquist_pair())
    b = nrr.Batch(descs, puncs)
    per, tot = b.relax(mode="fp32_dc", tol=1e-10)
    assert tot["status"] == 0
    assert per[-1]["iters"] == 0 and per[-1]["norm"] == 0.0
    u = np.ones(b.shapes[-1])
    b.get_u(len(descs) - 1, u)
    assert not u.any()
    assert all(p["iters"] > 0 for p in per[:-1])


def test_batch_limits_end_the_graph(gpu):
    """The WHILE loop stops at the step limit and at the device-timed
    wall-clock limit, reporting the status per solve."""
    descs, puncs = small_batch(count=3, seed=5)
    b = nrr.Batch(descs, puncs)
    per, tot = b.relax(mode="fp32_dc", tol=1e-10, max_iters=100,
                       raise_on_error=False)
    assert tot["status"] == nrr.ERR_NOT_CONVERGED
    assert all(p["status"] == nrr.ERR_NOT_CONVERGED and p["iters"] == 100
               for p in per)
    big = [W.q4_sinhsymtp_128()[0]]
    bb = nrr.Batch(big, [W.spinning_q4_pair()])
    per, tot = bb.relax(mode="fp32_dc", tol=1e-10, timeout_ms=1,
                        raise_on_error=False)
    assert tot["status"] == nrr.ERR_TIMEOUT
    assert per[0]["status"] == nrr.ERR_TIMEOUT and per[0]["iters"] < 6400


def aligned_batch(count=4, seed=5, coord="sinhsymtp"):
    """Order-8 grids that admit the tensor-copy stage variant (n0 % 32 == 0,
    n1 % 4 == 0), uneven sizes including the axis and theta-edge tiles."""
    rng = np.random.default_rng(seed)
    params = W.batch_parameters(count, seed)
    descs, puncs = [], []
    for p in params:
        n = (int(rng.choice([32, 64])), int(rng.choice([8, 12, 20])),
             int(rng.choice([4, 8])))
        descs.append(W.grid_desc(coord, n, 8, bscale=p["d"] / 2))
        puncs.append(p["punctures"])
    return descs, puncs


@pytest.mark.parametrize("coord,mode", [("sinhsymtp", "fp32_dc"),
                                        ("sinhsymtp", "fp64"),
                                        ("spherical", "fp32_dc")])
def test_batch_stage_variants_bitwise_equal(gpu, coord, mode):
    """The batch stage kernels (register-staged tiles, tensor-copy tiles,
    columns) evaluate the same arithmetic in the same order on the same
    operands: after 300 RK4 steps every solve agrees bit for bit, for each
    plane chunking."""
    descs, puncs = aligned_batch(coord=coord)
    results = []
    for var, zc in [(0, 4), (1, 2), (1, 4), (1, 16), (2, 1), (2, 2)]:
        b = nrr.Batch(descs, puncs, with_fp64=(mode == "fp64"))
        b.set_launch(var, zc, mode)
        per, _ = b.relax(mode=mode, tol=1e-30, max_iters=300, check_every=50,
                         raise_on_error=False)
        us = []
        for i in range(len(descs)):
            ub = np.zeros(b.shapes[i])
            b.get_u(i, ub)
            us.append(ub)
        results.append(([r["norm"] for r in per], us))
        b.close()
    norms0, us0 = results[0]
    assert all(np.isfinite(norms0)) and max(norms0) > 0
    for norms, us in results[1:]:
        assert norms == norms0
        for a, b_ in zip(us, us0):
            assert np.array_equal(a, b_)


def test_tensor_copy_variant_refused_for_unaligned_grids(gpu):
    descs, puncs = small_batch(count=2)
    b = nrr.Batch(descs, puncs)
    with pytest.raises(nrr.NrrError):
        b.set_launch(1, 4, "fp32_dc")
    b.set_launch(0, 4, "fp32_dc")
    b.close()


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_expires_and_context_survives(gpu, which):
    """A tensor-copy wait (0) and a grid barrier (1) on events that never
    happen give up, record their error and return; the next solve on the
    same context still converges."""
    import time
    t0 = time.perf_counter()
    assert nrr.selftest_wait_expiry(which)
    assert time.perf_counter() - t0 < 60.0
    desc, punc = W.small_equal_mass()
    g = nrr.Grid(desc)
    g.set_punctures(punc)
    r = g.relax(mode="fp64", tol=1e-10)
    assert r["status"] == 0 and r["norm"] < 1e-10
    g.close()


def test_full_sweep_sampled_solves_checked_by_oracle(gpu):
    """The 512-solve parameter sweep at full size, in the launch shape the
    bench times (autotuned, defect correction, one graph launch): every solve
    converges, and the oracle's residual of eight sampled solves (the largest
    and smallest grids among them) is below the threshold too."""
    params = W.batch_parameters(512, 20250124)
    descs = [p["desc"] for p in params]
    b = nrr.Batch(descs, [p["punctures"] for p in params])
    b.autotune("fp32_dc", 3)
    per, tot = b.relax(mode="fp32_dc", tol=1e-10)
    assert tot["status"] == 0
    assert all(r["status"] == 0 and r["norm"] < 1e-10 for r in per)
    size = [int(np.prod(d["n"])) for d in descs]
    order = np.argsort(size)
    rng = np.random.default_rng(9)
    pick = sorted({int(order[0]), int(order[-1]),
                   *map(int, rng.choice(512, size=6, replace=False))})
    for i in pick:
        ub = np.zeros(b.shapes[i])
        b.get_u(i, ub)
        og = oracle_grid(descs[i])
        alpha, beta = og.source(params[i]["punctures"])
        assert og.norm(og.residual(alpha, beta, ub)) < 1.02e-10, (i, descs[i]["n"])
    b.close()
