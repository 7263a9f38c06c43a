"""The learned warm start end to end at a small scale: solver-generated
coarse solutions train the network on the device; its predictions for
held-out parameters, prolonged to a finer grid, start relaxations that still
reach the 1e-10 residual (confirmed by the oracle) in fewer steps than the
same solves started from zero."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from paper_2501_14030_gb300 import nrr, workloads as W
from tests.helpers import oracle_grid

pytestmark = pytest.mark.gpu


def _descs(params, n):
    return [W.grid_desc("sinhsymtp", n, 8, bscale=p["d"] / 2) for p in params]


def test_prolongation_reproduces_smooth_field(gpu):
    """Trilinear prolongation of a field linear in xx is exact away from the
    boundaries."""
    coarse = W.grid_desc("sinhsymtp", (16, 8, 4), 8)
    fine = W.grid_desc("sinhsymtp", (32, 16, 8), 8)
    og_c, og_f = oracle_grid(coarse), oracle_grid(fine)
    ng = 4
    f = lambda g: 0.3 + 0.5 * g.field("xx0") - 0.2 * g.field("xx1")
    uc = f(og_c)[ng:-ng, ng:-ng, ng:-ng].astype(np.float32).copy()
    uf = torch.zeros(og_f.shape, dtype=torch.float64, device="cuda")
    nrr.prolong(coarse, torch.from_numpy(uc).cuda(), fine, uf)
    got = uf.cpu().numpy()
    exp = f(og_f)
    inner = (slice(ng, -ng), slice(ng + 1, -ng - 1), slice(ng + 1, -ng - 1))
    assert np.abs(got[inner] - exp[inner]).max() < 1e-6


def test_learned_warm_start_beats_cold_start(gpu):
    coarse_n, fine_n = (32, 16, 4), (64, 32, 8)
    train = W.batch_parameters(256, seed=1)
    b = nrr.Batch(_descs(train, coarse_n), [p["punctures"] for p in train])
    per, tot = b.relax(mode="fp32_dc", tol=1e-10)
    assert tot["status"] == 0
    n_out = int(np.prod(coarse_n))
    Y = torch.empty((len(train), n_out), dtype=torch.float32, device="cuda")
    b.get_interior(Y)
    X = torch.from_numpy(W.surrogate_inputs(train)).cuda()
    dims = [12, 256, 256, n_out]
    s = nrr.Surrogate(dims, W.mlp_init_params(dims, seed=3), batch=128)
    s.fit_scaling(Y)
    steps = 1500
    order = torch.from_numpy(W.minibatch_order(len(train), 128, steps, seed=4)).cuda()
    losses = s.train(X, Y, order, steps, lr=1e-3)
    assert losses[-50:].mean() < 0.05 * losses[:10].mean()

    held = W.batch_parameters(12, seed=2)
    fdescs = _descs(held, fine_n)
    cold = nrr.Batch(fdescs, [p["punctures"] for p in held])
    per_c, tot_c = cold.relax(mode="fp32_dc", tol=1e-10)
    assert tot_c["status"] == 0
    Xh = torch.from_numpy(W.surrogate_inputs(held)).cuda()
    pred = torch.empty((len(held), n_out), dtype=torch.float32, device="cuda")
    s.predict(Xh, pred)
    warm = nrr.Batch(fdescs, [p["punctures"] for p in held])
    shape = W.padded_shape(fdescs[0])
    for i, p in enumerate(held):
        uf = torch.zeros(shape, dtype=torch.float64, device="cuda")
        nrr.prolong(_descs([p], coarse_n)[0], pred[i].contiguous(), fdescs[i], uf)
        warm.set_u(i, uf)
    per_w, tot_w = warm.relax(mode="fp32_dc", tol=1e-10, initial=nrr.INIT_DEVICE)
    assert tot_w["status"] == 0
    it_c = np.array([r["iters"] for r in per_c])
    it_w = np.array([r["iters"] for r in per_w])
    assert it_w.mean() < 0.9 * it_c.mean(), (it_c, it_w)
    for i in (0, 5):
        og = oracle_grid(fdescs[i])
        alpha, beta = og.source(held[i]["punctures"])
        u = np.zeros(shape)
        warm.get_u(i, u)
        assert og.norm(og.residual(alpha, beta, u)) < 1.02e-10
