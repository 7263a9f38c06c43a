"""The warm-start network on the device against the CPU reference network:
gradients (per tensor), predictions, and that training lowers the loss."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import mlp
from paper_2501_14030_gb300 import nrr, workloads as W

pytestmark = pytest.mark.gpu

# BF16 operands round to 2^-9 relative; values near a rounding boundary can
# round differently on the device (FP32 sums) and in the reference (FP64
# sums), so a gradient tensor may differ by a few BF16 ulps of its largest
# entries: 2e-2 of its maximum.
GRAD_TOL = 2e-2


def _data(B, dims, seed):
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1, 1, (B, dims[0])).astype(np.float32)
    Y = rng.standard_normal((B, dims[-1])).astype(np.float32)
    return X, Y


@pytest.mark.parametrize("dims,batch", [([12, 128, 128, 256], 128),
                                        (W.mlp_dims(), 256)])
def test_gradients_match_reference(gpu, dims, batch):
    init = W.mlp_init_params(dims, seed=1)
    X, Y = _data(batch, dims, seed=2)
    s = nrr.Surrogate(dims, init, batch=batch)
    loss, g = s.gradients(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda())
    params = mlp.unpack(init.astype(np.float64), dims)
    loss_ref, grads_ref = mlp.loss_and_grads(params, X, Y, round_bf16=True)
    assert abs(loss - loss_ref) <= 1e-3 * loss_ref
    gd = mlp.unpack(g.astype(np.float64), dims)
    for l, ((dw, db), (rw, rb)) in enumerate(zip(gd, grads_ref)):
        assert np.abs(dw - rw).max() <= GRAD_TOL * np.abs(rw).max(), l
        assert np.abs(db - rb).max() <= GRAD_TOL * np.abs(rb).max(), l
        # and closely in the aggregate
        assert np.linalg.norm(dw - rw) <= 5e-3 * np.linalg.norm(rw), l
    s.close()


def test_training_lowers_loss_and_predict_matches_reference(gpu):
    dims, batch, n = [12, 128, 128, 256], 128, 2048
    rng = np.random.default_rng(5)
    X = rng.uniform(-1, 1, (n, 12)).astype(np.float32)
    A = rng.standard_normal((12, 256)).astype(np.float32)
    Y = (np.sin(0.3 * X @ A) + 0.05 * (0.3 * X @ A) ** 2).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    s = nrr.Surrogate(dims, W.mlp_init_params(dims, seed=6), batch=batch)
    s.fit_scaling(Yd)
    order = torch.from_numpy(W.minibatch_order(n, batch, 600, seed=7)).cuda()
    losses = s.train(Xd, Yd, order, 600, lr=2e-3)
    assert np.all(np.isfinite(losses))
    assert losses[-20:].mean() < 0.1 * losses[:5].mean(), (losses[:5], losses[-20:])
    out = torch.empty((n, 256), dtype=torch.float32, device="cuda")
    s.predict(Xd, out)
    p = mlp.unpack(s.params().astype(np.float64), dims)
    Zs, _ = mlp.forward(p, X[:300], round_bf16=True)
    mean, std = Y.mean(0), Y.std(0)
    ref = Zs[-1] * np.maximum(std, 1e-3 * std.max()) + mean
    got = out[:300].cpu().numpy()
    assert np.abs(got - ref).max() <= 2e-2 * np.abs(ref).max()
    s.close()


def test_replayed_training_steps_equal_host_launched_steps(gpu):
    """A call of several steps replays one captured training step (device
    step counter, per-step AdamW corrections); one-step calls launch each
    step from the host.  Five steps either way: identical parameters and
    losses, bit for bit."""
    dims, batch, n = [12, 128, 128, 256], 128, 1024
    rng = np.random.default_rng(8)
    X = rng.uniform(-1, 1, (n, 12)).astype(np.float32)
    Y = rng.standard_normal((n, 256)).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    order = torch.from_numpy(W.minibatch_order(n, batch, 5, seed=9)).cuda()
    init = W.mlp_init_params(dims, seed=10)
    a = nrr.Surrogate(dims, init, batch=batch)
    b = nrr.Surrogate(dims, init, batch=batch)
    for s in (a, b):
        s.fit_scaling(Yd)
    la = a.train(Xd, Yd, order, 5, lr=2e-3)
    lb = np.concatenate([b.train(Xd, Yd, order[t * batch:(t + 1) * batch].contiguous(),
                                 1, lr=2e-3) for t in range(5)])
    assert np.array_equal(la, lb)
    assert np.array_equal(a.params(), b.params())
    a.close()
    b.close()
