"""Pins of the CPU reference network (exact FP64 mode) to central
differences of its own loss, and of its BF16 rounding to known values."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp
from paper_2501_14030_gb300 import workloads as W


def test_bf16_rounding_known_values():
    x = np.array([1.0, 1.00390625, 1.005859375, 3.14159, -2.0e-3, 65504.0])
    r = mlp.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0          # tie to even: down
    assert r[2] == 1.0078125                     # above the tie: up
    assert r[3] == 3.140625
    assert abs(r[4] + 0.001998901) < 1e-9
    assert r[5] == 65536.0


def test_gelu_derivative_matches_difference():
    x = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.gelu(x + h) - mlp.gelu(x - h)) / (2 * h)
    assert np.abs(fd - mlp.gelu_grad(x)).max() < 1e-8


def test_reference_gradients_match_central_differences():
    dims = [12, 16, 16, 8]
    flat = W.mlp_init_params(dims, seed=3).astype(np.float64)
    rng = np.random.default_rng(4)
    X = rng.uniform(-1, 1, (5, 12))
    Y = rng.standard_normal((5, 8))
    params = mlp.unpack(flat, dims)
    loss, grads = mlp.loss_and_grads(params, X, Y, round_bf16=False)
    g = mlp.pack(grads)
    idx = rng.choice(flat.size, 40, replace=False)
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = mlp.loss_and_grads(mlp.unpack(fp, dims), X, Y, round_bf16=False)
        lm, _ = mlp.loss_and_grads(mlp.unpack(fm, dims), X, Y, round_bf16=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
