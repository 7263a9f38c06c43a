"""Plain FP64 CPU reference of the warm-start surrogate network.

TEST INFRASTRUCTURE ONLY (see the package docstring): the checker of the
device forward/backward.  Straight numpy: layers Z_l = A_{l-1} W_l^T + b_l,
A_l = GELU(Z_l) on hidden layers (GELU(x) = x Phi(x)), linear last layer, loss
= mean of (Z_L - (Y - mean)/std)^2.  With ``round_bf16`` the operands of
every product are rounded to BF16 (ties to even) where the device rounds
them: inputs, weights, hidden activations and the back-propagated dZ; sums
and everything else stay FP64.  Without it the reference is the exact
function, which ``tests`` pin with central differences.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)


def unpack(flat: np.ndarray, dims):
    """Logical packed parameters -> [(W [out][in], b [out])] per layer."""
    out, off = [], 0
    for din, dout in zip(dims[:-1], dims[1:]):
        W = flat[off:off + din * dout].reshape(dout, din)
        off += din * dout
        b = flat[off:off + dout]
        off += dout
        out.append((W.astype(np.float64), b.astype(np.float64)))
    assert off == flat.size
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def forward(params, X, round_bf16=True):
    R = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    A = R(X)
    Zs, As = [], [A]
    for l, (W, b) in enumerate(params):
        Z = A @ R(W).T + b
        Zs.append(Z)
        if l < len(params) - 1:
            A = R(gelu(Z))
            As.append(A)
    return Zs, As


def loss_and_grads(params, X, Y, mean=None, std=None, round_bf16=True):
    """Mean squared error of the scaled outputs and the parameter gradients
    (same nesting as params)."""
    R = bf16 if round_bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Zs, As = forward(params, X, round_bf16)
    Yn = np.asarray(Y, dtype=np.float64)
    if mean is not None:
        Yn = (Yn - mean) / std
    ZL = Zs[-1]
    B, O = ZL.shape
    loss = float(np.mean((ZL - Yn) ** 2))
    dZ = 2.0 * (ZL - Yn) / (B * O)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        W, _ = params[l]
        dW = R(dZ).T @ As[l]
        db = dZ.sum(axis=0)
        grads[l] = (dW, db)
        if l > 0:
            dA = R(dZ) @ R(W)
            dZ = dA * gelu_grad(Zs[l - 1])
    return loss, grads
