"""Host check (no GPU) of the index arithmetic of the batched tensor-copy
stage: it finds an operand's field index f in its precision's arena as
rint(float(f * stride) / float(stride)) in FP32 instead of a 64-bit integer
division.  Each float conversion and the division round once (relative
error at most 2^-24 each), so the quotient is within about 3 x 2^-24 f
(1.8e-7 f) of f and rounds back to f for any f below 2^20.  numpy's
float32 arithmetic rounds as the device does (round to nearest, correctly
rounded division), so the claim is checked here for every f an arena can
hold and for strides up to the 2^31-point limit of an arena.
"""
from __future__ import annotations

import numpy as np


def _field_index(off: np.ndarray, stride: np.ndarray) -> np.ndarray:
    return np.rint(off.astype(np.float32) / stride.astype(np.float32)).astype(np.int64)


def test_fp32_field_index_is_exact():
    rng = np.random.default_rng(20250124)
    strides = np.concatenate([
        np.array([1, 2, 3, 7, 2**20 - 1, 2**20 + 1, 2**24 - 1, 2**24 + 1,
                  2**30 + 3, 2**31 - 1, 2**31], dtype=np.int64),
        rng.integers(1, 2**31, size=4000, dtype=np.int64),
    ])
    f = np.arange(0, 65, dtype=np.int64)  # an arena holds 11 fields at most
    off = f[None, :] * strides[:, None]
    got = _field_index(off, np.broadcast_to(strides[:, None], off.shape))
    assert np.array_equal(got, np.broadcast_to(f[None, :], off.shape))


def test_fp32_field_index_would_fail_without_rounding():
    """Truncation instead of rounding is wrong for some strides (the
    quotient can land just below f), which is why the kernel rounds."""
    rng = np.random.default_rng(7)
    strides = rng.integers(2**24, 2**31, size=4000, dtype=np.int64)
    f = np.arange(1, 12, dtype=np.int64)
    off = f[None, :] * strides[:, None]
    q = off.astype(np.float32) / np.broadcast_to(strides[:, None], off.shape).astype(np.float32)
    assert (np.trunc(q).astype(np.int64) != f[None, :]).any()
