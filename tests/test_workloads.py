"""The seeded synthetic inputs against the workload definitions they stand
for: the named puncture configurations, the 512-solve parameter sweep's
ranges, the surrogate's input scaling and minibatch order, and the
determinism of every generator (CPU only)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2501_14030_gb300 import workloads as W


def test_named_configurations():
    small, pe = W.small_equal_mass()
    assert small["coord"] == "sinhsymtp" and small["n"] == (32, 16, 2)
    assert small["order"] == 4
    assert (small["amax"], small["bscale"], small["sinhwaa"]) == (1.0e4, 5.0, 0.07)
    assert [p["m"] for p in pe] == [0.5, 0.5]
    assert [p["x"] for p in pe] == [(0.0, 0.0, 5.0), (0.0, 0.0, -5.0)]
    assert [p["P"] for p in pe] == [(0.1, 0.0, 0.0), (-0.1, 0.0, 0.0)]
    assert all(p["S"] == (0.0, 0.0, 0.0) for p in pe)

    desc, pq = W.q4_sinhsymtp_128()
    assert desc["n"] == (128, 128, 16) and desc["order"] == 8
    assert [p["m"] for p in pq] == [0.8, 0.2]
    assert pq[0]["x"][2] - pq[1]["x"][2] == 10.0
    assert [p["P"] for p in pq] == [(0.09, 0.0, 0.0), (-0.09, 0.0, 0.0)]
    # spin angular momentum S = chi m^2 with the bare masses
    np.testing.assert_allclose(pq[0]["S"], np.array([0.3, -0.2, 0.5]) * 0.64)
    np.testing.assert_allclose(pq[1]["S"], np.array([0.0, 0.4, -0.1]) * 0.04)

    assert W.q4_sinhsymtp_256()[0]["n"] == (256, 256, 32)
    assert W.q4_spherical_128()[0]["n"] == (128, 64, 32)
    assert W.q4_cartesian_256()[0]["n"] == (256, 256, 256)
    assert all(p["P"] == (0.0, 0.0, 0.0) and p["S"] == (0.0, 0.0, 0.0)
               for p in W.brill_lindquist_pair())


def test_batch_sweep_ranges_and_determinism():
    params = W.batch_parameters(400, seed=7)
    assert params == W.batch_parameters(400, seed=7)
    assert params != W.batch_parameters(400, seed=8)
    for p in params:
        assert 1.0 <= p["q"] <= 8.0 and 6.0 <= p["d"] <= 16.0
        assert np.linalg.norm(p["P"]) <= 0.15 + 1e-15
        assert np.linalg.norm(p["chi1"]) <= 0.8 + 1e-15
        assert np.linalg.norm(p["chi2"]) <= 0.8 + 1e-15
        a, b = p["punctures"]
        assert a["m"] + b["m"] == pytest.approx(1.0)
        assert a["m"] / b["m"] == pytest.approx(p["q"])
        assert a["x"] == (0.0, 0.0, p["d"] / 2) and b["x"] == (0.0, 0.0, -p["d"] / 2)
        np.testing.assert_allclose(a["P"], -np.asarray(b["P"]))
        np.testing.assert_allclose(a["S"], np.asarray(p["chi1"]) * a["m"] ** 2)
        np.testing.assert_allclose(b["S"], np.asarray(p["chi2"]) * b["m"] ** 2)
        desc = p["desc"]
        assert desc["order"] == 8 and desc["bscale"] == p["d"] / 2
        n0, n1, n2 = desc["n"]
        assert n0 in (64, 96, 128) and n1 in (32, 64, 96, 128) and n2 in (8, 16)
    # the draws cover the ranges (uniform, 400 samples)
    q = np.array([p["q"] for p in params])
    d = np.array([p["d"] for p in params])
    assert q.min() < 1.5 and q.max() > 7.5 and d.min() < 7.0 and d.max() > 15.0
    assert {p["desc"]["n"][2] for p in params} == {8, 16}


def test_surrogate_inputs_are_scaled_to_unit_box():
    params = W.batch_parameters(300, seed=3)
    x = W.surrogate_inputs(params)
    assert x.shape == (300, 12) and x.dtype == np.float32
    assert np.abs(x).max() <= 1.0 + 1e-6
    assert np.all(x[:, 11] == 1.0)  # total mass


def test_minibatch_order_is_a_sequence_of_permutations():
    order = W.minibatch_order(n=100, batch=32, steps=20, seed=5)
    assert order.shape == (640,) and order.dtype == np.int32
    for k in range(6):
        assert sorted(order[100 * k:100 * (k + 1)]) == list(range(100))
    assert np.array_equal(order, W.minibatch_order(100, 32, 20, 5))


def test_smooth_random_field_is_seeded_and_bounded():
    desc = W.grid_desc("sinhsymtp", (44, 26, 6), 8)
    f = W.smooth_random_field(desc, seed=11, amplitude=0.2)
    assert f.shape == W.padded_shape(desc) == (14, 34, 52)
    assert np.array_equal(f, W.smooth_random_field(desc, seed=11, amplitude=0.2))
    assert 0.0 < np.abs(f).max() <= 0.2 + 1e-15
    g = W.smooth_random_field(desc, seed=11, amplitude=0.2, noise=0.01)
    assert 0.0 < np.abs(g - f).max() < 0.1


def test_mlp_initialisation_layout():
    dims = W.mlp_dims()
    assert dims == [12, 512, 512, 512, 512, 64 * 32 * 8]
    p = W.mlp_init_params(dims, seed=1)
    n = sum(o * i + o for i, o in zip(dims[:-1], dims[1:]))
    assert p.shape == (n,) and p.dtype == np.float32
    # first layer: W [512][12] with variance 2/12, then 512 zero biases
    w0 = p[:512 * 12]
    assert abs(w0.var() - 2.0 / 12) < 0.02
    assert not p[512 * 12:512 * 13].any()
