"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds inputs only -- puncture parameter sets, grid descriptors and
seeded random grid functions -- and none of the solver's arithmetic.  Both the
CUDA path and the CPU oracle receive their inputs from here.

Grid descriptors are plain dicts: ``coord`` ("sinhsymtp" | "spherical" |
"cartesian" | "sinhspherical" | "sinhcylindrical"), ``n`` (interior points
per direction), ``order`` (centred FD order) and the coordinate parameters
``amax``, ``bscale``, ``sinhwaa``, ``rmax``, ``xmax``, ``zmax``, ``sinhwz``
(SinhCylindrical: rho = amax sinh(xx0/sinhwaa)/sinh(1/sinhwaa), z = zmax
sinh(xx1/sinhwz)/sinh(1/sinhwz), stored as (rho, z, phi)).

Puncture dicts: ``m`` (bare mass), ``x`` (position), ``P`` (momentum), ``S``
(spin angular momentum; a dimensionless spin chi maps to S = chi m^2).
"""
from __future__ import annotations

import numpy as np

COORDS = {"sinhsymtp": 0, "spherical": 1, "cartesian": 2, "sinhspherical": 3,
          "sinhcylindrical": 4}


def grid_desc(coord: str, n, order: int, *, amax: float = 1.0e4,
              bscale: float = 5.0, sinhwaa: float = 0.07, rmax: float = 64.0,
              xmax: float = 32.0, zmax: float = 1.0e4,
              sinhwz: float = 0.07) -> dict:
    return {"coord": coord, "n": tuple(int(v) for v in n), "order": int(order),
            "amax": float(amax), "bscale": float(bscale),
            "sinhwaa": float(sinhwaa), "rmax": float(rmax),
            "xmax": float(xmax), "zmax": float(zmax), "sinhwz": float(sinhwz)}


def _punc(m, x, P, chi=(0.0, 0.0, 0.0)):
    return {"m": float(m), "x": tuple(map(float, x)), "P": tuple(map(float, P)),
            "S": tuple(float(c) * m * m for c in chi)}


def equal_mass_pair() -> list[dict]:
    """Equal masses 0.5 at z = +-5, momenta +-0.1 along x, no spin."""
    return [_punc(0.5, (0, 0, 5), (0.1, 0, 0)),
            _punc(0.5, (0, 0, -5), (-0.1, 0, 0))]


def spinning_q4_pair() -> list[dict]:
    """Masses 0.8/0.2 at z = +-5 (separation 10), momenta +-0.09 along x,
    spins chi = (0.3, -0.2, 0.5) and (0, 0.4, -0.1)."""
    return [_punc(0.8, (0, 0, 5), (0.09, 0, 0), (0.3, -0.2, 0.5)),
            _punc(0.2, (0, 0, -5), (-0.09, 0, 0), (0.0, 0.4, -0.1))]


def brill_lindquist_pair() -> list[dict]:
    """Two punctures at rest without spin: the source vanishes."""
    return [_punc(0.5, (0, 0, 5), (0, 0, 0)), _punc(0.5, (0, 0, -5), (0, 0, 0))]


# Named workloads: the small equal-mass case, the q=4 spinning case and its
# larger and other-coordinate variants.
def small_equal_mass():
    """SinhSymTP 32x16x2, AMAX 1e4, bScale 5, SINHWAA 0.07, 4th-order FD."""
    return grid_desc("sinhsymtp", (32, 16, 2), 4), equal_mass_pair()


def q4_sinhsymtp_128():
    """SinhSymTP 128x128x16, 8th-order FD, the q=4 spinning pair."""
    return grid_desc("sinhsymtp", (128, 128, 16), 8), spinning_q4_pair()


def q4_sinhsymtp_256():
    return grid_desc("sinhsymtp", (256, 256, 32), 8), spinning_q4_pair()


def q4_spherical_128():
    return grid_desc("spherical", (128, 64, 32), 8, rmax=64.0), spinning_q4_pair()


def q4_sinhspherical_128():
    """SinhSpherical 128x64x16 (AMAX 1e4, SINHWAA 0.07), order 8."""
    return grid_desc("sinhspherical", (128, 64, 16), 8), spinning_q4_pair()


def q4_cartesian_256():
    return grid_desc("cartesian", (256, 256, 256), 8, xmax=32.0), spinning_q4_pair()


def padded_shape(desc: dict) -> tuple[int, int, int]:
    ng = desc["order"] // 2
    n0, n1, n2 = desc["n"]
    return (n2 + 2 * ng, n1 + 2 * ng, n0 + 2 * ng)


def smooth_random_field(desc: dict, seed: int, amplitude: float = 0.1,
                        modes: int = 4, noise: float = 0.0) -> np.ndarray:
    """A seeded smooth field over the padded index box, shape (s2, s1, s0).

    Sum of ``modes`` low-frequency products of cosines in the normalised index
    coordinates t_d = (i_d + 1/2)/s_d, plus optional white noise.  It knows
    nothing about the coordinate map; callers that need boundary-consistent
    ghosts fill them with their own code.
    """
    rng = np.random.default_rng(seed)
    s2, s1, s0 = padded_shape(desc)
    t0 = (np.arange(s0) + 0.5) / s0
    t1 = (np.arange(s1) + 0.5) / s1
    t2 = (np.arange(s2) + 0.5) / s2
    f = np.zeros((s2, s1, s0))
    for _ in range(modes):
        k = rng.integers(0, 4, size=3)
        ph = rng.uniform(0, 2 * np.pi, size=3)
        a = rng.uniform(-1.0, 1.0)
        f += a * (np.cos(np.pi * k[2] * t2 + ph[2])[:, None, None]
                  * np.cos(np.pi * k[1] * t1 + ph[1])[None, :, None]
                  * np.cos(np.pi * k[0] * t0 + ph[0])[None, None, :])
    f *= amplitude / max(1.0, np.abs(f).max())
    if noise > 0.0:
        f += noise * rng.standard_normal(f.shape)
    return f


def batch_parameters(count: int, seed: int) -> list[dict]:
    """Parameter sweep for many-solve batches (uniform random draws).

    q in [1,8], separation d in [6,16], |P| <= 0.15 along a random direction
    (+P on the heavier puncture, -P on the other), |chi| <= 0.8 per puncture in
    random directions, total bare mass 1.  Punctures sit on the z axis at
    +-d/2; the SinhSymTP focus is placed on them (bScale = d/2).  Grid sizes
    are drawn from N0 in {64,96,128}, N1 in {32,64,96,128}, N2 in {8,16}.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        q = rng.uniform(1.0, 8.0)
        d = rng.uniform(6.0, 16.0)
        pmag = rng.uniform(0.0, 0.15)
        pdir = rng.standard_normal(3)
        pdir /= np.linalg.norm(pdir)
        chis = []
        for _a in range(2):
            cmag = rng.uniform(0.0, 0.8)
            cdir = rng.standard_normal(3)
            cdir /= np.linalg.norm(cdir)
            chis.append(tuple(cmag * cdir))
        n = (int(rng.choice([64, 96, 128])), int(rng.choice([32, 64, 96, 128])),
             int(rng.choice([8, 16])))
        m1, m2 = q / (1.0 + q), 1.0 / (1.0 + q)
        P = tuple(pmag * pdir)
        punct = [_punc(m1, (0, 0, d / 2), P, chis[0]),
                 _punc(m2, (0, 0, -d / 2), tuple(-c for c in P), chis[1])]
        out.append({"q": q, "d": d, "P": P, "chi1": chis[0], "chi2": chis[1],
                    "n": n, "punctures": punct,
                    "desc": grid_desc("sinhsymtp", n, 8, bscale=d / 2)})
    return out


def mlp_dims(n_in: int = 12, hidden: int = 512, depth: int = 4,
             n_out: int = 64 * 32 * 8) -> list[int]:
    return [n_in] + [hidden] * depth + [n_out]


def mlp_init_params(dims, seed: int) -> np.ndarray:
    """Seeded initial parameters in the logical packed layout (per layer W
    [out][in] then b [out]): normal weights with variance 2/in on hidden
    layers and 1/in on the output layer, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (din, dout) in enumerate(zip(dims[:-1], dims[1:])):
        scale = np.sqrt((1.0 if l == len(dims) - 2 else 2.0) / din)
        parts.append((rng.standard_normal((dout, din)) * scale).ravel())
        parts.append(np.zeros(dout))
    return np.concatenate(parts).astype(np.float32)


def surrogate_inputs(params: list[dict]) -> np.ndarray:
    """The 12 network inputs of each parameter draw, scaled to [-1, 1]:
    q in [1,8], d in [6,16], P (|P| <= 0.15), chi1, chi2 (|chi| <= 0.8),
    total mass (1)."""
    rows = []
    for p in params:
        rows.append([(p["q"] - 4.5) / 3.5, (p["d"] - 11.0) / 5.0,
                     *(c / 0.15 for c in p["P"]), *(c / 0.8 for c in p["chi1"]),
                     *(c / 0.8 for c in p["chi2"]), 1.0])
    return np.asarray(rows, dtype=np.float32)


def minibatch_order(n: int, batch: int, steps: int, seed: int) -> np.ndarray:
    """Sample indices for `steps` minibatches: concatenated seeded
    permutations of range(n), cut into batches."""
    rng = np.random.default_rng(seed)
    need = steps * batch
    out = []
    while sum(len(o) for o in out) < need:
        out.append(rng.permutation(n))
    return np.concatenate(out)[:need].astype(np.int32)
