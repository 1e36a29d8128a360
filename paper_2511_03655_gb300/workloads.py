"""Seeded synthetic workloads (initial conditions, step sizes, step counts).

This module holds no arithmetic of the integration method: it only draws
inputs.  Both the oracle-based tests and the GPU path take their inputs from
here.  Random numbers come from splitmix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) mapped to doubles
in [0, 1) with 53 random bits, so every host produces the same inputs.

Workloads (sizes as in the benchmark configurations):
  kepler_single    one planar Kepler orbit, e = 0.5, q0 = (0.5, 0), v0 = (0, sqrt 3),
                   h = 2 pi/200, 20,000 steps (100 periods).
  kepler_ensemble  B = 65,536 planar orbits, a = 1, e ~ U[0, 0.9) from the seed,
                   periapsis start q0 = (1 - e, 0), v0 = (0, sqrt((1+e)/(1-e))),
                   m = round(200 + 100 e) steps per period, h = 2 pi/m, 100 periods.
  henon_heiles     the Sec. 5.1 initial condition (q = (0, 0.3), p2 = 0.2, H = 1/12).
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 2511036550
MASK64 = (1 << 64) - 1


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n successive outputs of splitmix64 started at `seed` (uint64 array)."""
    state = np.uint64(seed & MASK64)
    gamma = np.uint64(0x9E3779B97F4A7C15)
    idx = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = state + gamma * idx
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): the top 53 bits of splitmix64 outputs times 2^-53."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def kepler_ic(e):
    """Periapsis state of the a = 1, GM = 1 orbit of eccentricity e."""
    e = np.asarray(e, dtype=np.float64)
    q = np.stack([1.0 - e, np.zeros_like(e)], axis=-1)
    v = np.stack([np.zeros_like(e), np.sqrt((1.0 + e) / (1.0 - e))], axis=-1)
    return q, v


def kepler_single():
    q, v = kepler_ic(np.array([0.5]))
    return {"name": "kepler_single", "kind": "kepler", "params": [1.0], "dim": 2,
            "q0": q, "v0": v, "h": np.array([2 * math.pi / 200]),
            "nsteps": np.array([20000], dtype=np.int64), "e": np.array([0.5])}


def kepler_ensemble(batch: int = 65536, periods: int = 100, emax: float = 0.9, seed_id: int = 2):
    e = emax * uniform(SEED_BASE + seed_id, batch)
    m = np.rint(200.0 + 100.0 * e).astype(np.int64)
    h = 2 * math.pi / m.astype(np.float64)
    q, v = kepler_ic(e)
    return {"name": f"kepler_ensemble_B{batch}_P{periods}", "kind": "kepler", "params": [1.0],
            "dim": 2, "q0": q, "v0": v, "h": h, "nsteps": periods * m, "e": e,
            "steps_per_period": m}


def henon_heiles_ic():
    q1, q2, p2 = 0.0, 0.3, 0.2
    rest = p2 * p2 / 2 + (q1 * q1 + q2 * q2) / 2 + (q1 * q1 * q2 - q2 ** 3 / 3)
    p1 = math.sqrt(2 * (1.0 / 12 - rest))
    return np.array([[q1, q2]]), np.array([[p1, p2]])


def similarity_order(key: np.ndarray, descending: bool = True) -> np.ndarray:
    """Processing order that puts trajectories with similar `key` (e.g. the
    eccentricity, or an estimated cost) next to each other, costliest first."""
    o = np.argsort(key, kind="stable")
    return (o[::-1] if descending else o).astype(np.int32)
