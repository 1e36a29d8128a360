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
  nbody_ensemble   a central mass 1 plus 5 bodies, masses log-uniform in [1e-5, 1e-3],
                   semi-major axes log-uniform in [5, 40], e ~ U[0, 0.05],
                   inclination ~ U[0, 2 deg], node / periapsis / mean anomaly ~ U[0, 2 pi),
                   G = 1; heliocentric elements with GM = 1 + m_i, shifted to the
                   barycentre at rest; 16,384 copies, copy 0 exact and the others with
                   positions scaled by (1 + 1e-8 xi), xi ~ U[-1, 1] per component;
                   h = 0.5 % of the innermost period, 1e5 steps.  (A synthetic
                   stand-in for the paper's 6-body outer Solar System, whose DE430
                   initial conditions are not available here.)
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


def _kepler_elements_to_state(a, e, inc, node, peri, M, mu):
    """Position and velocity of a two-body orbit from its elements
    (Kepler's equation solved by Newton's method)."""
    E = M.copy()
    for _ in range(60):
        E = E - (E - e * np.sin(E) - M) / (1.0 - e * np.cos(E))
    cE, sE = np.cos(E), np.sin(E)
    b = a * np.sqrt(1.0 - e * e)
    x, y = a * (cE - e), b * sE
    n = np.sqrt(mu / a ** 3)
    Edot = n / (1.0 - e * cE)
    vx, vy = -a * sE * Edot, b * cE * Edot
    # rotate: R_z(node) R_x(inc) R_z(peri)
    cw, sw, ci, si, cO, sO = np.cos(peri), np.sin(peri), np.cos(inc), np.sin(inc), np.cos(node), np.sin(node)
    r11, r12 = cO * cw - sO * sw * ci, -cO * sw - sO * cw * ci
    r21, r22 = sO * cw + cO * sw * ci, -sO * sw + cO * cw * ci
    r31, r32 = sw * si, cw * si
    pos = np.stack([r11 * x + r12 * y, r21 * x + r22 * y, r31 * x + r32 * y], axis=-1)
    vel = np.stack([r11 * vx + r12 * vy, r21 * vx + r22 * vy, r31 * vx + r32 * vy], axis=-1)
    return pos, vel


def nbody_system(nbodies: int = 6, seed_id: int = 3, amin: float = 5.0, amax: float = 40.0):
    """One planetary system: central mass 1 plus nbodies - 1 bodies (G = 1),
    barycentric positions q and velocities v (flattened [3 * nbodies])."""
    k = nbodies - 1
    u = uniform(SEED_BASE + seed_id, 7 * k).reshape(7, k)
    m = 10.0 ** (-5.0 + 2.0 * u[0])
    a = np.exp(np.log(amin) + (np.log(amax) - np.log(amin)) * u[1])
    e = 0.05 * u[2]
    inc = np.deg2rad(2.0) * u[3]
    node, peri, M = 2 * math.pi * u[4], 2 * math.pi * u[5], 2 * math.pi * u[6]
    pos, vel = _kepler_elements_to_state(a, e, inc, node, peri, M, 1.0 + m)
    masses = np.concatenate([[1.0], m])
    q = np.concatenate([np.zeros((1, 3)), pos])
    v = np.concatenate([np.zeros((1, 3)), vel])
    msum = masses.sum()
    q -= (masses[:, None] * q).sum(0) / msum
    v -= (masses[:, None] * v).sum(0) / msum
    inner = int(np.argmin(a))
    period = 2 * math.pi * math.sqrt(a[inner] ** 3 / (1.0 + m[inner]))
    return {"masses": masses, "q": q.reshape(-1), "v": v.reshape(-1), "a": a, "period_inner": period}


def nbody_ensemble(copies: int = 16384, nbodies: int = 6, steps: int = 100000, seed_id: int = 3,
                   perturb: float = 1e-8, h_fraction: float = 0.005):
    sysd = nbody_system(nbodies, seed_id)
    d = 3 * nbodies
    xi = 2.0 * uniform(SEED_BASE + seed_id + 500, copies * d).reshape(copies, d) - 1.0
    xi[0] = 0.0
    q0 = sysd["q"][None, :] * (1.0 + perturb * xi)
    v0 = np.repeat(sysd["v"][None, :], copies, axis=0)
    h = h_fraction * sysd["period_inner"]
    return {"name": f"nbody{nbodies}_ensemble_C{copies}", "kind": "nbody",
            "params": [1.0] + list(sysd["masses"]), "dim": d, "q0": q0, "v0": v0,
            "h": np.full(copies, h), "nsteps": np.full(copies, steps, dtype=np.int64),
            "masses": sysd["masses"]}
