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
                   h = 0.5 % of the innermost period, 1e5 steps; masses and axes are
                   redrawn until neighbours are >= 8 mutual Hill radii apart, as in
                   the outer Solar System.  (A synthetic stand-in for the paper's
                   6-body outer Solar System, whose DE430 initial conditions are not
                   available here.)
  fput_chain       FPUT alpha chain, n interior particles, fixed ends, alpha = 0.25,
                   unit harmonic energy in mode 1: q_j = A sin(j pi/(n+1)),
                   A = 2/(omega_1 sqrt(n+1)), omega_1 = 2 sin(pi/(2(n+1))), v = 0.
  uneven_batch     4,096 instances, half N-body (N ~ U{3..64}: central mass + N-1
                   bodies as in nbody_ensemble, one system per instance) and half
                   FPUT (n ~ U{8..512}); per-instance h from a step table.
  serving_requests Poisson arrivals (rate lambda); each request takes one family of
                   the workloads above (Kepler orbits, 6-body copies, N-body with
                   N ~ U{7..nb_max}, FPUT with n ~ U{8..n_max}), a batch ~ logU[1, B_max]
                   and a horizon ~ logU[1e2, T_max] steps.
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


def henon_heiles_ensemble(batch: int, energy: float = 1.0 / 12, seed_id: int = 7,
                          t_max: float = 2 * math.pi):
    """`batch` Henon-Heiles initial states on the energy surface H = energy
    (the paper's H = 1/12 by default, Sec. 5.1): q1 = 0, (q2, p2) drawn
    uniformly from the box [-0.35, 0.45] x [-0.3, 0.3] and kept where the
    remaining energy leaves p1^2 > 0; p1 = +sqrt(2 (energy - rest)).  Also a
    start time t0 ~ U[0, t_max) per state, for the non-autonomous system
    of Sec. 3 (forcing lambda + xi sin t).  Returns (q0, v0, t0)."""
    q, v = [], []
    u = uniform(SEED_BASE + seed_id, 4 * batch + 64)
    k = 0
    while len(q) < batch:
        if k + 2 > len(u):
            u = np.concatenate([u, uniform(SEED_BASE + seed_id + 7919 * (k + 1), 4 * batch + 64)])
        q2 = -0.35 + 0.8 * u[k]
        p2 = -0.3 + 0.6 * u[k + 1]
        k += 2
        rest = p2 * p2 / 2 + q2 * q2 / 2 - q2 ** 3 / 3
        if energy - rest > 1e-3:
            q.append([0.0, q2])
            v.append([math.sqrt(2 * (energy - rest)), p2])
    t0 = t_max * uniform(SEED_BASE + seed_id + 1, batch)
    return np.array(q), np.array(v), t0


SBH_PARAMS = (0.995, 4.6, 8.9e-4)  # E, L, beta of Sec. 5.1


def schwarzschild_ensemble(batch: int, r_lo: float = 9.5, r_hi: float = 16.0, seed_id: int = 8,
                           params=SBH_PARAMS):
    """`batch` initial states of the Schwarzschild black-hole system of
    Sec. 5.1 (Eq. Ham_SBH), y = (r, theta, p_r, p_theta): r0 ~ U[r_lo, r_hi),
    theta = pi/2, p_r = 0 and p_theta > 0 from the energy condition H = -1/2
    (the paper's single orbit is r0 = 11).  Returns y0 [batch, 4]."""
    E, L, beta = params
    r = r_lo + (r_hi - r_lo) * uniform(SEED_BASE + seed_id, batch)
    u = 1.0 - 2.0 / r
    a = L - 0.5 * beta * r * r
    p2 = 2.0 * r * r * (-0.5 + E * E / (2.0 * u) - a * a / (2.0 * r * r))
    if np.any(p2 <= 0):
        raise ValueError("r range admits no p_theta with H = -1/2")
    return np.stack([r, np.full(batch, math.pi / 2), np.zeros(batch), np.sqrt(p2)], axis=1)


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


def _min_hill_separation(a, m) -> float:
    """Smallest gap between neighbouring semi-major axes, in mutual Hill
    radii ((m_i + m_j)/3)^(1/3) (a_i + a_j)/2 (central mass 1)."""
    o = np.argsort(a)
    gaps = [(a[y] - a[x]) / (((m[x] + m[y]) / 3.0) ** (1.0 / 3.0) * (a[x] + a[y]) / 2.0)
            for x, y in zip(o[:-1], o[1:])]
    return min(gaps) if gaps else math.inf


def nbody_system(nbodies: int = 6, seed_id: int = 3, amin: float = 5.0, amax: float = 40.0,
                 min_hill: float | None = None):
    """One planetary system: central mass 1 plus nbodies - 1 bodies (G = 1),
    barycentric positions q and velocities v (flattened [3 * nbodies]).
    With min_hill, masses and semi-major axes are redrawn (from the next
    seed stream) until neighbouring orbits are at least min_hill mutual Hill
    radii apart, as the planets of the outer Solar System are (8 or more)."""
    k = nbodies - 1
    for attempt in range(1000):
        u = uniform(SEED_BASE + seed_id + 7919 * attempt, 7 * k).reshape(7, k)
        m = 10.0 ** (-5.0 + 2.0 * u[0])
        a = np.exp(np.log(amin) + (np.log(amax) - np.log(amin)) * u[1])
        if min_hill is None or _min_hill_separation(a, m) >= min_hill:
            break
    else:
        raise ValueError(f"no {nbodies}-body system with {min_hill} mutual Hill radii spacing in [{amin}, {amax}]")
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
                   perturb: float = 1e-8, h_fraction: float = 0.005, min_hill: float | str | None = "auto"):
    """Perturbed copies of one planetary system.  min_hill = "auto" spaces
    systems of up to 6 bodies (the outer Solar System stand-in) >= 8 mutual
    Hill radii apart; larger systems rarely fit that spacing in [5, 40] and
    are drawn unspaced."""
    if min_hill == "auto":
        min_hill = 8.0 if nbodies <= 6 else None
    sysd = nbody_system(nbodies, seed_id, min_hill=min_hill)
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


def fput_chain(n: int, alpha: float = 0.25):
    """Mode-1 initial condition of the FPUT alpha chain with unit harmonic energy."""
    j = np.arange(1, n + 1, dtype=np.float64)
    w1 = 2.0 * math.sin(math.pi / (2.0 * (n + 1)))
    A = 2.0 / (w1 * math.sqrt(n + 1.0))
    return {"q": A * np.sin(j * math.pi / (n + 1)), "v": np.zeros(n), "params": [alpha],
            "omega_max": 2.0 * math.sin(n * math.pi / (2.0 * (n + 1)))}


# Default step table (kind, size bucket) -> h rule.  N-body: a fraction of the
# innermost period; FPUT: an absolute step.  The autotuner
# (paper_2511_03655_gb300.autotune) refines these by pilot runs.
DEFAULT_STEP_TABLE = {
    "nbody": {"fraction_of_inner_period": 0.005},
    "fput": {"h": 0.25},
}


def uneven_batch(ninst: int = 4096, steps: int = 10000, seed_id: int = 4, nmax_body: int = 64,
                 nmax_chain: int = 512, step_table: dict | None = None):
    """Ragged batch: instance list (kind, dim, offset, param_offset, nparams, h, nsteps)
    plus packed q0, v0 and parameters."""
    table = step_table or DEFAULT_STEP_TABLE
    u = uniform(SEED_BASE + seed_id, 2 * ninst).reshape(2, ninst)
    kinds, dims, hs, params, qs, vs = [], [], [], [], [], []
    for k in range(ninst):
        if k % 2 == 0:
            nb = 3 + int(u[0, k] * (nmax_body - 2))
            sysd = nbody_system(nb, seed_id=10000 + k)
            h = _nbody_fraction(table, nb) * sysd["period_inner"]
            kinds.append(2)
            dims.append(3 * nb)
            params.append([1.0] + list(sysd["masses"]))
            qs.append(sysd["q"])
            vs.append(sysd["v"])
        else:
            n = 8 + int(u[1, k] * (nmax_chain - 7))
            c = fput_chain(n)
            fput_h = table["fput"]
            h = fput_h["h"] if "h" in fput_h else fput_h["by_bucket"][_bucket(n)]
            kinds.append(3)
            dims.append(n)
            params.append(c["params"])
            qs.append(c["q"])
            vs.append(c["v"])
        hs.append(h)
    offsets = np.concatenate([[0], np.cumsum(dims)[:-1]]).astype(np.int64)
    pcount = np.array([len(p) for p in params])
    poffsets = np.concatenate([[0], np.cumsum(pcount)[:-1]]).astype(np.int64)
    return {"name": f"uneven_batch_{ninst}", "kind": np.array(kinds, dtype=np.int32),
            "dim": np.array(dims, dtype=np.int32), "offset": offsets,
            "param_offset": poffsets.astype(np.int32), "nparams": pcount.astype(np.int32),
            "h": np.array(hs), "nsteps": np.full(ninst, steps, dtype=np.int64),
            "params": np.concatenate([np.asarray(p, dtype=np.float64) for p in params]),
            "q0": np.concatenate(qs), "v0": np.concatenate(vs)}


def _nbody_fraction(table: dict, nb: int) -> float:
    """Step as a fraction of the innermost period: a number, or a table by
    body count (the entry for the smallest tabulated count >= nb, else the
    largest count)."""
    f = table["nbody"]["fraction_of_inner_period"]
    if not isinstance(f, dict):
        return float(f)
    keys = sorted(int(k) for k in f)
    for k in keys:
        if k >= nb:
            return float(f[str(k)])
    return float(f[str(keys[-1])])


def _bucket(n: int) -> str:
    for lim in (16, 32, 64, 128, 256, 512, 1024, 1536):
        if n <= lim:
            return str(lim)
    return "inf"


def _logu(u, lo, hi):
    return math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u)


def serving_requests(n: int = 200, rate: float = 2000.0, seed_id: int = 5, batch_max: int = 4096,
                     horizon_max: int = 100000, nb_max: int = 64, n_max: int = 1536,
                     families=("kepler", "nbody6", "nbody", "fput")):
    """Request descriptions for the serving loop (dicts; see serve.Request).

    Poisson arrivals at `rate`; each request picks a family of the Kepler
    ensemble, the 6-body ensemble, the ragged batch's N-body systems (N in
    {3..nb_max}) or its FPUT chains (n in {8..n_max}), with batch ~
    logU[1, batch_max] and horizon ~ logU[1e2, horizon_max] steps.  The
    defaults are the full ranges (D = 2d up to 3072)."""
    u = uniform(SEED_BASE + seed_id, 8 * n).reshape(n, 8)
    t = np.cumsum(-np.log(1.0 - u[:, 0]) / rate)  # exponential inter-arrival times
    out = []
    for k in range(n):
        fam = families[int(u[k, 1] * len(families)) % len(families)]
        B = max(1, int(round(_logu(u[k, 2], 1, batch_max))))
        T = int(round(_logu(u[k, 3], 100, horizon_max)))
        sid = 20000 + k
        if fam == "kepler":
            e = 0.9 * uniform(SEED_BASE + sid, B)
            q, v = kepler_ic(e)
            m = np.rint(200.0 + 100.0 * e)
            h = 2 * math.pi / m
            req = dict(kind="kepler", params=[1.0], dim=2, q0=q, v0=v, h=h, nsteps=T)
        elif fam == "nbody6":
            w = nbody_ensemble(copies=B, steps=T, seed_id=sid)
            req = dict(kind="nbody", params=w["params"], dim=18, q0=w["q0"], v0=w["v0"],
                       h=float(w["h"][0]), nsteps=T)
        elif fam == "nbody":
            nb = 3 + int(u[k, 4] * (nb_max - 2))
            w = nbody_ensemble(copies=B, nbodies=nb, steps=T, seed_id=sid)
            req = dict(kind="nbody", params=w["params"], dim=3 * nb, q0=w["q0"], v0=w["v0"],
                       h=float(w["h"][0]), nsteps=T)
        else:
            nn = 8 + int(u[k, 5] * (n_max - 7))
            c = fput_chain(nn)
            q = np.repeat(c["q"][None, :], B, axis=0) * (1.0 + 1e-8 * (2 * uniform(SEED_BASE + sid, B * nn).reshape(B, nn) - 1))
            req = dict(kind="fput", params=c["params"], dim=nn, q0=q, v0=np.zeros((B, nn)),
                       h=DEFAULT_STEP_TABLE["fput"]["h"], nsteps=T)
        req["arrival"] = float(t[k])
        req["rid"] = k
        out.append(req)
    return out


def config4_requests(ninst: int = 4096, rate: float = 2000.0, steps: int = 10000, seed_id: int = 4,
                     step_table: dict | None = None, arrival_seed_id: int = 6):
    """The ragged batch's instances as serving requests: each N-body system
    or FPUT chain of ``uneven_batch`` (same seed, sizes and step table) is
    one request of batch 1, arriving by a Poisson process at `rate`."""
    w = uneven_batch(ninst=ninst, steps=steps, seed_id=seed_id, step_table=step_table)
    u = uniform(SEED_BASE + arrival_seed_id, ninst)
    t = np.cumsum(-np.log(1.0 - u) / rate)
    out = []
    for k in range(ninst):
        o, d = int(w["offset"][k]), int(w["dim"][k])
        po, pn = int(w["param_offset"][k]), int(w["nparams"][k])
        kind = {2: "nbody", 3: "fput", 5: "harmonic"}[int(w["kind"][k])]
        out.append(dict(rid=k, kind=kind, params=list(w["params"][po:po + pn]), dim=d,
                        q0=w["q0"][o:o + d][None, :].copy(), v0=w["v0"][o:o + d][None, :].copy(),
                        h=float(w["h"][k]), nsteps=int(w["nsteps"][k]), arrival=float(t[k])))
    return out
