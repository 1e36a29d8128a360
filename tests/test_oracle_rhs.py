"""Pins of the oracle's N-body and FPUT right-hand sides against facts that
do not come from the oracle itself.

N-body (Eq. Ham2 of Sec. 5.1: H = sum_a m_a |v_a|^2 / 2 - sum_{a<b} G m_a m_b / r_ab):
  * g_a = -(1/m_a) dH/dq_a, with the gradient taken by central differences of
    H in 60-digit arithmetic (N = 3 and 5, unequal masses, G != 1);
  * two bodies of unequal mass: the relative motion is the Kepler orbit with
    mu = G (m_1 + m_2), solved in closed form by Kepler's equation, and the
    barycentre stays at rest;
  * Lagrange's equilateral solution: three unequal masses at the corners of
    an equilateral triangle of side L rotate rigidly about the barycentre
    with omega^2 = G M / L^3 (M the total mass), here in a tilted plane so
    that all three coordinates take part.

FPUT alpha chain with fixed ends (q_0 = q_{n+1} = 0, V(r) = r^2/2 + alpha r^3/3):
  * g_j = -dH/dq_j by 60-digit central differences (n = 8, alpha = 0.25);
  * g equals the Fermi-Pasta-Ulam equation of motion written in its usual
    form, q_j'' = (q_{j+1} - 2 q_j + q_{j-1})
                 + alpha [(q_{j+1} - q_j)^2 - (q_j - q_{j-1})^2];
  * alpha = 0: the chain's normal modes are closed form, mode k with shape
    sin(j k pi/(n+1)) and frequency 2 sin(k pi / (2 (n+1)));
  * the energy error of a mode-1 run (n = 16, 1e4 steps) stays bounded with
    no linear drift.

The helpers take the right-hand side (or a runner) as an argument so that
``tests/test_oracle_mutations.py`` can check that planted mistakes fail them.
"""
import math
import random
from decimal import Decimal, localcontext

import numpy as np
import pytest

from oracle import cbind, coeffs
from oracle import irkgl as P
from tests.closed_forms import dec_pi, dec_sin_cos, kepler_state

TAB = coeffs.fp64_tables()


# ------------------------------------------------------------------ helpers
def grad_residual(rhs, q, v, mass, eps="1e-25"):
    """max_l |g_l + dH/dq_l / mass_l| / max_l |g_l| in 60 digits."""
    with localcontext() as ctx:
        ctx.prec = 60
        q = [Decimal(x) for x in q]
        v = [Decimal(x) for x in v]
        e = Decimal(eps)
        g = rhs.g(q)
        worst = Decimal(0)
        for l in range(len(q)):
            qp, qm = list(q), list(q)
            qp[l] += e
            qm[l] -= e
            dH = (rhs.H(qp, v) - rhs.H(qm, v)) / (2 * e)
            worst = max(worst, abs(g[l] + dH / Decimal(mass[l])))
        return float(worst / max(abs(x) for x in g))


def _rot(axis, ang):
    """Rotation matrix about the unit vector ``axis`` by ``ang`` (Rodrigues),
    as Decimals."""
    s, c = dec_sin_cos(ang)
    x, y, z = axis
    C = 1 - c
    return [[c + x * x * C, x * y * C - z * s, x * z * C + y * s],
            [y * x * C + z * s, c + y * y * C, y * z * C - x * s],
            [z * x * C - y * s, z * y * C + x * s, c + z * z * C]]


def _apply(M, r):
    return [M[0][0] * r[0] + M[0][1] * r[1] + M[0][2] * r[2],
            M[1][0] * r[0] + M[1][1] * r[1] + M[1][2] * r[2],
            M[2][0] * r[0] + M[2][1] * r[1] + M[2][2] * r[2]]


def _unit(v):
    n = (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]).sqrt()
    return [x / n for x in v]


def _cross(a, b):
    return [a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]]


def run_c(kind, params):
    """A runner (q0, v0, h, n) -> (q, v) through the C oracle, the form the
    GPU parity tests compare with."""
    def go(q0, v0, h, n):
        r = cbind.run(kind, params, q0, v0, h, n)
        assert r["status"][0] == 0
        return r["q"][0] + r["q_lo"][0], r["v"][0] + r["v_lo"][0]
    return go


def run_py(rhs):
    """The same through the Python oracle (used with planted mistakes)."""
    def go(q0, v0, h, n):
        p = P.integrate(q0, v0, h, n, TAB, rhs)
        assert p["status"] == P.OK
        st = p["state"]
        return (np.asarray(st.q) + np.asarray(st.q_lo), np.asarray(st.v) + np.asarray(st.v_lo))
    return go


# ------------------------------------------------------------------ N-body
LAGRANGE_G = "1.3"
LAGRANGE_M = ("1.0", "0.01", "0.001")   # 27 sum m_a m_b < M^2: the stable (Routh) case
TILT = ("0.3", "-0.2", "1")


def lagrange_triangle(side="1.7", G=LAGRANGE_G, masses=LAGRANGE_M, tilt=TILT):
    """Initial state and angular rate of Lagrange's equilateral solution:
    corners on the unit circle of the plane normal to ``tilt``, scaled to
    side L and shifted to the barycentre; v_a = omega n x r_a with
    omega^2 = G M / L^3.  Returns FP64 (q0, v0), omega, and the exact
    barycentric corners as Decimals."""
    with localcontext() as ctx:
        ctx.prec = 60
        G = Decimal(G)
        m = [Decimal(x) for x in masses]
        L = Decimal(side)
        n = _unit([Decimal(x) for x in tilt])
        # two orthonormal vectors spanning the plane
        e1 = _unit(_cross(n, [Decimal(1), Decimal(0), Decimal(0)]))
        e2 = _cross(n, e1)
        pi = dec_pi()
        R = L / Decimal(3).sqrt()
        pts = []
        for k in range(3):
            s, c = dec_sin_cos(2 * pi * k / 3 + Decimal("0.4"))
            pts.append([R * (c * e1[i] + s * e2[i]) for i in range(3)])
        M = sum(m)
        com = [sum(m[a] * pts[a][i] for a in range(3)) / M for i in range(3)]
        pts = [[p[i] - com[i] for i in range(3)] for p in pts]
        om = (G * M / L ** 3).sqrt()
        vel = [[om * x for x in _cross(n, p)] for p in pts]
        q0 = [float(x) for p in pts for x in p]
        v0 = [float(x) for p in vel for x in p]
        return q0, v0, om, n, pts


def lagrange_error(runner, periods="1", steps_per_period=200):
    """Relative state error of a run against the rigid rotation."""
    q0, v0, om, n, _ = lagrange_triangle()
    with localcontext() as ctx:
        ctx.prec = 60
        T = 2 * dec_pi() / om
        h = float(T / steps_per_period)
        nst = int(Decimal(periods) * steps_per_period)
        t = Decimal(h) * nst
        # rotate the FP64 initial state exactly (the solution from the rounded
        # start differs from the rigid one by roundoff only)
        Mr = _rot(n, om * t)
        qe, ve = [], []
        for a in range(3):
            qe += _apply(Mr, [Decimal(x) for x in q0[3 * a:3 * a + 3]])
            ve += _apply(Mr, [Decimal(x) for x in v0[3 * a:3 * a + 3]])
        qe = np.array([float(x) for x in qe])
        ve = np.array([float(x) for x in ve])
    q, v = runner(q0, v0, h, nst)
    return max(np.abs(q - qe).max() / np.abs(qe).max(), np.abs(v - ve).max() / np.abs(ve).max())


TWO_BODY_G, TWO_BODY_M, TWO_BODY_E = "1.3", ("1.0", "0.3"), "0.5"


def two_body_state(t, G=TWO_BODY_G, masses=TWO_BODY_M, e=TWO_BODY_E):
    """Barycentric state of two bodies whose relative orbit is the Kepler
    ellipse a = 1, eccentricity e, mu = G (m_1 + m_2), periapsis at t = 0,
    in a tilted plane.  Returns (q, v) as Decimals (6 components each)."""
    with localcontext() as ctx:
        ctx.prec = 60
        G = Decimal(G)
        m1, m2 = (Decimal(x) for x in masses)
        M = m1 + m2
        rq, rv = kepler_state(Decimal(e), t, mu=G * M)
        Mr = _rot(_unit([Decimal(x) for x in TILT]), Decimal("0.7"))
        r = _apply(Mr, [rq[0], rq[1], Decimal(0)])
        w = _apply(Mr, [rv[0], rv[1], Decimal(0)])
        q = [-m2 / M * x for x in r] + [m1 / M * x for x in r]
        v = [-m2 / M * x for x in w] + [m1 / M * x for x in w]
        return q, v


def two_body_error(runner, periods="1", steps_per_period=200):
    with localcontext() as ctx:
        ctx.prec = 60
        mu = Decimal(TWO_BODY_G) * sum(Decimal(x) for x in TWO_BODY_M)
        T = 2 * dec_pi() / mu.sqrt()
        h = float(T / steps_per_period)
        nst = int(Decimal(periods) * steps_per_period)
        q0, v0 = two_body_state(Decimal(0))
        q0 = [float(x) for x in q0]
        v0 = [float(x) for x in v0]
        qe, ve = two_body_state(Decimal(h) * nst)
        qe = np.array([float(x) for x in qe])
        ve = np.array([float(x) for x in ve])
    q, v = runner(q0, v0, h, nst)
    return max(np.abs(q - qe).max() / np.abs(qe).max(), np.abs(v - ve).max() / np.abs(ve).max())


def nbody_random_state(nb, seed):
    rnd = random.Random(seed)
    q = [rnd.uniform(-3, 3) for _ in range(3 * nb)]
    v = [rnd.uniform(-1, 1) for _ in range(3 * nb)]
    m = [10 ** rnd.uniform(-3, 0) for _ in range(nb)]
    return q, v, m


@pytest.mark.parametrize("nb,seed", [(3, 1), (5, 2)])
def test_nbody_g_is_minus_grad_H_over_m(nb, seed):
    q, v, m = nbody_random_state(nb, seed)
    with localcontext() as ctx:
        ctx.prec = 60
        rhs = P.NBody([Decimal(x) for x in m], G=Decimal("1.3"))
    assert grad_residual(rhs, q, v, [m[a] for a in range(nb) for _ in range(3)]) < 1e-30


def test_nbody_two_body_is_kepler():
    """Two unequal bodies: one period of the relative Kepler orbit (mu =
    G (m_1 + m_2)) at h = T/200, 1e-12 of the state (the method's
    truncation error is far below roundoff at this step)."""
    params = [float(TWO_BODY_G)] + [float(x) for x in TWO_BODY_M]
    assert two_body_error(run_c(cbind.NBODY, params), periods="2") <= 1e-12


def test_nbody_lagrange_equilateral_rotates_rigidly():
    params = [float(LAGRANGE_G)] + [float(x) for x in LAGRANGE_M]
    assert lagrange_error(run_c(cbind.NBODY, params), periods="2") <= 1e-12


def test_nbody_python_form_passes_the_same_pins():
    """The Python form (the one the mutation tests plant mistakes in) passes
    the closed-form pins too, over a quarter period."""
    rhs3 = P.NBody([float(x) for x in LAGRANGE_M], G=float(LAGRANGE_G))
    assert lagrange_error(run_py(rhs3), periods="0.25", steps_per_period=100) <= 1e-12
    rhs2 = P.NBody([float(x) for x in TWO_BODY_M], G=float(TWO_BODY_G))
    assert two_body_error(run_py(rhs2), periods="0.25", steps_per_period=100) <= 1e-12


def test_nbody_momentum_conserved():
    """Newton's third law: sum_a m_a g_a = 0, so total momentum is constant
    (to roundoff) along a 6-body run of the oracle."""
    q, v, m = nbody_random_state(6, 9)
    for a in range(6):
        q[3 * a:3 * a + 3] = [x * (a + 2) for x in q[3 * a:3 * a + 3]]   # keep bodies apart
    params = [1.0] + m
    p0 = np.array([sum(m[a] * v[3 * a + k] for a in range(6)) for k in range(3)])
    r = cbind.run(cbind.NBODY, params, q, v, 0.01, 200)
    vv = r["v"][0] + r["v_lo"][0]
    p1 = np.array([sum(m[a] * vv[3 * a + k] for a in range(6)) for k in range(3)])
    scale = sum(m[a] * np.abs(vv[3 * a:3 * a + 3]).max() for a in range(6))
    assert np.abs(p1 - p0).max() <= 1e-14 * scale


# ------------------------------------------------------------------ FPUT
def fput_random_state(n, seed):
    rnd = random.Random(seed)
    return [rnd.uniform(-0.5, 0.5) for _ in range(n)], [rnd.uniform(-0.5, 0.5) for _ in range(n)]


def fpu_equation_residual(rhs, n, alpha, seed=3):
    """max |g - (second difference + alpha (difference of squared bonds))|
    in 60 digits, with q_0 = q_{n+1} = 0."""
    q, _ = fput_random_state(n, seed)
    with localcontext() as ctx:
        ctx.prec = 60
        a = Decimal(alpha)
        qd = [Decimal(x) for x in q]
        ext = [Decimal(0)] + qd + [Decimal(0)]
        g = rhs.g(qd)
        worst = Decimal(0)
        for j in range(1, n + 1):
            fpu = (ext[j + 1] - 2 * ext[j] + ext[j - 1]) + \
                a * ((ext[j + 1] - ext[j]) ** 2 - (ext[j] - ext[j - 1]) ** 2)
            worst = max(worst, abs(g[j - 1] - fpu))
        return float(worst)


def normal_mode_error(runner, n=8, h=0.5, nsteps=400, seed=11):
    """alpha = 0: the run against the closed-form normal-mode solution
    q_j(t) = sum_k s_jk (a_k cos w_k t + b_k sin(w_k t)/w_k),
    s_jk = sin(j k pi/(n+1)), w_k = 2 sin(k pi/(2(n+1)))."""
    rnd = random.Random(seed)
    amp = [rnd.uniform(-0.3, 0.3) for _ in range(n)]
    vel = [rnd.uniform(-0.3, 0.3) for _ in range(n)]
    with localcontext() as ctx:
        ctx.prec = 60
        pi = dec_pi()
        S = [[dec_sin_cos(Decimal(j * k) * pi / (n + 1))[0] for k in range(1, n + 1)]
             for j in range(1, n + 1)]
        w = [2 * dec_sin_cos(Decimal(k) * pi / (2 * (n + 1)))[0] for k in range(1, n + 1)]
        q0 = [float(sum(S[j][k] * Decimal(amp[k]) for k in range(n))) for j in range(n)]
        v0 = [float(sum(S[j][k] * Decimal(vel[k]) for k in range(n))) for j in range(n)]
        # modal coordinates of the rounded start: S is symmetric and
        # S S = (n+1)/2 I
        a = [sum(S[k][j] * Decimal(q0[j]) for j in range(n)) * 2 / (n + 1) for k in range(n)]
        b = [sum(S[k][j] * Decimal(v0[j]) for j in range(n)) * 2 / (n + 1) for k in range(n)]
        t = Decimal(h) * nsteps
        qe, ve = [], []
        for j in range(n):
            sq, sv = Decimal(0), Decimal(0)
            for k in range(n):
                s, c = dec_sin_cos(w[k] * t)
                sq += S[j][k] * (a[k] * c + b[k] * s / w[k])
                sv += S[j][k] * (-a[k] * w[k] * s + b[k] * c)
            qe.append(float(sq))
            ve.append(float(sv))
    q, v = runner(q0, v0, h, nsteps)
    qe, ve = np.array(qe), np.array(ve)
    return max(np.abs(q - qe).max() / np.abs(qe).max(), np.abs(v - ve).max() / np.abs(ve).max())


@pytest.mark.parametrize("n", [8, 5])
def test_fput_g_is_minus_grad_H(n):
    q, v = fput_random_state(n, n)
    with localcontext() as ctx:
        ctx.prec = 60
        rhs = P.FPUT(n, Decimal("0.25"))
    assert grad_residual(rhs, q, v, [1.0] * n) < 1e-30


@pytest.mark.parametrize("n", [8, 1, 2])
def test_fput_g_is_the_fpu_equation_of_motion(n):
    with localcontext() as ctx:
        ctx.prec = 60
        rhs = P.FPUT(n, Decimal("0.25"))
    assert fpu_equation_residual(rhs, n, "0.25") < 1e-55


def test_fput_linear_chain_normal_modes():
    """alpha = 0, n = 8, h = 0.5, 400 steps: every one of the 8 modes
    excited; the run matches the closed form to 1e-12 of the state."""
    assert normal_mode_error(run_c(cbind.FPUT, [0.0])) <= 1e-12
    assert normal_mode_error(run_py(P.FPUT(8, 0.0)), nsteps=40) <= 1e-12


def test_fput_energy_bounded_no_drift():
    """n = 16, alpha = 0.25, unit harmonic energy in mode 1, h = 0.5,
    1e4 steps: the energy error stays at roundoff, below the 1e-13 that
    qualifies a run, and a linear fit over the run shows a drift below a
    tenth of one rounding unit per step."""
    n, h, N, chunks = 16, 0.5, 10000, 100
    w1 = 2 * math.sin(math.pi / (2 * (n + 1)))
    A = 2 / (w1 * math.sqrt(n + 1))
    q0 = [A * math.sin((j + 1) * math.pi / (n + 1)) for j in range(n)]
    v0 = [0.0] * n
    # unit harmonic energy: the quadratic part of H is 1
    assert abs(cbind.hamiltonian(cbind.FPUT, [0.0], q0, v0) - 1.0) < 1e-14
    H0 = cbind.hamiltonian(cbind.FPUT, [0.25], q0, v0)
    st = dict(q=q0, v=v0, q_lo=None, v_lo=None, r_prev=None)
    ts, dHs = [], []
    for c in range(chunks):
        r = cbind.run(cbind.FPUT, [0.25], st["q"], st["v"], h, N // chunks,
                      q_lo=st["q_lo"], v_lo=st["v_lo"], r_prev=st["r_prev"])
        assert r["status"][0] == 0
        st = dict(q=r["q"][0], v=r["v"][0], q_lo=r["q_lo"][0], v_lo=r["v_lo"][0], r_prev=r["r_prev"][0])
        ts.append((c + 1) * (N // chunks) * h)
        dHs.append((cbind.hamiltonian(cbind.FPUT, [0.25], st["q"], st["v"]) - H0) / H0)
    assert max(abs(x) for x in dHs) <= 1e-13
    slope = np.polyfit(ts, dHs, 1)[0]
    assert abs(slope * ts[-1]) <= 0.1 * N * 2.0 ** -53, slope * ts[-1]
