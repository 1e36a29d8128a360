"""Pins of the oracle's step (arXiv 2511.03655, Eqs. IRK_init2, IRK_FP2,
Delta_n, stopping, qnvn2) against closed forms, brute force and invariants.

  * C form == Python form, bit for bit (same operation sequence);
  * one step on q'' = -w^2 q equals the [8/8] Pade approximant of exp(hA),
    the stability function of the 8-stage Gauss method (closed form);
  * one step equals the IRKN collocation solution of Eq. Qi solved by brute
    force in 60 digits with the exact coefficients (Kepler, Henon-Heiles, N-body);
  * order 16 against the closed-form Kepler solution (Kepler's equation), in
    60-digit arithmetic where the asymptotic regime is visible;
  * the extrapolated initial guess (Eq. Pol0) is O(h^10) after the first step;
  * 100 Kepler periods at h = T/200 against the closed form;
  * symmetry (step +h then -h), symplecticity M^T J M = J via Dual numbers;
  * bounded energy error without linear drift (Henon-Heiles, Sec. 5.1);
  * the stopping rule against its literal definition on random sequences;
  * status codes (iteration cap, non-finite stage values).
"""
import math
import os
import random
from decimal import Decimal, localcontext

import numpy as np
import pytest

from oracle import cbind, coeffs
from oracle import irkgl as P
from tests.closed_forms import dec_pi, kepler_state, pade_88_harmonic

TAB = coeffs.fp64_tables()
GOLD = os.path.join(os.path.dirname(__file__), "golden")


def hh_ic():
    with open(os.path.join(GOLD, "henon_heiles_ic.txt")) as f:
        vals = [float.fromhex(x) for x in f.read().splitlines()[-1].split()]
    return vals[:2], vals[2:]


def kepler_ic(e):
    return [1.0 - e, 0.0], [0.0, math.sqrt((1.0 + e) / (1.0 - e))]


# ---------------------------------------------------------------- C == Python
@pytest.mark.parametrize("kind,params,rhs,q0,v0,h", [
    (cbind.KEPLER, [1.0], P.Kepler(1.0), *kepler_ic(0.7), 2 * math.pi / 150),
    (cbind.HENON_HEILES, [1.0], P.HenonHeiles(1.0), *hh_ic(), 0.7),
    (cbind.HARMONIC, [1.3], P.Harmonic(1.3, 3), [1.0, -0.5, 0.25], [0.0, 0.3, -0.2], 0.4),
    (cbind.NBODY, [1.0, 1.0, 1e-3, 3e-4], P.NBody([1.0, 1e-3, 3e-4]),
     [0.0, 0.0, 0.0, 5.0, 0.0, 0.1, 0.0, 9.0, -0.2], [0.0, 0.0, 0.0, 0.0, 0.447, 0.0, -0.333, 0.0, 0.01],
     0.3),
    (cbind.FPUT, [0.25], P.FPUT(8, 0.25), [0.1 * math.sin(math.pi * (j + 1) / 9) for j in range(8)],
     [0.0] * 8, 0.5),
])
def test_c_equals_python_bitwise(kind, params, rhs, q0, v0, h):
    n = 25
    r = cbind.run(kind, params, q0, v0, h, n, iters_len=n)
    p = P.integrate(q0, v0, h, n, TAB, rhs)
    st = p["state"]
    assert list(r["iters"][0]) == p["iters"]
    for a, b in ((r["q"][0], st.q), (r["v"][0], st.v), (r["q_lo"][0], st.q_lo), (r["v_lo"][0], st.v_lo)):
        assert np.array_equal(np.asarray(a), np.asarray(b, dtype=np.float64))
    assert np.array_equal(r["r_prev"][0], np.asarray(st.r_prev))
    assert r["dH_max"][0] == p["dH_max"]


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("wh", [0.1, 0.5, 1.0])
def test_harmonic_step_is_pade_88(wh):
    q0, v0 = 1.0, 0.3
    R = pade_88_harmonic(1, Decimal(wh))
    r = cbind.run(cbind.HARMONIC, [1.0], [q0], [v0], wh, 1)
    with localcontext() as ctx:
        ctx.prec = 60
        eq = float(R[0][0] * Decimal(q0) + R[0][1] * Decimal(v0))
        ev = float(R[1][0] * Decimal(q0) + R[1][1] * Decimal(v0))
    assert abs(r["q"][0][0] - eq) <= 3e-16
    assert abs(r["v"][0][0] - ev) <= 3e-16
    # |R(i w h)| = 1: the quadratic invariant is kept to roundoff
    H0 = (v0 * v0 + q0 * q0) / 2
    H1 = (r["v"][0][0] ** 2 + r["q"][0][0] ** 2) / 2
    assert abs(H1 - H0) / H0 <= 4e-16


def _collocation_brute_force(rhs, q, v, h, ex, prec=60):
    """Solve Eq. Qi, Q_i = q + h c_i v + h^2 sum_j alpha_ij g(Q_j), by plain
    fixed-point iteration with the exact coefficients to 1e-50, then
    Eq. qnvn: q1 = q + h v + h^2 sum beta_i g_i, v1 = v + h sum b_i g_i."""
    with localcontext() as ctx:
        ctx.prec = prec
        d = len(q)
        q = [Decimal(x) for x in q]
        v = [Decimal(x) for x in v]
        h = Decimal(h)
        c, b, al, be = ex["c"], ex["b"], ex["alpha"], ex["beta"]
        Q = [[q[l] + h * c[i] * v[l] for l in range(d)] for i in range(8)]
        for _ in range(300):
            G = [rhs.g(Q[i]) for i in range(8)]
            Qn = [[q[l] + h * c[i] * v[l] + h * h * sum(al[i][j] * G[j][l] for j in range(8))
                   for l in range(d)] for i in range(8)]
            err = max(abs(Qn[i][l] - Q[i][l]) for i in range(8) for l in range(d))
            Q = Qn
            if err < Decimal("1e-50"):
                break
        G = [rhs.g(Q[i]) for i in range(8)]
        q1 = [q[l] + h * v[l] + h * h * sum(be[i] * G[i][l] for i in range(8)) for l in range(d)]
        v1 = [v[l] + h * sum(b[i] * G[i][l] for i in range(8)) for l in range(d)]
        return q1, v1


@pytest.mark.parametrize("case", ["kepler", "henon_heiles", "nbody3"])
def test_step_matches_brute_force_collocation(case):
    ex = coeffs.exact_tables()
    if case == "kepler":
        q0, v0 = kepler_ic(0.5)
        kind, params, h = cbind.KEPLER, [1.0], 2 * math.pi / 100
        rhs_mp = P.Kepler(Decimal(1))
    elif case == "henon_heiles":
        q0, v0 = hh_ic()
        kind, params, h = cbind.HENON_HEILES, [1.0], 0.8
        rhs_mp = P.HenonHeiles(Decimal(1))
    else:
        q0 = [0.0, 0.0, 0.0, 5.0, 0.0, 0.1, 0.0, 9.0, -0.2]
        v0 = [0.0, -0.001, 0.0, 0.0, 0.447, 0.0, -0.333, 0.0, 0.01]
        kind, params, h = cbind.NBODY, [1.0, 1.0, 1e-3, 3e-4], 0.5
        rhs_mp = P.NBody([Decimal(1), Decimal("1e-3"), Decimal("3e-4")], G=Decimal(1))
    # take one FP64 step from a state reached after 3 steps (nonzero Rprev)
    r = cbind.run(kind, params, q0, v0, h, 3)
    qs, vs = r["q"][0], r["v"][0]
    r1 = cbind.run(kind, params, qs, vs, h, 1, q_lo=r["q_lo"], v_lo=r["v_lo"], r_prev=r["r_prev"])
    with localcontext() as ctx:
        ctx.prec = 60
        qx = [Decimal(a) + Decimal(b) for a, b in zip(qs, r["q_lo"][0])]
        vx = [Decimal(a) + Decimal(b) for a, b in zip(vs, r["v_lo"][0])]
    # the FP64 stages see only the hi parts, so solve from those too and add lo
    q1, v1 = _collocation_brute_force(rhs_mp, list(qs), list(vs), h, ex)
    with localcontext() as ctx:
        ctx.prec = 60
        q1 = [a + (x - Decimal(s)) for a, x, s in zip(q1, qx, qs)]
        v1 = [a + (x - Decimal(s)) for a, x, s in zip(v1, vx, vs)]
        scale_q = max(abs(x) for x in q1)
        scale_v = max(abs(x) for x in v1)
        got_q = [Decimal(a) + Decimal(b) for a, b in zip(r1["q"][0], r1["q_lo"][0])]
        got_v = [Decimal(a) + Decimal(b) for a, b in zip(r1["v"][0], r1["v_lo"][0])]
        eq = max(abs(a - b) for a, b in zip(got_q, q1)) / scale_q
        ev = max(abs(a - b) for a, b in zip(got_v, v1)) / scale_v
    assert float(eq) <= 1e-15 and float(ev) <= 1e-15, (float(eq), float(ev))


def test_order_16_kepler_high_precision():
    """Order 2s = 16 (Sec. 2.2): global error after one period of the e = 0.1
    Kepler orbit vs Kepler's equation, run in 60-digit arithmetic."""
    tab = coeffs.decimal_tables()
    with localcontext() as ctx:
        ctx.prec = 60
        pi = dec_pi()
        e = Decimal("0.1")
        q0 = [1 - e, Decimal(0)]
        v0 = [Decimal(0), ((1 + e) / (1 - e)).sqrt()]
        hs, errs = [], []
        for N in (32, 48, 64, 96):
            h = 2 * pi / N
            r = P.integrate(q0, v0, h, N, tab, P.Kepler(Decimal(1)))
            qe, _ = kepler_state(e, h * N)
            errs.append(float(max(abs(r["state"].q[i] - qe[i]) for i in range(2))))
            hs.append(float(h))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all((slopes > 15.5) & (slopes < 16.5)), slopes


def test_initial_guess_order():
    """Eq. Pol0: after the first step the extrapolated guess Q^[0] differs
    from the converged stages by O(h^10); the first step (Rprev = 0) by O(h^2)."""
    tab = coeffs.decimal_tables()
    with localcontext() as ctx:
        ctx.prec = 60
        pi = dec_pi()
        e = Decimal("0.1")
        q0 = [1 - e, Decimal(0)]
        v0 = [Decimal(0), ((1 + e) / (1 - e)).sqrt()]
        first, later = [], []
        for N in (64, 128):
            st = P.State(q0, v0)
            errs = []
            for _ in range(3):
                dg = {}
                st, _, _ = P.step(st, 2 * pi / N, tab, P.Kepler(Decimal(1)), diag=dg)
                errs.append(float(max(abs(dg["Q0"][i][l] - dg["Q"][i][l])
                                      for i in range(8) for l in range(2))))
            first.append(errs[0])
            later.append(max(errs[1:]))
    assert 3.5 < first[0] / first[1] < 4.5          # O(h^2)
    assert later[0] / later[1] > 2 ** 8.5            # >= O(h^8.5); measured ~2^10


def test_kepler_100_periods_closed_form():
    """Single Kepler orbit e = 0.5, h = T/200, 100 periods (20,000 steps)."""
    q0, v0 = kepler_ic(0.5)
    h = 2 * math.pi / 200
    r = cbind.run(cbind.KEPLER, [1.0], q0, v0, h, 20000)
    qe, ve = kepler_state(Decimal("0.5"), Decimal(h) * 20000)
    exact = np.array([float(x) for x in qe + ve])
    got = np.concatenate([r["q"][0], r["v"][0]])
    assert np.abs(got - exact).max() / np.abs(exact).max() <= 1e-9
    assert r["dH_max"][0] <= 1e-13
    assert r["status"][0] == 0


def test_symmetry_forward_backward():
    """The method is symmetric: a step of -h from y1 returns to y0."""
    for kind, params, (q0, v0), h in ((cbind.KEPLER, [1.0], kepler_ic(0.5), 2 * math.pi / 100),
                                      (cbind.HENON_HEILES, [1.0], hh_ic(), 0.8)):
        r1 = cbind.run(kind, params, q0, v0, h, 1)
        r2 = cbind.run(kind, params, r1["q"][0], r1["v"][0], -h, 1,
                       q_lo=r1["q_lo"], v_lo=r1["v_lo"])
        y0 = np.array(q0 + v0)
        y2 = np.concatenate([r2["q"][0] + r2["q_lo"][0], r2["v"][0] + r2["v_lo"][0]])
        assert np.abs(y2 - y0).max() / np.abs(y0).max() <= 1e-14


def _jacobian_one_step(rhs, q0, v0, h, masses, nsteps=1):
    d = len(q0)
    n = 2 * d
    q = [P.Dual(q0[l], [1.0 if c == l else 0.0 for c in range(n)]) for l in range(d)]
    # p = m v is the canonical momentum; differentiate with respect to p0
    v = [P.Dual(v0[l], [1.0 / masses[l] if c == d + l else 0.0 for c in range(n)]) for l in range(d)]
    st = P.State(q, v)
    for _ in range(nsteps):
        st, _, status = P.step(st, h, TAB, rhs)
        assert status == P.OK
    outs = [st.q[l] + st.q_lo[l] for l in range(d)] + \
           [(st.v[l] + st.v_lo[l]) * masses[l] for l in range(d)]
    return np.array([o.grad for o in outs])


@pytest.mark.parametrize("case", ["kepler", "henon_heiles", "nbody3"])
def test_symplecticity_dual_numbers(case):
    """Sec. 2.3: the step map is symplectic, M^T J M = J."""
    if case == "kepler":
        (q0, v0), h, rhs, m = kepler_ic(0.5), 2 * math.pi / 100, P.Kepler(1.0), [1.0, 1.0]
    elif case == "henon_heiles":
        (q0, v0), h, rhs, m = hh_ic(), 0.8, P.HenonHeiles(1.0), [1.0, 1.0]
    else:
        ms = [1.0, 1e-3, 3e-4]
        q0 = [0.0, 0.0, 0.0, 5.0, 0.0, 0.1, 0.0, 9.0, -0.2]
        v0 = [0.0, -0.001, 0.0, 0.0, 0.447, 0.0, -0.333, 0.0, 0.01]
        h, rhs, m = 0.5, P.NBody(ms), [x for x in ms for _ in range(3)]
    M = _jacobian_one_step(rhs, q0, v0, h, m, nsteps=2)
    d = len(q0)
    # mass-weighted canonical coordinates (sqrt(m) q, p / sqrt(m)) are a
    # symplectic change of variables that keeps the entries of M near O(1)
    w = np.sqrt(np.asarray(m))
    D = np.diag(np.concatenate([w, 1.0 / w]))
    M = D @ M @ np.linalg.inv(D)
    J = np.block([[np.zeros((d, d)), np.eye(d)], [-np.eye(d), np.zeros((d, d))]])
    err = np.abs(M.T @ J @ M - J).max()
    assert err <= 1e-13, err
    # and the map is far from the identity, so the check is not vacuous
    assert np.abs(M - np.eye(2 * d)).max() > 1e-3


def test_energy_bounded_no_drift_henon_heiles():
    """Sec. 5.1 Henon-Heiles ICs over 2 pi 1e4 at h = 1.0 (local energy
    error ~1e-14, the paper's reference regime): the global energy error stays
    at roundoff level with no linear drift (the stopping rule of Eq. stopping
    is what prevents drift)."""
    q0, v0 = hh_ic()
    h = 1.0
    N = int(round(2 * math.pi * 1e4 / h))
    chunks = 100
    per = N // chunks
    H0 = cbind.hamiltonian(cbind.HENON_HEILES, [1.0], q0, v0)
    st = dict(q=q0, v=v0, q_lo=None, v_lo=None, r_prev=None)
    ts, dHs, gmax = [], [], 0.0
    for c in range(chunks):
        r = cbind.run(cbind.HENON_HEILES, [1.0], st["q"], st["v"], h, per,
                      q_lo=st["q_lo"], v_lo=st["v_lo"], r_prev=st["r_prev"])
        assert r["status"][0] == 0
        st = dict(q=r["q"][0], v=r["v"][0], q_lo=r["q_lo"][0], v_lo=r["v_lo"][0], r_prev=r["r_prev"][0])
        Hn = cbind.hamiltonian(cbind.HENON_HEILES, [1.0], st["q"], st["v"])
        ts.append((c + 1) * per * h)
        dHs.append((Hn - H0) / H0)
        gmax = max(gmax, abs(dHs[-1]))
    slope = np.polyfit(ts, dHs, 1)[0]
    T = ts[-1]
    assert gmax <= 5e-13
    # a drift of one rounding unit per step would give ~6e-12 over T
    assert abs(slope * T) <= 2e-13, slope * T


# ---------------------------------------------------------------- stopping rule
def test_stop_rule_matches_definition():
    """Incremental bookkeeping == the literal Eq. stopping on random sequences."""
    rnd = random.Random(2511036550)
    for _ in range(3000):
        n = rnd.randint(1, 12)
        deltas = [rnd.choice([0.0, 1e-16, 2e-16, 3e-16, rnd.random() * 1e-15]) for _ in range(n)]
        dmin, dprev = float("inf"), float("inf")
        for k in range(1, n + 1):
            cond, dmin, dprev = P.stop_test(deltas[k - 1], dmin, dprev)
            earlier = deltas[:max(k - 2, 0)]
            lit = (deltas[k - 1] == 0) or (
                min(earlier) <= min(deltas[k - 2], deltas[k - 1]) if earlier else False)
            assert cond == lit, (deltas, k)


def test_status_codes():
    q0, v0 = kepler_ic(0.5)
    # the first step needs several sweeps (Rprev = 0): a cap of 2 trips it
    r = cbind.run(cbind.KEPLER, [1.0], q0, v0, 0.05, 5, kmax=2, iters_len=5)
    assert r["status"][0] == P.MAXITER and r["steps"][0] == 0
    assert list(r["q"][0]) == q0 and list(r["v"][0]) == v0
    p = P.integrate(q0, v0, 0.05, 5, TAB, P.Kepler(1.0), kmax=2)
    assert p["status"] == P.MAXITER and p["steps"] == 0
    # a collision (q = 0) gives non-finite stage values
    r = cbind.run(cbind.KEPLER, [1.0], [0.0, 0.0], [0.0, 0.0], 0.05, 3)
    assert r["status"][0] == P.NONFINITE and r["steps"][0] == 0
    # zero steps leave the state untouched
    r = cbind.run(cbind.KEPLER, [1.0], q0, v0, 0.05, 0)
    assert r["status"][0] == 0 and r["steps"][0] == 0 and list(r["q"][0]) == q0
