"""Pins of the oracle's time-dependent path: g(t, q) evaluated at the stage
times t_n + c_i h (arXiv 2511.03655, Eq. IRK_FP first line, and the
non-autonomous Henon-Heiles system printed in Sec. 3).

  * C form == Python form, bit for bit, from a nonzero start time;
  * xi = 0 reduces to the autonomous Henon-Heiles kind bit for bit;
  * one step equals the collocation solution with the stage times
    t + c_i h, solved by brute force in 60 digits with the exact
    coefficients (a misplaced stage time fails it by many orders);
  * order 16 in 60-digit arithmetic (a stage time at t_n instead of
    t_n + c_i h drops the order to 1);
  * the time is carried as a compensated pair: two runs of n steps equal
    one run of 2n steps bit for bit, and t_n = t_0 + n h to roundoff.
"""
import math
from decimal import Decimal, localcontext

import numpy as np
import pytest

from oracle import cbind, coeffs
from oracle import irkgl as P
from tests.test_oracle_step import hh_ic

TAB = coeffs.fp64_tables()
LAM, XI = 1.0, 0.5


def test_sin_decimal_matches_float():
    with localcontext() as ctx:
        ctx.prec = 50
        for x in ("0.3", "2.5", "-7.25", "40.125"):
            assert abs(float(P.sin(Decimal(x))) - math.sin(float(x))) <= 2e-16


def test_c_equals_python_bitwise_forced():
    q0, v0 = hh_ic()
    n, h, t0 = 20, 0.6, 1.25
    r = cbind.run(cbind.HH_FORCED, [LAM, XI], q0, v0, h, n, t0=t0, iters_len=n)
    p = P.integrate(q0, v0, h, n, TAB, P.HenonHeilesForced(LAM, XI), t0=t0)
    st = p["state"]
    assert list(r["iters"][0]) == p["iters"]
    for a, b in ((r["q"][0], st.q), (r["v"][0], st.v), (r["q_lo"][0], st.q_lo), (r["v_lo"][0], st.v_lo)):
        assert np.array_equal(np.asarray(a), np.asarray(b, dtype=np.float64))
    assert r["t"][0] == st.t and r["t_lo"][0] == st.t_lo
    assert r["dH_max"][0] == 0.0 and p["dH_max"] == 0.0


def test_xi_zero_is_autonomous_henon_heiles():
    q0, v0 = hh_ic()
    a = cbind.run(cbind.HH_FORCED, [LAM, 0.0], q0, v0, 0.5, 200, t0=3.0, iters_len=200)
    b = cbind.run(cbind.HENON_HEILES, [LAM], q0, v0, 0.5, 200, iters_len=200)
    for f in ("q", "v", "q_lo", "v_lo", "r_prev", "iters"):
        assert np.array_equal(a[f], b[f]), f


def _collocation_brute_force_t(rhs, t, q, v, h, ex, prec=60):
    """Eq. Qi with a time-dependent g: Q_i = q + h c_i v
    + h^2 sum_j alpha_ij g(t + c_j h, Q_j), solved by plain fixed-point
    iteration to 1e-50; then q1 = q + h v + h^2 sum beta_i g_i,
    v1 = v + h sum b_i g_i."""
    with localcontext() as ctx:
        ctx.prec = prec
        d = len(q)
        q = [Decimal(x) for x in q]
        v = [Decimal(x) for x in v]
        h, t = Decimal(h), Decimal(t)
        c, b, al, be = ex["c"], ex["b"], ex["alpha"], ex["beta"]
        tau = [t + c[i] * h for i in range(8)]
        Q = [[q[l] + h * c[i] * v[l] for l in range(d)] for i in range(8)]
        for _ in range(300):
            G = [rhs.g(Q[i], tau[i]) for i in range(8)]
            Qn = [[q[l] + h * c[i] * v[l] + h * h * sum(al[i][j] * G[j][l] for j in range(8))
                   for l in range(d)] for i in range(8)]
            err = max(abs(Qn[i][l] - Q[i][l]) for i in range(8) for l in range(d))
            Q = Qn
            if err < Decimal("1e-50"):
                break
        G = [rhs.g(Q[i], tau[i]) for i in range(8)]
        q1 = [q[l] + h * v[l] + h * h * sum(be[i] * G[i][l] for i in range(8)) for l in range(d)]
        v1 = [v[l] + h * sum(b[i] * G[i][l] for i in range(8)) for l in range(d)]
        return q1, v1


@pytest.mark.parametrize("t0,h", [(0.0, 0.8), (2.75, 0.6), (-1.5, 0.9)])
def test_step_matches_brute_force_collocation_forced(t0, h):
    ex = coeffs.exact_tables()
    q0, v0 = hh_ic()
    # one FP64 step from a state reached after 3 steps (nonzero Rprev, t != t0)
    r = cbind.run(cbind.HH_FORCED, [LAM, XI], q0, v0, h, 3, t0=t0)
    qs, vs, ts = r["q"][0], r["v"][0], r["t"][0]
    r1 = cbind.run(cbind.HH_FORCED, [LAM, XI], qs, vs, h, 1, q_lo=r["q_lo"], v_lo=r["v_lo"],
                   r_prev=r["r_prev"], t0=ts, t_lo=r["t_lo"])
    rhs_mp = P.HenonHeilesForced(Decimal(LAM), Decimal(XI))
    q1, v1 = _collocation_brute_force_t(rhs_mp, ts, list(qs), list(vs), h, ex)
    with localcontext() as ctx:
        ctx.prec = 60
        q1 = [a + Decimal(lo) for a, lo in zip(q1, r["q_lo"][0])]
        v1 = [a + Decimal(lo) for a, lo in zip(v1, r["v_lo"][0])]
        got_q = [Decimal(a) + Decimal(b) for a, b in zip(r1["q"][0], r1["q_lo"][0])]
        got_v = [Decimal(a) + Decimal(b) for a, b in zip(r1["v"][0], r1["v_lo"][0])]
        eq = max(abs(a - b) for a, b in zip(got_q, q1)) / max(abs(x) for x in q1)
        ev = max(abs(a - b) for a, b in zip(got_v, v1)) / max(abs(x) for x in v1)
    assert float(eq) <= 1e-15 and float(ev) <= 1e-15, (float(eq), float(ev))


def test_order_16_forced_high_precision():
    """Order 2s = 16 for the non-autonomous system, 60-digit arithmetic:
    the error at T = 3 against the same method at h = 3/128 falls like h^16
    (N = 8..16 steps; below 8 the error constants are not yet asymptotic)."""
    tab = coeffs.decimal_tables()
    q0f, v0f = hh_ic()
    with localcontext() as ctx:
        ctx.prec = 60
        q0 = [Decimal(x) for x in q0f]
        v0 = [Decimal(x) for x in v0f]
        rhs = P.HenonHeilesForced(Decimal(LAM), Decimal(XI))
        T, t0 = Decimal(3), Decimal("0.7")

        def run(N):
            r = P.integrate(q0, v0, T / N, N, tab, rhs, t0=t0)
            return r["state"].q

        ref = run(128)
        hs, errs = [], []
        for N in (8, 10, 12, 16):
            qN = run(N)
            errs.append(float(max(abs(qN[i] - ref[i]) for i in range(2))))
            hs.append(float(T / N))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all((slopes > 15.5) & (slopes < 16.5)), (slopes, errs)


def test_time_continuation_bitwise_and_exact():
    q0, v0 = hh_ic()
    h, n, t0 = 0.3, 150, 0.1
    one = cbind.run(cbind.HH_FORCED, [LAM, XI], q0, v0, h, 2 * n, t0=t0)
    a = cbind.run(cbind.HH_FORCED, [LAM, XI], q0, v0, h, n, t0=t0)
    b = cbind.run(cbind.HH_FORCED, [LAM, XI], a["q"], a["v"], h, n, q_lo=a["q_lo"], v_lo=a["v_lo"],
                  r_prev=a["r_prev"], t0=a["t"], t_lo=a["t_lo"])
    for f in ("q", "v", "q_lo", "v_lo", "r_prev", "t", "t_lo"):
        assert np.array_equal(one[f], b[f]), f
    from fractions import Fraction
    exact = Fraction(t0) + 2 * n * Fraction(h)
    got = Fraction(float(one["t"][0])) + Fraction(float(one["t_lo"][0]))
    assert abs(float(got - exact)) <= 1e-30 + 4 * 2.0 ** -104 * float(exact)


def test_planted_stage_time_mistake_is_caught(monkeypatch):
    """A stage time at t_n (instead of t_n + c_i h), planted in the Python
    oracle, moves one step far outside the brute-force bound."""
    ex = coeffs.exact_tables()
    q0, v0 = hh_ic()
    h, t0 = 0.6, 2.75
    rhs_mp = P.HenonHeilesForced(Decimal(LAM), Decimal(XI))
    q1, v1 = _collocation_brute_force_t(rhs_mp, t0, q0, v0, h, ex)

    def err(state):
        return max(abs(float(Decimal(a) - b)) for a, b in zip(state.q + state.v, q1 + v1))

    good, _, _ = P.step(P.State(q0, v0, t=t0), h, TAB, P.HenonHeilesForced(LAM, XI))
    monkeypatch.setattr(P, "stage_times", lambda t, hh, c: [t] * P.S)
    bad, _, _ = P.step(P.State(q0, v0, t=t0), h, TAB, P.HenonHeilesForced(LAM, XI))
    assert err(good) <= 1e-15
    assert err(bad) > 1e-6
