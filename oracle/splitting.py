"""Explicit symplectic splitting baselines (oracle side).

Test infrastructure only (see ``oracle/__init__.py``).

arXiv 2511.03655, Sec. 4: for H = T(v) + U(q) the exact flows are the drift
phi^A_t(q, v) = (q + t v, v) and the kick phi^B_t(q, v) = (q, v + t g(q))
(Eq. flowAB).  A symmetric composition of s Strang steps
(Eqs. Strang, comp_method) with weights gamma_1..gamma_s (gamma_{s+1-j} =
gamma_j) is the drift-kick sequence of Eq. high_order_splitting,

    A_{a_{s+1} h} B_{b_s h} A_{a_s h} ... B_{b_1 h} A_{a_1 h},
    a_1 = gamma_1 / 2,  a_j = (gamma_{j-1} + gamma_j) / 2,  a_{s+1} = gamma_s / 2,
    b_j = gamma_j,

applied right to left (A_{a_1 h} first).  Schemes:

  strang   s = 1, gamma = (1,): second order.
  suz90    s = 5, Suzuki's fourth-order composition: gamma_1 = gamma_2 =
           gamma_4 = gamma_5 = p, gamma_3 = 1 - 4 p, p = 1 / (4 - 4^(1/3))
           (the real root of 4 p^3 + (1 - 4 p)^3 = 0, so the third-order
           error terms of the five second-order steps cancel).

The coefficients are computed here in 50-digit arithmetic and rounded once.
Every update is a compensated sum: q and v are (hi, lo) pairs updated by the
same TwoSum + Fast2Sum rule as the IRKGL oracle (the paper applies
compensated summation to the splitting methods of its second-order tests);
the flows see the hi parts only.  A step costs s evaluations of g.
"""
from __future__ import annotations

from decimal import Decimal, localcontext

from .irkgl import MAXITER, NONFINITE, OK, _isfinite, two_sum_add, value, zero_like  # noqa: F401

SCHEMES = ("strang", "suz90")


def gammas(scheme: str, prec: int = 50) -> list[Decimal]:
    with localcontext() as ctx:
        ctx.prec = prec
        if scheme == "strang":
            return [Decimal(1)]
        if scheme == "suz90":
            p = 1 / (4 - Decimal(4) ** (Decimal(1) / 3))
            return [p, p, 1 - 4 * p, p, p]
    raise ValueError(scheme)


def coefficients(scheme: str, exact: bool = False):
    """(a[0..s], b[0..s-1]) of Eq. high_order_splitting; floats rounded once
    from 50-digit values, or the Decimals themselves (exact=True)."""
    g = gammas(scheme)
    s = len(g)
    with localcontext() as ctx:
        ctx.prec = 50
        a = [g[0] / 2] + [(g[j - 1] + g[j]) / 2 for j in range(1, s)] + [g[s - 1] / 2]
        b = list(g)
    if exact:
        return a, b
    return [float(x) for x in a], [float(x) for x in b]


class SplitState:
    def __init__(self, q, v, q_lo=None, v_lo=None):
        d = len(q)
        z = zero_like(q[0])
        self.q, self.v = list(q), list(v)
        self.q_lo = list(q_lo) if q_lo is not None else [z] * d
        self.v_lo = list(v_lo) if v_lo is not None else [z] * d


def split_step(st: SplitState, h, coef, rhs):
    """One step of the drift-kick sequence; returns (new_state, g_evals, status)."""
    a, b = coef
    s = len(b)
    q, v = list(st.q), list(st.v)
    ql, vl = list(st.q_lo), list(st.v_lo)
    d = len(q)
    for j in range(s):
        # drift A_{a_j h}: q += (a_j h) v
        ah = a[j] * h
        for l in range(d):
            q[l], ql[l] = two_sum_add(q[l], ql[l], ah * v[l])
        # kick B_{b_j h}: v += (b_j h) g(q)
        G = rhs.g(q)
        bh = b[j] * h
        for l in range(d):
            v[l], vl[l] = two_sum_add(v[l], vl[l], bh * G[l])
    ah = a[s] * h
    for l in range(d):
        q[l], ql[l] = two_sum_add(q[l], ql[l], ah * v[l])
    if not all(_isfinite(x) for x in q + v):
        return st, s, NONFINITE
    return SplitState(q, v, ql, vl), s, OK


def split_integrate(q0, v0, h, nsteps, scheme, rhs, local=False):
    """nsteps steps; final state, g evaluations, status, steps and the max
    energy error (global |(H_n - H_0)/H_0|, or local (Eq. DHlocmax))."""
    coef = coefficients(scheme)
    st = SplitState(q0, v0)
    H0 = Hp = rhs.H(st.q, st.v)
    dmax = 0.0
    evals = 0
    status = OK
    n = 0
    for n in range(1, nsteps + 1):
        st2, e, status = split_step(st, h, coef, rhs)
        evals += e
        if status != OK:
            n -= 1
            break
        st = st2
        Hn = rhs.H(st.q, st.v)
        ref = Hp if local else H0
        dH = abs(value((Hn - ref) / ref))
        dmax = max(dmax, dH)
        Hp = Hn
    return {"state": st, "g_evals": evals, "status": status, "steps": n, "dH_max": dmax}
