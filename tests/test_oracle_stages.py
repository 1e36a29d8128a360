"""Pins of the s-stage IRKGL schemes, s = 2, 4, 6 (arXiv 2511.03655,
Sec. 2.2: s-stage Gauss collocation, order 2s; Sec. 5.2 compares them with
s = 8), in the oracle's first-order form and its tables.

  * nodes and weights against numpy's Gauss-Legendre routine (library
    special case), mu_ij + mu_ji = 1 exactly;
  * one step on q' = p, p' = -w^2 q equals the [s/s] Pade approximant of
    exp(hA), the s-stage Gauss stability function (closed form);
  * order 2s in 50-digit arithmetic on the Schwarzschild system;
  * the s-stage tables compiled into the library equal the oracle's.
"""
import os
import re
from decimal import Decimal, localcontext

import numpy as np
import pytest

from oracle import coeffs
from oracle import first_order as F
from tests.closed_forms import pade_harmonic

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.mark.parametrize("s", [2, 4, 6])
def test_tables_gauss_legendre(s):
    t = coeffs.fp64_tables(s)
    x, w = np.polynomial.legendre.leggauss(s)
    assert np.allclose(t["c"], (1 + x) / 2, rtol=0, atol=2e-16)
    assert np.allclose(t["b"], w / 2, rtol=0, atol=2e-16)
    for i in range(s):
        for j in range(s):
            if i != j:
                assert t["mu"][i][j] + t["mu"][j][i] == 1.0


@pytest.mark.parametrize("s", [2, 4, 6])
@pytest.mark.parametrize("wh", [0.1, 0.5])
def test_harmonic_step_is_pade_ss(s, wh):
    tab = coeffs.fp64_tables(s)
    st, k, status = F.step1(F.State1([1.0, 0.3], s=s), wh, tab, F.Harmonic1(1.0))
    assert status == 0
    R = pade_harmonic(s, 1, Decimal(wh))
    with localcontext() as ctx:
        ctx.prec = 60
        eq = float(R[0][0] * Decimal(1.0) + R[0][1] * Decimal(0.3))
        ep = float(R[1][0] * Decimal(1.0) + R[1][1] * Decimal(0.3))
    assert abs(st.y[0] + st.y_lo[0] - eq) <= 3e-16 and abs(st.y[1] + st.y_lo[1] - ep) <= 3e-16


@pytest.mark.parametrize("s,Ns", [(2, (40, 60, 80)), (4, (16, 20, 24)), (6, (12, 16, 20))])
def test_order_2s_schwarzschild(s, Ns):
    tab = coeffs.decimal_tables(s)
    with localcontext() as ctx:
        ctx.prec = 50
        y0 = F.schwarzschild_ic(Decimal(11), Decimal("0.995"), Decimal("4.6"), Decimal("8.9e-4"))
        rhs = F.Schwarzschild(Decimal("0.995"), Decimal("4.6"), Decimal("8.9e-4"))
        T = Decimal(60)

        def run(N):
            return F.integrate1(y0, T / N, N, tab, rhs)["state"].y

        ref = run(4 * Ns[-1])
        errs = [float(max(abs(a - b) for a, b in zip(run(N), ref))) for N in Ns]
    slopes = np.diff(np.log(errs)) / np.diff(np.log([float(T) / N for N in Ns]))
    assert np.all(np.abs(slopes - 2 * s) < 0.6), (slopes, errs)


def test_library_tables_equal_oracle():
    txt = open(os.path.join(HERE, "..", "paper_2511_03655_gb300", "csrc", "irkgl_tables.h")).read()

    def arr(name):
        m = re.search(r"static const double %s\[\d+\] = \{(.*?)\};" % name, txt, re.S)
        return [float.fromhex(v.strip()) for v in m.group(1).split(",")]

    for s in (2, 4, 6):
        t = coeffs.fp64_tables(s)
        assert arr(f"IRKGL_TAB{s}_C") == t["c"] and arr(f"IRKGL_TAB{s}_B") == t["b"]
        assert arr(f"IRKGL_TAB{s}_MU") == [x for r in t["mu"] for x in r]
        assert arr(f"IRKGL_TAB{s}_NU") == [x for r in t["nu"] for x in r]
