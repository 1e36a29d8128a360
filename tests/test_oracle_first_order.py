"""Pins of the oracle's first-order form (arXiv 2511.03655, Eq. Yi2 with
Eqs. IRK_init / IRK_FP, stopping rule on all D components, Eq. yn2) and of
the Schwarzschild black-hole right-hand side (Eq. Ham_SBH).

  * f = J grad H against central differences of H in 60 digits (pins the
    hand-derived gradient of Eq. Ham_SBH);
  * C form == Python form, bit for bit;
  * one step on q' = p, p' = -w^2 q equals the [8/8] Pade approximant of
    exp(hA) (closed form);
  * one step equals the collocation solution of Eq. Yi with the exact
    coefficients, solved by brute force in 60 digits;
  * order 16 in 60-digit arithmetic;
  * symplecticity M^T J M = J through Dual numbers, symmetry (+h then -h);
  * bounded energy error over a long FP64 run (Sec. 5.1 initial condition:
    r = 11, theta = pi/2, p_r = 0, p_theta from H = -1/2).
"""
import math
from decimal import Decimal, localcontext

import numpy as np
import pytest

from oracle import cbind, coeffs
from oracle import first_order as F
from oracle.irkgl import Dual
from tests.closed_forms import pade_88_harmonic

TAB = coeffs.fp64_tables()
PAR = [0.995, 4.6, 8.9e-4]


def sbh_dec():
    return F.Schwarzschild(Decimal("0.995"), Decimal("4.6"), Decimal("8.9e-4"))


@pytest.mark.parametrize("y", [["11.3", "1.2", "0.05", "2.1"], ["20.0", "1.5707963", "-0.3", "1.0"],
                               ["9.0", "0.7", "0.2", "-3.0"]])
def test_schwarzschild_f_is_symplectic_gradient(y):
    with localcontext() as ctx:
        ctx.prec = 60
        rhs = sbh_dec()
        y = [Decimal(x) for x in y]
        f = rhs.f(y)
        eps = Decimal("1e-25")
        g = []
        for k in range(4):
            yp, ym = list(y), list(y)
            yp[k] += eps
            ym[k] -= eps
            g.append((rhs.H(yp) - rhs.H(ym)) / (2 * eps))
        Jg = [g[2], g[3], -g[0], -g[1]]
        err = max(abs(a - b) for a, b in zip(f, Jg)) / max(abs(x) for x in f)
    assert err < Decimal("1e-30")


def test_initial_condition_energy():
    y0 = F.schwarzschild_ic(11.0)
    assert y0[3] > 0 and abs(F.Schwarzschild().H(y0) + 0.5) <= 1e-15
    assert F.schwarzschild_ic(7.0) is None  # no p_theta reaches H = -1/2 there


@pytest.mark.parametrize("kind,rhs,y0,h,par", [
    (cbind.SCHWARZSCHILD, F.Schwarzschild(), None, 2.0, PAR),
    (cbind.HARMONIC1, F.Harmonic1(1.3), [1.0, 0.3], 0.4, [1.3]),
])
def test_c_equals_python_bitwise(kind, rhs, y0, h, par):
    y0 = y0 or F.schwarzschild_ic(11.0)
    n = 30
    r = cbind.run1(kind, par, [y0], h, n, iters_len=n)
    p = F.integrate1(y0, h, n, TAB, rhs)
    st = p["state"]
    assert list(r["iters"][0]) == p["iters"]
    assert np.array_equal(r["y"][0], np.asarray(st.y)) and np.array_equal(r["y_lo"][0], np.asarray(st.y_lo))
    assert np.array_equal(r["l_prev"][0], np.asarray(st.l_prev))
    assert r["dH_max"][0] == p["dH_max"]


@pytest.mark.parametrize("wh", [0.1, 0.5, 1.0])
def test_harmonic_first_order_step_is_pade_88(wh):
    q0, p0 = 1.0, 0.3
    R = pade_88_harmonic(1, Decimal(wh))
    r = cbind.run1(cbind.HARMONIC1, [1.0], [[q0, p0]], wh, 1)
    with localcontext() as ctx:
        ctx.prec = 60
        eq = float(R[0][0] * Decimal(q0) + R[0][1] * Decimal(p0))
        ep = float(R[1][0] * Decimal(q0) + R[1][1] * Decimal(p0))
    assert abs(r["y"][0][0] - eq) <= 3e-16 and abs(r["y"][0][1] - ep) <= 3e-16


def _collocation_brute_force_1(rhs, y, h, ex, prec=60):
    """Eq. Yi: Y_i = y + h sum_j a_ij f(Y_j), plain fixed-point iteration to
    1e-50 with the exact coefficients; then y1 = y + h sum_i b_i f(Y_i)."""
    with localcontext() as ctx:
        ctx.prec = prec
        D = len(y)
        y = [Decimal(x) for x in y]
        h = Decimal(h)
        a, b = ex["a"], ex["b"]
        Y = [list(y) for _ in range(8)]
        for _ in range(400):
            Fv = [rhs.f(Y[i]) for i in range(8)]
            Yn = [[y[l] + h * sum(a[i][j] * Fv[j][l] for j in range(8)) for l in range(D)] for i in range(8)]
            err = max(abs(Yn[i][l] - Y[i][l]) for i in range(8) for l in range(D))
            Y = Yn
            if err < Decimal("1e-50"):
                break
        Fv = [rhs.f(Y[i]) for i in range(8)]
        return [y[l] + h * sum(b[i] * Fv[i][l] for i in range(8)) for l in range(D)]


@pytest.mark.parametrize("case", ["schwarzschild", "harmonic"])
def test_step_matches_brute_force_collocation(case):
    ex = coeffs.exact_tables()
    if case == "schwarzschild":
        kind, par, y0, h, rhs_mp = cbind.SCHWARZSCHILD, PAR, F.schwarzschild_ic(11.0), 3.0, sbh_dec()
    else:
        kind, par, y0, h, rhs_mp = cbind.HARMONIC1, [1.0], [1.0, 0.3], 0.7, F.Harmonic1(Decimal(1))
    r = cbind.run1(kind, par, [y0], h, 3)
    ys = r["y"][0]
    r1 = cbind.run1(kind, par, r["y"], h, 1, y_lo=r["y_lo"], l_prev=r["l_prev"])
    y1 = _collocation_brute_force_1(rhs_mp, list(ys), h, ex)
    with localcontext() as ctx:
        ctx.prec = 60
        y1 = [a + Decimal(lo) for a, lo in zip(y1, r["y_lo"][0])]
        got = [Decimal(a) + Decimal(b) for a, b in zip(r1["y"][0], r1["y_lo"][0])]
        err = max(abs(a - b) for a, b in zip(got, y1)) / max(abs(x) for x in y1)
    assert float(err) <= 1e-15, float(err)


def test_order_16_schwarzschild_high_precision():
    """Order 16: error at T = 60 against the method at h = 60/160, 60 digits
    (N = 10..20 steps, where the slope has settled within 0.4 of 16)."""
    tab = coeffs.decimal_tables()
    with localcontext() as ctx:
        ctx.prec = 60
        y0 = F.schwarzschild_ic(Decimal(11), Decimal("0.995"), Decimal("4.6"), Decimal("8.9e-4"))
        rhs = sbh_dec()
        T = Decimal(60)

        def run(N):
            return F.integrate1(y0, T / N, N, tab, rhs)["state"].y

        ref = run(160)
        hs, errs = [], []
        for N in (10, 12, 16, 20):
            yN = run(N)
            errs.append(float(max(abs(yN[i] - ref[i]) for i in range(4))))
            hs.append(float(T / N))
    slopes = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all((slopes > 15.6) & (slopes < 16.5)), (slopes, errs)


def test_symplecticity_dual_numbers():
    y0 = F.schwarzschild_ic(11.0)
    r = cbind.run1(cbind.SCHWARZSCHILD, PAR, [y0], 2.0, 5)
    ys = list(r["y"][0])
    yd = [Dual(ys[k], [1.0 if j == k else 0.0 for j in range(4)]) for k in range(4)]
    st = F.State1(yd)
    for _ in range(2):
        st, _, status = F.step1(st, 2.0, TAB, F.Schwarzschild())
        assert status == 0
    M = np.array([[st.y[i].grad[j] for j in range(4)] for i in range(4)])
    J = np.block([[np.zeros((2, 2)), np.eye(2)], [-np.eye(2), np.zeros((2, 2))]])
    assert np.abs(M.T @ J @ M - J).max() <= 1e-13


def test_symmetry_forward_backward():
    y0 = F.schwarzschild_ic(11.0)
    a = cbind.run1(cbind.SCHWARZSCHILD, PAR, [y0], 2.0, 1)
    b = cbind.run1(cbind.SCHWARZSCHILD, PAR, a["y"], -2.0, 1, y_lo=a["y_lo"])
    back = b["y"][0] + b["y_lo"][0]
    assert np.abs(back - np.array(y0)).max() / np.abs(y0).max() <= 1e-14


def test_energy_bounded_long_run():
    y0 = F.schwarzschild_ic(11.0)
    r = cbind.run1(cbind.SCHWARZSCHILD, PAR, [y0], 2.0, 20000)
    assert r["status"][0] == 0 and r["steps"][0] == 20000
    assert r["dH_max"][0] <= 1e-14
