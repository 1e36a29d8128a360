"""Pins of the explicit splitting baselines (arXiv 2511.03655, Sec. 4:
Eqs. Strang, flowAB, comp_method, high_order_splitting; Suzuki's
fourth-order composition SUZ90).

  * coefficients: consistency sum a = sum b = 1, symmetry, and the
    defining cubic of Suzuki's weight 4 p^3 + (1 - 4 p)^3 = 0;
  * C form == Python form, bit for bit;
  * one Strang step on q'' = -w^2 q equals the Stormer-Verlet matrix
    [[1 - z^2/2, h (1 - z^2/4)], [-w^2 h, 1 - z^2/2]], z = w h (closed form);
  * orders 2 and 4 against the closed-form Kepler solution (60 digits);
  * symplecticity (Dual numbers) and time reversibility.
"""
import math
from decimal import Decimal, localcontext

import numpy as np
import pytest

from oracle import cbind
from oracle import irkgl as P
from oracle import splitting as SP
from oracle.irkgl import Dual
from tests.closed_forms import dec_pi, kepler_state


@pytest.mark.parametrize("scheme", SP.SCHEMES)
def test_coefficients(scheme):
    a, b = SP.coefficients(scheme, exact=True)
    with localcontext() as ctx:
        ctx.prec = 50
        assert abs(sum(a) - 1) < Decimal("1e-45") and abs(sum(b) - 1) < Decimal("1e-45")
        assert all(abs(a[i] - a[-1 - i]) < Decimal("1e-45") for i in range(len(a)))
        assert all(abs(b[i] - b[-1 - i]) < Decimal("1e-45") for i in range(len(b)))
        if scheme == "suz90":
            p = b[0]
            assert abs(4 * p ** 3 + (1 - 4 * p) ** 3) < Decimal("1e-45")


@pytest.mark.parametrize("scheme", SP.SCHEMES)
@pytest.mark.parametrize("kind,params,rhs,q0,v0,h", [
    (cbind.HENON_HEILES, [1.0], P.HenonHeiles(1.0), [0.0, 0.3], [0.2338090388900024, 0.2], 0.1),
    (cbind.KEPLER, [1.0], P.Kepler(1.0), [0.5, 0.0], [0.0, math.sqrt(3.0)], 2 * math.pi / 400),
    (cbind.NBODY, [1.0, 1.0, 1e-3, 3e-4], P.NBody([1.0, 1e-3, 3e-4]),
     [0.0, 0.0, 0.0, 5.0, 0.0, 0.1, 0.0, 9.0, -0.2], [0.0, 0.0, 0.0, 0.0, 0.447, 0.0, -0.333, 0.0, 0.01], 0.2),
])
def test_c_equals_python_bitwise(scheme, kind, params, rhs, q0, v0, h):
    r = cbind.run_split(scheme, kind, params, [q0], [v0], h, 60, local=True)
    p = SP.split_integrate(q0, v0, h, 60, scheme, rhs, local=True)
    st = p["state"]
    for a, b in ((r["q"][0], st.q), (r["v"][0], st.v), (r["q_lo"][0], st.q_lo), (r["v_lo"][0], st.v_lo)):
        assert np.array_equal(np.asarray(a), np.asarray(b, dtype=np.float64))
    assert r["dH_max"][0] == p["dH_max"]


@pytest.mark.parametrize("wh", [0.05, 0.3, 1.0])
def test_strang_harmonic_is_stormer_verlet_matrix(wh):
    q0, v0 = 1.0, 0.3
    r = cbind.run_split("strang", cbind.HARMONIC, [1.0], [[q0]], [[v0]], wh, 1)
    z2 = wh * wh
    eq = (1 - z2 / 2) * q0 + wh * (1 - z2 / 4) * v0
    ev = -wh * q0 + (1 - z2 / 2) * v0
    assert abs(r["q"][0][0] + r["q_lo"][0][0] - eq) <= 4e-16
    assert abs(r["v"][0][0] + r["v_lo"][0][0] - ev) <= 4e-16


@pytest.mark.parametrize("scheme,order,Ns", [("strang", 2, (400, 800, 1600)), ("suz90", 4, (100, 200, 400))])
def test_order_against_kepler_closed_form(scheme, order, Ns):
    with localcontext() as ctx:
        ctx.prec = 40
        e = Decimal("0.1")
        q0 = [1 - e, Decimal(0)]
        v0 = [Decimal(0), ((1 + e) / (1 - e)).sqrt()]
        T = 2 * dec_pi()
        errs = []
        a, b = SP.coefficients(scheme, exact=True)
        for N in Ns:
            h = T / N
            st = SP.SplitState(q0, v0)
            for _ in range(N):
                st, _, _ = SP.split_step(st, h, (a, b), P.Kepler(Decimal(1)))
            qe, _ = kepler_state(e, T)
            errs.append(float(max(abs(st.q[i] + st.q_lo[i] - qe[i]) for i in range(2))))
    slopes = -np.diff(np.log(errs)) / np.diff(np.log(Ns))
    assert np.all(np.abs(slopes - order) < 0.15), (slopes, errs)


def test_symplectic_and_reversible():
    q0, v0 = [0.0, 0.3], [0.2338090388900024, 0.2]
    coef = SP.coefficients("suz90")
    qd = [Dual(q0[k], [1.0 if j == k else 0.0 for j in range(4)]) for k in range(2)]
    vd = [Dual(v0[k], [1.0 if j == k + 2 else 0.0 for j in range(4)]) for k in range(2)]
    st = SP.SplitState(qd, vd)
    for _ in range(3):
        st, _, _ = SP.split_step(st, 0.3, coef, P.HenonHeiles(1.0))
    M = np.array([[x.grad[j] for j in range(4)] for x in st.q + st.v])
    J = np.block([[np.zeros((2, 2)), np.eye(2)], [-np.eye(2), np.zeros((2, 2))]])
    assert np.abs(M.T @ J @ M - J).max() <= 1e-14
    f = cbind.run_split("suz90", cbind.HENON_HEILES, [1.0], [q0], [v0], 0.3, 50)
    b = cbind.run_split("suz90", cbind.HENON_HEILES, [1.0], f["q"], f["v"], -0.3, 50,
                        q_lo=f["q_lo"], v_lo=f["v_lo"])
    back = np.concatenate([b["q"][0] + b["q_lo"][0], b["v"][0] + b["v_lo"][0]])
    assert np.abs(back - np.array(q0 + v0)).max() <= 1e-14
