"""Pins of the oracle's coefficient tables (Sec. 2.2-2.4 of arXiv 2511.03655).

Every check compares against something other than the oracle's own
construction: a library routine (numpy's Gauss-Legendre rule), the
quadrature order conditions B(2s) that only Gauss nodes satisfy, an
independent construction by integrating the Lagrange basis, the
symplecticity conditions Eq. sym / Eq. sym2 (not imposed by the
construction), and the golden text file written by tests/golden/make_golden.py.
"""
import os
from decimal import Decimal, localcontext
from fractions import Fraction

import numpy as np
import pytest

from oracle import coeffs

S = 8
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "irkgl16_coeffs_fp64.txt")


@pytest.fixture(scope="module")
def ex():
    return coeffs.exact_tables(S)


@pytest.fixture(scope="module")
def fp():
    return coeffs.fp64_tables(S)


def test_nodes_weights_match_numpy_leggauss(fp):
    # library special case: numpy's Golub-Welsch Gauss-Legendre rule on [-1, 1]
    # (1 + x)/2 rounds once in absolute terms (~1.1e-16), so compare on x
    x, w = np.polynomial.legendre.leggauss(S)
    for i in range(S):
        assert abs((2 * Fraction(fp["c"][i]) - 1) - Fraction(x[i])) <= Fraction(3, 10 ** 16)
        assert abs(fp["b"][i] - w[i] / 2) <= 1e-15  # numpy weights carry ~1e-15 error


def test_quadrature_order_2s(ex):
    # B(16): sum_j b_j c_j^(k-1) = 1/k for k = 1..16 holds only for Gauss nodes
    with localcontext() as ctx:
        ctx.prec = 80
        for k in range(1, 2 * S + 1):
            lhs = sum(ex["b"][j] * ex["c"][j] ** (k - 1) for j in range(S))
            assert abs(lhs - Decimal(1) / k) < Decimal("1e-70")
        lhs = sum(ex["b"][j] * ex["c"][j] ** (2 * S) for j in range(S))
        assert abs(lhs - Decimal(1) / (2 * S + 1)) > Decimal("1e-12")  # B(17) fails


def test_node_weight_symmetry(ex, fp):
    for i in range(S):
        assert abs(ex["c"][i] + ex["c"][S - 1 - i] - 1) < Decimal("1e-75")
        assert abs(ex["b"][i] - ex["b"][S - 1 - i]) < Decimal("1e-75")
        assert fp["b"][i] == fp["b"][S - 1 - i]


def _lagrange_integrals(c, lo_of_i, hi_of_i):
    """integral_{lo(i)}^{hi(i)} l_j(u) du with l_j the Lagrange basis on c,
    by expanding l_j into monomials and integrating term by term."""
    n = len(c)
    out = [[None] * n for _ in range(n)]
    with localcontext() as ctx:
        ctx.prec = 80
        for j in range(n):
            poly = [Decimal(1)]  # coefficients, lowest degree first
            den = Decimal(1)
            for m in range(n):
                if m == j:
                    continue
                new = [Decimal(0)] * (len(poly) + 1)
                for p, a in enumerate(poly):
                    new[p + 1] += a
                    new[p] -= a * c[m]
                poly = new
                den *= c[j] - c[m]
            prim = [Decimal(0)] + [a / (p + 1) for p, a in enumerate(poly)]

            def F(u):
                acc = Decimal(0)
                for a in reversed(prim):  # Horner
                    acc = acc * u + a
                return acc

            for i in range(n):
                out[i][j] = (F(hi_of_i(i)) - F(lo_of_i(i))) / den
    return out


def test_A_matches_lagrange_integration(ex):
    # a_ij = integral_0^{c_i} l_j: collocation (Sec. 2.2), independent route
    c = ex["c"]
    a2 = _lagrange_integrals(c, lambda i: Decimal(0), lambda i: c[i])
    b2 = _lagrange_integrals(c, lambda i: Decimal(0), lambda i: Decimal(1))
    with localcontext() as ctx:
        ctx.prec = 80
        for i in range(S):
            assert abs(b2[0][i] - ex["b"][i]) < Decimal("1e-70")
            for j in range(S):
                assert abs(a2[i][j] - ex["a"][i][j]) < Decimal("1e-70")


def test_nu_matches_lagrange_extrapolation(ex, fp):
    # nut_ij = integral_1^{1+c_i} l_j (Eq. Pol0, extrapolation of the
    # previous step's collocation polynomial); nu = nut / b
    c = ex["c"]
    n2 = _lagrange_integrals(c, lambda i: Decimal(1), lambda i: 1 + c[i])
    with localcontext() as ctx:
        ctx.prec = 80
        for i in range(S):
            for j in range(S):
                assert abs(n2[i][j] - ex["nut"][i][j]) < Decimal("1e-60")
                assert fp["nu"][i][j] == float(n2[i][j] / ex["b"][j])


def test_irk_symplecticity_eq_sym(ex):
    # Eq. sym: b_i a_ij + b_j a_ji = b_i b_j (not imposed by the construction)
    a, b = ex["a"], ex["b"]
    with localcontext() as ctx:
        ctx.prec = 80
        for i in range(S):
            for j in range(S):
                assert abs(b[i] * a[i][j] + b[j] * a[j][i] - b[i] * b[j]) < Decimal("1e-70")


def test_irkn_conditions_eq_sym2(ex):
    # Eq. sym2: beta_i = b_i (1 - c_i); b_i (beta_j - alpha_ij) = b_j (beta_i - alpha_ji)
    a, b, c, al, be = ex["a"], ex["b"], ex["c"], ex["alpha"], ex["beta"]
    with localcontext() as ctx:
        ctx.prec = 80
        for i in range(S):
            assert abs(be[i] - b[i] * (1 - c[i])) < Decimal("1e-70")
            assert abs(sum(a[i]) - c[i]) < Decimal("1e-70")  # c_i = sum_k a_ik (Sec. 2.3)
            for j in range(S):
                lhs = b[i] * (be[j] - al[i][j])
                rhs = b[j] * (be[i] - al[j][i])
                assert abs(lhs - rhs) < Decimal("1e-70")


def test_mu_exact_complement(fp, ex):
    # Sec. 2.4: mu_ij + mu_ji = 1 exactly in FP64; mu_ii = 1/2 (a_ii = b_i/2 by Eq. sym)
    mu = fp["mu"]
    for i in range(S):
        assert mu[i][i] == 0.5
        for j in range(S):
            if i != j:
                assert Fraction(mu[i][j]) + Fraction(mu[j][i]) == 1
            with localcontext() as ctx:
                ctx.prec = 80
                assert abs(Decimal(mu[i][j]) * ex["b"][j] - ex["a"][i][j]) < Decimal("1e-16")


def test_eta_exact_symplectic_condition(fp, ex):
    # Eq. sympl_cond_2 holds exactly over the FP64 numbers ...
    eta, c = fp["eta"], fp["c"]
    for i in range(S):
        for j in range(S):
            assert Fraction(eta[i][j]) + Fraction(c[j]) == Fraction(eta[j][i]) + Fraction(c[i])
    # ... and eta_ij b_j reproduces alpha_ij in every entry (this rejects the
    # upper-triangle sign as printed in Sec. 2.4, which misses by up to ~1.9)
    with localcontext() as ctx:
        ctx.prec = 80
        for i in range(S):
            for j in range(S):
                assert abs(Decimal(eta[i][j]) * ex["b"][j] - ex["alpha"][i][j]) < Decimal("1e-16")


def test_printed_eta_sign_is_rejected(fp, ex):
    # the literal printed rule eta_ij = c_i - c_j - eta_ji (i < j) is far off alpha/b
    eta, c = fp["eta"], fp["c"]
    worst = max(abs(Decimal(c[i] - c[j] - eta[j][i]) - ex["alpha"][i][j] / ex["b"][j])
                for i in range(S) for j in range(i + 1, S))
    assert worst > Decimal("0.5")


def test_golden_file_matches_oracle(fp):
    with open(GOLDEN) as f:
        lines = [ln for ln in f.read().splitlines() if ln and not ln.startswith("#")]
    assert "\n".join(lines) + "\n" == coeffs.hexdump(fp)
