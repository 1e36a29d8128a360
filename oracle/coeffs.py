"""IRKGL coefficient tables, derived from the paper's definitions (oracle side).

Test infrastructure only (see ``oracle/__init__.py``).

Everything is computed in 80-significant-digit ``decimal`` arithmetic and
rounded ONCE to FP64 with Python's correctly rounded ``float()`` conversion,
so the tables are bit-identical on every host.

Definitions followed (arXiv 2511.03655):

* nodes      c_i = (1 + x_i)/2, x_i the zeros of the Legendre polynomial P_s,
             increasing (Sec. 2.2, after the collocation conditions).
* A, b       the collocation conditions of Sec. 2.2:
               sum_j a_ij c_j^(k-1) = c_i^k / k,  sum_j b_j c_j^(k-1) = 1/k,
             k = 1..s, solved as linear systems.
* alpha, beta  the IRKN coefficients of Eq. Qi / Eq. qnvn:
             alpha = A A,  beta_i = sum_k b_k a_ki.
* mu         Sec. 2.4 (first-order floating-point form, Eq. Yi2):
             mu_ij = fl(a_ij / b_j) for j <= i, mu_ij = 1 - mu_ji for i < j.
* eta        Sec. 2.4 (second-order form, Eq. Qi2):
             eta_ij = fl(alpha_ij / b_j) for j <= i and, for i < j, the value
             that makes Eq. sympl_cond_2 (eta_ij + c_j = eta_ji + c_i) hold
             exactly:  eta_ij = eta_ji + c_i - c_j.  The paper prints the
             upper-triangle rule with the opposite sign (c_i - c_j - eta_ji);
             that form contradicts Eq. sympl_cond_2, which it claims to
             guarantee, so the sign of Eq. sympl_cond_2 is taken.  The sum is
             evaluated exactly in rationals from the FP64 values and must be
             an FP64 number (the paper states it is, for s <= 16).
* nu         Eq. Pol0: P_{n-1}(t_{n-1} + h c_i) = y_{n-1} + sum_j nu_ij L_{n-1,j}.
             The printed moment system writes (c_i - 1)^(k-1) inside the sum
             over j, which makes it singular; the extrapolation of the
             collocation polynomial gives (c_j - 1)^(k-1):
               sum_j nut_ij (c_j - 1)^(k-1) = c_i^k / k,
             i.e. nut_ij = integral_1^(1+c_i) l_j(u) du.  Since the paper
             applies nu to L = h b F (Eqs. IRK_init, IRK_init2) while nut
             multiplies h F, nu_ij = fl(nut_ij / b_j).

Parity pins (tests/test_oracle_coeffs.py): nodes and weights against
``numpy.polynomial.legendre.leggauss`` (a library routine), the quadrature
order conditions B(2s), the simplifying conditions C(s), exact
mu_ij + mu_ji = 1 and exact Eq. sympl_cond_2 in rationals, beta = b(1-c)
(Eq. sym2), the IRK symplecticity condition Eq. sym on the exact values, and
nu against direct integration of the Lagrange basis.
"""
from __future__ import annotations

import math
from decimal import Decimal, getcontext, localcontext
from fractions import Fraction
from functools import lru_cache

DIGITS = 80


def _legendre_and_derivative(n: int, x: Decimal):
    """P_n(x) and P_n'(x) by the three-term recurrence (Bonnet)."""
    p0, p1 = Decimal(1), x
    if n == 0:
        return p0, Decimal(0)
    for k in range(1, n):
        p0, p1 = p1, ((2 * k + 1) * x * p1 - k * p0) / (k + 1)
    dp = n * (x * p1 - p0) / (x * x - 1)
    return p1, dp


def legendre_roots(n: int) -> list[Decimal]:
    """Zeros of P_n, increasing, by Newton's method from the classical
    cos(pi (i - 1/4)/(n + 1/2)) starting points."""
    roots = []
    for i in range(1, n + 1):
        x = Decimal(repr(math.cos(math.pi * (i - 0.25) / (n + 0.5))))
        for _ in range(200):
            p, dp = _legendre_and_derivative(n, x)
            dx = p / dp
            x -= dx
            if abs(dx) < Decimal(10) ** (-(DIGITS - 5)):
                break
        roots.append(x)
    return sorted(roots)


def _solve(mat: list[list[Decimal]], rhs: list[Decimal]) -> list[Decimal]:
    """Gaussian elimination with partial pivoting (small dense system)."""
    n = len(rhs)
    a = [row[:] + [rhs[i]] for i, row in enumerate(mat)]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(a[r][col]))
        a[col], a[piv] = a[piv], a[col]
        for r in range(col + 1, n):
            f = a[r][col] / a[col][col]
            for cc in range(col, n + 1):
                a[r][cc] -= f * a[col][cc]
    x = [Decimal(0)] * n
    for r in range(n - 1, -1, -1):
        acc = a[r][n]
        for cc in range(r + 1, n):
            acc -= a[r][cc] * x[cc]
        x[r] = acc / a[r][r]
    return x


def _fl(x: Decimal) -> float:
    """Round a decimal number to the nearest FP64 number (ties to even)."""
    return float(x)


@lru_cache(maxsize=None)
def exact_tables(s: int = 8) -> dict:
    """High-precision (80-digit Decimal) c, b, A, alpha, beta, nut for the
    s-stage Gauss-Legendre collocation method (Sec. 2.2-2.3)."""
    with localcontext() as ctx:
        ctx.prec = DIGITS
        x = legendre_roots(s)
        c = [(1 + xi) / 2 for xi in x]
        # sum_j b_j c_j^(k-1) = 1/k
        vand = [[c[j] ** (k - 1) for j in range(s)] for k in range(1, s + 1)]
        b = _solve(vand, [Decimal(1) / k for k in range(1, s + 1)])
        # sum_j a_ij c_j^(k-1) = c_i^k / k, one system per row i
        a = [_solve(vand, [c[i] ** k / k for k in range(1, s + 1)]) for i in range(s)]
        alpha = [[sum(a[i][k] * a[k][j] for k in range(s)) for j in range(s)] for i in range(s)]
        beta = [sum(b[k] * a[k][i] for k in range(s)) for i in range(s)]
        # sum_j nut_ij (c_j - 1)^(k-1) = c_i^k / k  (extrapolation, Eq. Pol0)
        vand1 = [[(c[j] - 1) ** (k - 1) for j in range(s)] for k in range(1, s + 1)]
        nut = [_solve(vand1, [c[i] ** k / k for k in range(1, s + 1)]) for i in range(s)]
    return {"s": s, "c": c, "b": b, "a": a, "alpha": alpha, "beta": beta, "nut": nut}


@lru_cache(maxsize=None)
def fp64_tables(s: int = 8) -> dict:
    """The machine-number tables used by the FP64 step (Sec. 2.4).

    Returns a dict of Python floats: c[s], b[s], mu[s][s], eta[s][s],
    nu[s][s] (row index i = stage being formed, column j = summed stage).
    """
    ex = exact_tables(s)
    with localcontext() as ctx:
        ctx.prec = DIGITS
        c = [_fl(v) for v in ex["c"]]
        b = [_fl(v) for v in ex["b"]]
        mu = [[0.0] * s for _ in range(s)]
        eta = [[0.0] * s for _ in range(s)]
        nu = [[0.0] * s for _ in range(s)]
        for i in range(s):
            for j in range(i + 1):
                mu[i][j] = _fl(ex["a"][i][j] / ex["b"][j])
                eta[i][j] = _fl(ex["alpha"][i][j] / ex["b"][j])
            for j in range(s):
                nu[i][j] = _fl(ex["nut"][i][j] / ex["b"][j])
    for i in range(s):
        for j in range(i + 1, s):
            # Sec. 2.4: mu_ij = 1 - mu_ji, evaluated in FP64 as printed.
            mu[i][j] = 1.0 - mu[j][i]
            # Eq. sympl_cond_2 solved exactly over the FP64 values.
            exact = Fraction(eta[j][i]) + Fraction(c[i]) - Fraction(c[j])
            eta[i][j] = float(exact)
            if Fraction(eta[i][j]) != exact:
                raise ArithmeticError(
                    f"eta[{i}][{j}] = eta_ji + c_i - c_j is not an FP64 number")
    return {"s": s, "c": c, "b": b, "mu": mu, "eta": eta, "nu": nu}


@lru_cache(maxsize=None)
def decimal_tables(s: int = 8) -> dict:
    """The same keys as fp64_tables() but with the exact (80-digit) values
    mu = a/b, eta = alpha/b, nu = nut/b, for running the generic step in
    high precision (order checks).  These satisfy mu_ij + mu_ji = 1 and
    Eq. sympl_cond_2 up to the working precision by construction of the
    Gauss coefficients, not by rounding rules."""
    ex = exact_tables(s)
    with localcontext() as ctx:
        ctx.prec = DIGITS
        mu = [[ex["a"][i][j] / ex["b"][j] for j in range(s)] for i in range(s)]
        eta = [[ex["alpha"][i][j] / ex["b"][j] for j in range(s)] for i in range(s)]
        nu = [[ex["nut"][i][j] / ex["b"][j] for j in range(s)] for i in range(s)]
    return {"s": s, "c": list(ex["c"]), "b": list(ex["b"]), "mu": mu, "eta": eta, "nu": nu}


def hexdump(tables: dict) -> str:
    """Text form (one 'name i j hexfloat' per line) used by tests/golden."""
    lines = []
    s = tables["s"]
    for name in ("c", "b"):
        for i in range(s):
            lines.append(f"{name} {i} - {float.hex(tables[name][i])}")
    for name in ("mu", "eta", "nu"):
        for i in range(s):
            for j in range(s):
                lines.append(f"{name} {i} {j} {float.hex(tables[name][i][j])}")
    return "\n".join(lines) + "\n"


getcontext().prec = max(getcontext().prec, 28)
