"""Closed-form solutions and high-precision helpers used to pin the oracle.

Independent of both the oracle and the CUDA library: plain textbook
formulas (Kepler's equation, the diagonal Pade approximant of exp) evaluated
in 60-digit ``decimal`` arithmetic.
"""
from __future__ import annotations

from decimal import Decimal, localcontext
from math import factorial

PREC = 60


def dec_pi() -> Decimal:
    """pi by Machin's formula."""
    with localcontext() as ctx:
        ctx.prec = PREC + 10

        def arctan_inv(x):
            x = Decimal(x)
            x2 = x * x
            term = 1 / x
            total = term
            n = 1
            sign = -1
            while True:
                term /= x2
                t = term / (2 * n + 1)
                if t < Decimal(10) ** (-(PREC + 8)):
                    break
                total += sign * t
                sign = -sign
                n += 1
            return total

        return +(4 * (4 * arctan_inv(5) - arctan_inv(239)))


def dec_sin_cos(x: Decimal):
    """sin and cos by Taylor series after reduction to [-pi, pi]."""
    with localcontext() as ctx:
        ctx.prec = PREC + 10
        pi = dec_pi()
        two_pi = 2 * pi
        x = Decimal(x)
        k = (x / two_pi).to_integral_value()
        x = x - k * two_pi
        s, c = Decimal(0), Decimal(0)
        term = x
        n = 1
        while abs(term) > Decimal(10) ** (-(PREC + 8)):
            s += term
            term = -term * x * x / ((n + 1) * (n + 2))
            n += 2
        term = Decimal(1)
        n = 0
        while abs(term) > Decimal(10) ** (-(PREC + 8)):
            c += term
            term = -term * x * x / ((n + 1) * (n + 2))
            n += 2
        return s, c


def kepler_state(e, t, mu=1, a=1):
    """Exact planar Kepler orbit with the periapsis at t = 0 on the +x axis:
    solve Kepler's equation E - e sin E = n t (n = sqrt(mu/a^3)) by Newton's
    method and return (q, v) as Decimals."""
    with localcontext() as ctx:
        ctx.prec = PREC + 10
        e = Decimal(e)
        a = Decimal(a)
        mu = Decimal(mu)
        n = (mu / a ** 3).sqrt()
        M = n * Decimal(t)
        pi = dec_pi()
        k = (M / (2 * pi)).to_integral_value()
        Mr = M - k * 2 * pi
        E = Mr if e < Decimal("0.8") else pi if Mr > 0 else -pi
        for _ in range(200):
            s, c = dec_sin_cos(E)
            f = E - e * s - Mr
            dE = f / (1 - e * c)
            E -= dE
            if abs(dE) < Decimal(10) ** (-(PREC + 5)):
                break
        s, c = dec_sin_cos(E)
        b = a * (1 - e * e).sqrt()
        x = a * (c - e)
        y = b * s
        Edot = n / (1 - e * c)
        vx = -a * s * Edot
        vy = b * c * Edot
        return [+x, +y], [+vx, +vy]


def pade_88_harmonic(omega, h):
    """The [8/8] diagonal Pade approximant R(z) = P(z)/P(-z) of exp(z),
    P(z) = sum_k (16-k)! 8! / (16! k! (8-k)!) z^k, evaluated at the matrix
    z = h A with A = [[0, 1], [-omega^2, 0]] (q' = v, v' = -omega^2 q).
    This is the stability function of the 8-stage Gauss method, so one
    converged IRKGL16 step maps (q, v) to R(hA) (q, v)."""
    return pade_harmonic(8, omega, h)


def pade_harmonic(s, omega, h):
    """The [s/s] diagonal Pade approximant of exp(z) at z = h A (as above),
    P(z) = sum_k (2s-k)! s! / ((2s)! k! (s-k)!) z^k: the stability function
    of the s-stage Gauss method."""
    with localcontext() as ctx:
        ctx.prec = PREC + 10
        w = Decimal(omega)
        hh = Decimal(h)
        Z = [[Decimal(0), hh], [-w * w * hh, Decimal(0)]]

        def mm(X, Y):
            return [[X[0][0] * Y[0][0] + X[0][1] * Y[1][0], X[0][0] * Y[0][1] + X[0][1] * Y[1][1]],
                    [X[1][0] * Y[0][0] + X[1][1] * Y[1][0], X[1][0] * Y[0][1] + X[1][1] * Y[1][1]]]

        coef = [Decimal(factorial(2 * s - k) * factorial(s)) /
                Decimal(factorial(2 * s) * factorial(k) * factorial(s - k)) for k in range(s + 1)]
        P = [[Decimal(0)] * 2 for _ in range(2)]
        Pm = [[Decimal(0)] * 2 for _ in range(2)]
        Zk = [[Decimal(1), Decimal(0)], [Decimal(0), Decimal(1)]]
        for k in range(s + 1):
            sgn = 1 if k % 2 == 0 else -1
            for r in range(2):
                for cc in range(2):
                    P[r][cc] += coef[k] * Zk[r][cc]
                    Pm[r][cc] += sgn * coef[k] * Zk[r][cc]
            Zk = mm(Zk, Z)
        det = Pm[0][0] * Pm[1][1] - Pm[0][1] * Pm[1][0]
        inv = [[Pm[1][1] / det, -Pm[0][1] / det], [-Pm[1][0] / det, Pm[0][0] / det]]
        return mm(P, inv)
