"""Planted mistakes: each plausible error in the oracle's tables or update
must make one of the pins fail.  Mutations are applied to copies of the
oracle's FP64 tables on the CPU; nothing here touches the GPU library."""
import copy
import math
import random
from decimal import Decimal, localcontext
from fractions import Fraction

import pytest

from oracle import cbind, coeffs
from oracle import irkgl as P
from tests.closed_forms import pade_88_harmonic

TAB = coeffs.fp64_tables()


def pade_error(tab, wh=0.5):
    q0, v0 = 1.0, 0.3
    R = pade_88_harmonic(1, Decimal(wh))
    r = cbind.run(cbind.HARMONIC, [1.0], [q0], [v0], wh, 1, tab=tab)
    with localcontext() as ctx:
        ctx.prec = 60
        eq = float(R[0][0] * Decimal(q0) + R[0][1] * Decimal(v0))
        ev = float(R[1][0] * Decimal(q0) + R[1][1] * Decimal(v0))
    return max(abs(r["q"][0][0] - eq), abs(r["v"][0][0] - ev))


def guess_ratio(tab, first=False):
    """|Q^[0] - Q| for h and h/2 (FP64 Kepler e = 0.1); the pinned oracle
    gives ratios ~4 (first step) and ~2^10 (later steps)."""
    out = []
    for N in (16, 32):
        st = P.State([0.9, 0.0], [0.0, math.sqrt(1.1 / 0.9)])
        errs = []
        for _ in range(3):
            dg = {}
            st, _, status = P.step(st, 2 * math.pi / N, tab, P.Kepler(1.0), diag=dg)
            errs.append(max(abs(dg["Q0"][i][l] - dg["Q"][i][l]) for i in range(8) for l in range(2)))
        out.append(errs[0] if first else max(errs[1:]))
    return out[0] / out[1]


def mutated(**kw):
    t = copy.deepcopy(TAB)
    for k, f in kw.items():
        t[k] = f(t[k])
    return t


def test_unmutated_baseline():
    assert pade_error(TAB) <= 3e-16
    assert guess_ratio(TAB) > 2 ** 8.5
    assert 3.5 < guess_ratio(TAB, first=True) < 4.5


@pytest.mark.parametrize("name,tab", [
    ("eta printed sign", mutated(eta=lambda e: [[(e[i][j] if j <= i else
                                                  TAB["c"][i] - TAB["c"][j] - e[j][i])
                                                 for j in range(8)] for i in range(8)])),
    ("eta transposed", mutated(eta=lambda e: [[e[j][i] for j in range(8)] for i in range(8)])),
    ("eta one entry off by 1e-12", mutated(eta=lambda e: [[e[i][j] + (1e-12 if (i, j) == (5, 2) else 0.0)
                                                            for j in range(8)] for i in range(8)])),
    ("c reversed", mutated(c=lambda c: c[::-1])),
    ("b scaled", mutated(b=lambda b: [x * (1 + 1e-9) for x in b])),
])
def test_pade_pin_catches(name, tab):
    # the pin in test_oracle_step.py allows 3e-16
    assert pade_error(tab) > 3e-16, name


@pytest.mark.parametrize("name,tab", [
    ("nu transposed", mutated(nu=lambda n: [[n[j][i] for j in range(8)] for i in range(8)])),
    ("nu unscaled by 1/b (nut)", mutated(nu=lambda n: [[n[i][j] * TAB["b"][j] for j in range(8)]
                                                      for i in range(8)])),
    ("nu with (c_i - 1) as printed -> row-constant", mutated(
        nu=lambda n: [[sum(n[i]) / 8 for _ in range(8)] for i in range(8)])),
])
def test_guess_pin_catches_nu(name, tab):
    assert guess_ratio(tab) < 2 ** 7, name


def test_guess_pin_catches_mu():
    tab = mutated(mu=lambda m: [[m[j][i] for j in range(8)] for i in range(8)])
    assert not (3.5 < guess_ratio(tab, first=True) < 4.5)


def test_two_sum_add_is_error_free():
    """The compensated update (Sec. 5): (hi, lo) + x loses at most one rounding
    of the small lo part, and the result is normalised (|lo| <= ulp(hi)/2)."""
    rnd = random.Random(7)
    for _ in range(20000):
        hi = rnd.uniform(-4, 4)
        lo = math.ulp(hi) * rnd.uniform(-0.5, 0.5)
        x = rnd.uniform(-1, 1) * 10 ** rnd.uniform(-8, 0)
        h2, l2 = P.two_sum_add(hi, lo, x)
        exact = Fraction(hi) + Fraction(lo) + Fraction(x)
        got = Fraction(h2) + Fraction(l2)
        assert abs(got - exact) <= Fraction(abs(h2)) * Fraction(1, 2 ** 100)
        assert abs(l2) <= math.ulp(h2) / 2


def test_compensation_matters_over_long_runs():
    """Dropping the compensation (lo kept at 0) is visible as a larger energy
    error on a long harmonic run; the pinned update keeps it near roundoff."""
    h, n = 2 * math.pi / 4000, 400000
    r = cbind.run(cbind.HARMONIC, [1.0], [1.0], [0.0], h, n)
    comp = r["dH_max"][0]
    st = P.State([1.0], [0.0])
    # plain (uncompensated) variant: reuse the step but reset lo every step
    worst = 0.0
    for _ in range(20000):
        st, _, _ = P.step(st, h, TAB, P.Harmonic(1.0, 1))
        st.q_lo, st.v_lo = [0.0], [0.0]
        Hn = (st.v[0] ** 2 + st.q[0] ** 2) / 2
        worst = max(worst, abs(Hn - 0.5) / 0.5)
    assert comp <= 1e-15          # 400,000 compensated steps
    assert worst >= 1e-14         # 20,000 uncompensated steps already drift


# ---------------------------------------------------------------- right-hand sides
# Planted mistakes in the N-body (Eq. Ham2) and FPUT right-hand sides; each
# must fail one of the pins of tests/test_oracle_rhs.py, none of which takes
# its expected values from the oracle.
from tests import test_oracle_rhs as RP  # noqa: E402


class NBodyMassSwap(P.NBody):
    """g_a weighted by m_a instead of m_b."""

    def g(self, q):
        out = []
        for a in range(self.n):
            acc = [P.zero_like(q[0])] * 3
            for b in range(self.n):
                if b != a:
                    dx = [q[3 * b + k] - q[3 * a + k] for k in range(3)]
                    r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]
                    w = (self.G * self.m[a]) / (r2 * P.sqrt(r2))
                    acc = [acc[k] + w * dx[k] for k in range(3)]
            out.extend(acc)
        return out


class NBodyCubeLaw(P.NBody):
    """A force falling as 1/r^3, paired with the potential it derives from
    (-G m_a m_b / (2 r^2)): g and H stay consistent."""

    def g(self, q):
        out = []
        for a in range(self.n):
            acc = [P.zero_like(q[0])] * 3
            for b in range(self.n):
                if b != a:
                    dx = [q[3 * b + k] - q[3 * a + k] for k in range(3)]
                    r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]
                    w = (self.G * self.m[b]) / (r2 * r2)
                    acc = [acc[k] + w * dx[k] for k in range(3)]
            out.extend(acc)
        return out

    def H(self, q, v):
        kin = sum((self.m[a] * (v[3 * a] ** 2 + v[3 * a + 1] ** 2 + v[3 * a + 2] ** 2) / 2
                   for a in range(self.n)), P.zero_like(q[0]))
        pot = P.zero_like(q[0])
        for a in range(self.n):
            for b in range(a + 1, self.n):
                dx = [q[3 * b + k] - q[3 * a + k] for k in range(3)]
                pot = pot + (self.G * self.m[a] * self.m[b]) / (2 * (dx[0] ** 2 + dx[1] ** 2 + dx[2] ** 2))
        return kin - pot


class NBodyDoubleCount(P.NBody):
    """The potential summed over ordered pairs (every pair twice)."""

    def H(self, q, v):
        return P.NBody.H(self, q, v) * 2 - self._kin(q, v)

    def _kin(self, q, v):
        return sum((self.m[a] * (v[3 * a] ** 2 + v[3 * a + 1] ** 2 + v[3 * a + 2] ** 2) / 2
                    for a in range(self.n)), P.zero_like(q[0]))


class NBodyNoZ(P.NBody):
    """The distance in g misses the z component."""

    def g(self, q):
        out = []
        for a in range(self.n):
            acc = [P.zero_like(q[0])] * 3
            for b in range(self.n):
                if b != a:
                    dx = [q[3 * b + k] - q[3 * a + k] for k in range(3)]
                    r2 = dx[0] * dx[0] + dx[1] * dx[1]
                    w = (self.G * self.m[b]) / (r2 * P.sqrt(r2))
                    acc = [acc[k] + w * dx[k] for k in range(3)]
            out.extend(acc)
        return out


class FPUTAlphaSignG(P.FPUT):
    """The cubic force term with the wrong sign in g only."""

    def g(self, q):
        out = []
        for j in range(1, self.d + 1):
            rr, rl = self._bond(q, j), self._bond(q, j - 1)
            out.append((rr - self.alpha * rr * rr) - (rl - self.alpha * rl * rl))
        return out


class FPUTAlphaSignBoth(P.FPUT):
    """-alpha in g and in H: consistent, but not the FPU alpha chain."""

    def __init__(self, n, alpha=0.25):
        super().__init__(n, -alpha)


class FPUTFreeEnd(P.FPUT):
    """The bond to the right wall dropped (a free end), in g and in H."""

    def _bond(self, q, j):
        if j == self.d:
            return P.zero_like(q[0])
        return P.FPUT._bond(self, q, j)


class FPUTBondShift(P.FPUT):
    """g_j formed from the bonds j+1 and j instead of j and j-1."""

    def g(self, q):
        out = []
        for j in range(1, self.d + 1):
            rr = self._bond(q, j + 1) if j + 1 <= self.d else P.zero_like(q[0])
            rl = self._bond(q, j)
            out.append((rr + self.alpha * rr * rr) - (rl + self.alpha * rl * rl))
        return out


def _nbody_pins_fail(cls):
    """True when the planted class fails the gradient pin or one of the two
    closed forms (quarter-period Python runs)."""
    q, v, m = RP.nbody_random_state(3, 1)
    with localcontext() as ctx:
        ctx.prec = 60
        rhs = cls([Decimal(x) for x in m], G=Decimal("1.3"))
    grad = RP.grad_residual(rhs, q, v, [m[a] for a in range(3) for _ in range(3)]) >= 1e-30
    lag = RP.lagrange_error(RP.run_py(cls([float(x) for x in RP.LAGRANGE_M], G=float(RP.LAGRANGE_G))),
                            periods="0.25", steps_per_period=100) > 1e-12
    two = RP.two_body_error(RP.run_py(cls([float(x) for x in RP.TWO_BODY_M], G=float(RP.TWO_BODY_G))),
                            periods="0.25", steps_per_period=100) > 1e-12
    return grad, lag, two


@pytest.mark.parametrize("cls,expect", [
    (NBodyMassSwap, "grad"),
    (NBodyCubeLaw, "closed"),
    (NBodyDoubleCount, "grad"),
    (NBodyNoZ, "grad"),
])
def test_nbody_pins_catch(cls, expect):
    grad, lag, two = _nbody_pins_fail(cls)
    if expect == "grad":
        assert grad, cls.__name__
    else:
        # g and H agree with each other; only the closed forms can tell
        assert not grad and lag and two, cls.__name__


def _fput_pins_fail(cls):
    q, v = RP.fput_random_state(8, 8)
    with localcontext() as ctx:
        ctx.prec = 60
        rhs = cls(8, Decimal("0.25"))
    grad = RP.grad_residual(rhs, q, v, [1.0] * 8) >= 1e-30
    fpu = RP.fpu_equation_residual(rhs, 8, "0.25") >= 1e-55
    modes = RP.normal_mode_error(RP.run_py(cls(8, 0.0)), nsteps=40) > 1e-12
    return grad, fpu, modes


@pytest.mark.parametrize("cls,which", [
    (FPUTAlphaSignG, "grad"),
    (FPUTAlphaSignBoth, "fpu"),
    (FPUTFreeEnd, "modes"),
    (FPUTBondShift, "grad"),
])
def test_fput_pins_catch(cls, which):
    grad, fpu, modes = _fput_pins_fail(cls)
    assert {"grad": grad, "fpu": fpu, "modes": modes}[which], cls.__name__
