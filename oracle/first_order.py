"""IRKGL first-order step (the mu form), generic over the scalar type (oracle side).

Test infrastructure only (see ``oracle/__init__.py``).

The method of arXiv 2511.03655 for y' = f(y) in the exactly-symplectic
floating-point form of Sec. 2.4 (Eq. Yi2), with the fixed-point iteration
of Eqs. IRK_init / IRK_FP and the stopping rule of Eqs. Delta_n / stopping
checked on all D components.  Sequential sums j = 1..s, every operation
rounded separately, as in ``oracle/irkgl.py``.  One step n:

  init (Eq. IRK_init, extrapolation Eq. Pol0)
      Y_i   = y + sum_j nu_ij Lprev_j
  sweep k = 1, 2, ... (Eq. IRK_FP)
      F_i   = f(Y_i)
      L_i   = h (b_i F_i)
      Yn_i  = y + sum_j mu_ij L_j                       (Eq. Yi2)
      Delta_l = max_i |Yn_il - Y_il|, l = 1..D          (Eq. Delta_n)
      stop by Eq. stopping on every l; Y = Yn
  update (Eq. yn2) with the L of the last sweep
      y_n = y + sum_i L_i, compensated (Sec. 5: TwoSum + Fast2Sum pair)

Readings, as for the second-order form: Lprev = 0 on the first step; the
update uses the L of the last sweep; kmax = 100 -> status MAXITER; a
non-finite stage value -> status NONFINITE, the state left as it was at the
start of the step; stages see only the hi parts of y.

Right-hand sides (autonomous):
  Schwarzschild  charged particle near a Schwarzschild black hole in a
                 magnetic field, Eq. Ham_SBH, y = (r, theta, p_r, p_theta),
                 f = (dH/dp_r, dH/dp_theta, -dH/dr, -dH/dtheta), the
                 derivatives written out by hand (pinned against
                 high-precision finite differences of H in the tests).
  Harmonic1      q' = p, p' = -omega^2 q as a first-order system (D = 2).
"""
from __future__ import annotations

import math
from decimal import Decimal

from .irkgl import MAXITER, NONFINITE, OK, KMAX, Dual, _isfinite, stop_test, two_sum_add, value, zero_like
from .irkgl import sin as _sin
from .irkgl import _dec_pi


def sin(x):
    if isinstance(x, Dual):
        return Dual(math.sin(x.val), [math.cos(x.val) * g for g in x.grad])
    return _sin(x)


def cos(x):
    if isinstance(x, Dual):
        return Dual(math.cos(x.val), [-math.sin(x.val) * g for g in x.grad])
    if isinstance(x, float):
        return math.cos(x)
    return _sin(_dec_pi() / 2 - x)


class Schwarzschild:
    """Eq. Ham_SBH with parameters (E, L, beta):
    H = 1/2 (1 - 2/r) p_r^2 - 1/2 (1 - 2/r)^-1 E^2 + p_theta^2 / (2 r^2)
        + (L - beta/2 r^2 sin^2 theta)^2 / (2 r^2 sin^2 theta).
    With u = 1 - 2/r and s = sin^2 theta:
      dH/dp_r     = u p_r
      dH/dp_theta = p_theta / r^2
      dH/dr       = p_r^2 / r^2 + E^2 / (r^2 u^2) - p_theta^2 / r^3
                    - L^2 / (r^3 s) + beta^2 r s / 4
      dH/dtheta   = (-L^2 / (r^2 s^2) + beta^2 r^2 / 4) sin theta cos theta
    """

    D = 2 * 2

    def __init__(self, E=0.995, L=4.6, beta=8.9e-4):
        self.E, self.L, self.beta = E, L, beta

    def f(self, y):
        r, th, pr, pth = y
        sn, cs = sin(th), cos(th)
        s = sn * sn
        u = 1 - 2 / r
        r2 = r * r
        r3 = r2 * r
        E2, L2, b2 = self.E * self.E, self.L * self.L, self.beta * self.beta
        dr = pr * pr / r2 + E2 / (r2 * (u * u)) - pth * pth / r3 - L2 / (r3 * s) + b2 * r * s / 4
        dth = (-L2 / (r2 * (s * s)) + b2 * r2 / 4) * (sn * cs)
        return [u * pr, pth / r2, -dr, -dth]

    def H(self, y):
        r, th, pr, pth = y
        sn = sin(th)
        s = sn * sn
        u = 1 - 2 / r
        a = self.L - self.beta / 2 * (r * r) * s
        return (u * (pr * pr) / 2 - self.E * self.E / (2 * u) + pth * pth / (2 * (r * r))
                + a * a / (2 * (r * r) * s))


class Harmonic1:
    """q' = p, p' = -omega^2 q (D = 2), H = (p^2 + omega^2 q^2)/2."""

    D = 2

    def __init__(self, omega=1.0):
        self.omega = omega

    def f(self, y):
        return [y[1], -(self.omega * self.omega * y[0])]

    def H(self, y):
        return (y[1] * y[1] + self.omega * self.omega * y[0] * y[0]) / 2


class State1:
    """Compensated state y (hi, lo) and the previous step's L."""

    def __init__(self, y, y_lo=None, l_prev=None, s=8):
        D = len(y)
        zero = zero_like(y[0])
        self.y = list(y)
        self.y_lo = list(y_lo) if y_lo is not None else [zero] * D
        self.l_prev = [list(r) for r in l_prev] if l_prev is not None else [[zero] * D for _ in range(s)]

    def copy(self):
        return State1(self.y, self.y_lo, self.l_prev, len(self.l_prev))


def step1(state: State1, h, tab: dict, rhs, kmax: int = KMAX, diag: dict | None = None):
    """One first-order step of size h; returns (new_state, k, status)."""
    b, mu, nu = tab["b"], tab["mu"], tab["nu"]
    s = len(b)
    y = state.y
    D = len(y)
    lp = state.l_prev
    # init, Eq. IRK_init
    Y = []
    for i in range(s):
        row = []
        for l in range(D):
            acc = nu[i][0] * lp[0][l]
            for j in range(1, s):
                acc = acc + nu[i][j] * lp[j][l]
            row.append(y[l] + acc)
        Y.append(row)
    if diag is not None:
        diag["Y0"] = [list(r) for r in Y]
    inf = float("inf")
    dmin = [inf] * D
    dprev = [inf] * D
    k = 0
    while True:
        k += 1
        F = [rhs.f(Y[i]) for i in range(s)]
        L = [[h * (b[i] * F[i][l]) for l in range(D)] for i in range(s)]
        Yn = []
        for i in range(s):
            row = []
            for l in range(D):
                acc = mu[i][0] * L[0][l]
                for j in range(1, s):
                    acc = acc + mu[i][j] * L[j][l]
                row.append(y[l] + acc)
            Yn.append(row)
        if not all(_isfinite(Yn[i][l]) for i in range(s) for l in range(D)):
            return state.copy(), k, NONFINITE
        stop = True
        for l in range(D):
            delta = 0.0
            for i in range(s):
                a = abs(value(Yn[i][l]) - value(Y[i][l]))
                if a > delta:
                    delta = a
            cond, dmin[l], dprev[l] = stop_test(delta, dmin[l], dprev[l])
            stop = stop and cond
        Y = Yn
        if diag is not None:
            diag["Y"] = Y
        if stop:
            break
        if k >= kmax:
            return state.copy(), k, MAXITER
    # update, Eq. yn2, compensated
    new = State1(state.y, state.y_lo, L, s)
    for l in range(D):
        sL = L[0][l]
        for i in range(1, s):
            sL = sL + L[i][l]
        new.y[l], new.y_lo[l] = two_sum_add(state.y[l], state.y_lo[l], sL)
    return new, k, OK


def integrate1(y0, h, nsteps, tab, rhs, kmax=KMAX):
    """nsteps first-order steps from y0 (Lprev = 0); final state, per-step
    sweep counts, status, steps completed and max_n |(H_n - H_0)/H_0|."""
    st = State1(y0, s=len(tab["b"]))
    H0 = rhs.H(st.y)
    dmax = 0.0
    iters = []
    status = OK
    n = 0
    for n in range(1, nsteps + 1):
        st2, k, status = step1(st, h, tab, rhs, kmax)
        iters.append(k)
        if status != OK:
            n -= 1
            break
        st = st2
        dH = abs(value((rhs.H(st.y) - H0) / H0))
        if dH > dmax:
            dmax = dH
    return {"state": st, "iters": iters, "status": status, "steps": n, "dH_max": dmax}


def schwarzschild_ic(r0, E=0.995, L=4.6, beta=8.9e-4):
    """theta = pi/2, p_r = 0 and p_theta > 0 from H = -1/2 (Sec. 5.1), as a
    list of floats or of Decimals (the type of r0); None if no such
    p_theta exists at r0."""
    one = type(r0)(1)
    half_pi = (math.pi / 2) if isinstance(r0, float) else _dec_pi() / 2
    u = one - 2 / r0
    a = L - beta / 2 * r0 * r0
    rest = -E * E / (2 * u) + a * a / (2 * r0 * r0)
    p2 = 2 * r0 * r0 * (-one / 2 - rest)
    if p2 <= 0:
        return None
    pth = p2.sqrt() if isinstance(p2, Decimal) else math.sqrt(p2)
    return [r0, half_pi, zero_like(r0), pth]
