"""IRKGL16 second-order step, generic over the scalar type (oracle side).

Test infrastructure only (see ``oracle/__init__.py``).

This is the method of arXiv 2511.03655 for q'' = g(q) written out step by
step, in the paper's notation and order, with sequential sums j = 1..s and
no fused multiply-add (Python floats round every operation).  It works for
any scalar type supporting + - * / and a ``sqrt`` (float, Decimal, Dual),
so the same code drives the FP64 checks, the symplecticity check through
forward-mode derivatives, and the comparisons with the C form in
``irkgl_oracle.c`` (which performs the identical operation sequence).

One step n (s = 8 stages, d position components):

  init (Eq. IRK_init2)
      V_i   = v + sum_j nu_ij Rprev_j          (velocity extrapolation, Eq. Pol0)
      Lq_i  = h (b_i V_i)
      Q_i   = q + sum_j mu_ij Lq_j
  fixed-point sweep k = 1, 2, ... (Eq. IRK_FP2)
      G_i   = g(Q_i)                            (Eq. Gi)
      R_i   = h (b_i G_i)
      Qn_i  = q + h (c_i v + sum_j eta_ij R_j)  (Eq. Qi2)
      Delta_l = max_i |Qn_il - Q_il|            (Eq. Delta_n, positions only)
      stop iff for every l: Delta_l == 0 or
               min(Delta^[1..k-2]) <= min(Delta^[k-1], Delta^[k])   (Eq. stopping)
      Q = Qn
  update (Eq. qnvn2) with the R of the last sweep
      v_n = v + sum_i R_i
      q_n = q + h v_n - h sum_i c_i R_i

Readings where the paper is silent:
  * first step: Rprev = 0;
  * min over an empty set is +inf, so for k <= 2 only Delta == 0 stops;
  * iteration cap kmax = 100 -> status MAXITER; a non-finite Qn -> status
    NONFINITE; on either, the step is abandoned and the state is left as it
    was at the start of the step;
  * the update uses the R of the last sweep (no extra evaluation of g);
  * compensated state (Sec. 5, improved summation): q and v are kept as
    (hi, lo) pairs; an increment x is added with Knuth's TwoSum,
    the rounding error joins lo, and the pair is renormalised with Dekker's
    Fast2Sum.  The position increment is dq = h v_hi + (h v_lo - h sum c_i R_i),
    using the new velocity pair.  Stages and g only see the hi parts.

Parity pins live in tests/test_oracle_*.py (closed-form Kepler, Pade
approximant for the harmonic oscillator, brute-force collocation solve in 60
digits, symmetry, symplecticity via Dual numbers, energy behaviour).
"""
from __future__ import annotations

import math
from decimal import Decimal

S = 8
OK, MAXITER, NONFINITE = 0, 1, 2
KMAX = 100


# --------------------------------------------------------------------------
# scalar helpers
# --------------------------------------------------------------------------
class Dual:
    """Forward-mode dual number: value plus a gradient vector (list)."""

    __slots__ = ("val", "grad")

    def __init__(self, val, grad):
        self.val = float(val)
        self.grad = list(grad)

    @staticmethod
    def _lift(x, n):
        return x if isinstance(x, Dual) else Dual(x, [0.0] * n)

    def __add__(self, o):
        o = Dual._lift(o, len(self.grad))
        return Dual(self.val + o.val, [a + b for a, b in zip(self.grad, o.grad)])

    __radd__ = __add__

    def __sub__(self, o):
        o = Dual._lift(o, len(self.grad))
        return Dual(self.val - o.val, [a - b for a, b in zip(self.grad, o.grad)])

    def __rsub__(self, o):
        return Dual._lift(o, len(self.grad)) - self

    def __mul__(self, o):
        o = Dual._lift(o, len(self.grad))
        return Dual(self.val * o.val,
                    [a * o.val + self.val * b for a, b in zip(self.grad, o.grad)])

    __rmul__ = __mul__

    def __truediv__(self, o):
        o = Dual._lift(o, len(self.grad))
        q = self.val / o.val
        return Dual(q, [(a - q * b) / o.val for a, b in zip(self.grad, o.grad)])

    def __rtruediv__(self, o):
        return Dual._lift(o, len(self.grad)) / self

    def __neg__(self):
        return Dual(-self.val, [-a for a in self.grad])

    def sqrt(self):
        r = math.sqrt(self.val)
        return Dual(r, [a / (2.0 * r) for a in self.grad])


def value(x) -> float:
    """The plain number behind a scalar (the stopping rule uses values)."""
    return x.val if isinstance(x, Dual) else x


def sqrt(x):
    if isinstance(x, float):
        return math.sqrt(x)
    return x.sqrt()


def sin(x):
    """sin of a float (the C library's) or of a Decimal (Taylor series at the
    current context precision, argument reduced by multiples of 2 pi)."""
    if isinstance(x, float):
        return math.sin(x)
    if isinstance(x, Decimal):
        from decimal import getcontext, localcontext
        prec = getcontext().prec
        with localcontext() as ctx:
            ctx.prec = prec + 10
            two_pi = 2 * _dec_pi()
            y = x - two_pi * (x / two_pi).to_integral_value()
            term, acc, k = y, y, 1
            eps = Decimal(10) ** (-(prec + 5))
            while abs(term) > eps:
                term = -term * y * y / ((2 * k) * (2 * k + 1))
                acc += term
                k += 1
        return +acc
    raise TypeError("sin: unsupported scalar type %r" % type(x))


def _dec_pi():
    """pi at the current Decimal precision (Machin's formula)."""
    from decimal import getcontext, localcontext
    prec = getcontext().prec
    with localcontext() as ctx:
        ctx.prec = prec + 10

        def arctan_inv(n):
            x = Decimal(1) / n
            x2 = x * x
            term, acc, k = x, x, 1
            eps = Decimal(10) ** (-(prec + 8))
            while abs(term) > eps:
                term = -term * x2
                acc += term / (2 * k + 1)
                k += 1
            return acc

        pi = 16 * arctan_inv(5) - 4 * arctan_inv(239)
    return +pi


def zero_like(x):
    """An exact zero of the same scalar type as x."""
    if isinstance(x, Dual):
        return Dual(0.0, [0.0] * len(x.grad))
    return type(x)(0)


def _isfinite(x) -> bool:
    x = value(x)
    if isinstance(x, Decimal):
        return x.is_finite()
    return math.isfinite(x)


# --------------------------------------------------------------------------
# right-hand sides g(q) and Hamiltonians (unit masses unless stated)
# --------------------------------------------------------------------------
class Kepler:
    """Planar two-body problem in relative coordinates, GM = mu:
    H = |v|^2/2 - mu/|q|,  g(q) = -mu q / |q|^3 (d = 2)."""

    d = 2

    def __init__(self, mu=1.0):
        self.mu = mu

    def g(self, q):
        r2 = q[0] * q[0] + q[1] * q[1]
        r3 = r2 * sqrt(r2)
        return [-(self.mu * q[0]) / r3, -(self.mu * q[1]) / r3]

    def H(self, q, v):
        r2 = q[0] * q[0] + q[1] * q[1]
        return (v[0] * v[0] + v[1] * v[1]) / 2 - self.mu / sqrt(r2)


class HenonHeiles:
    """Henon-Heiles (Sec. 5.1): H = (p1^2+p2^2)/2 + (q1^2+q2^2)/2
    + lam (q1^2 q2 - q2^3/3); lam = 1 is the classical system.  The
    autonomous case (xi = 0) of the right-hand side printed in Sec. 3."""

    d = 2

    def __init__(self, lam=1.0):
        self.lam = lam

    def g(self, q):
        return [-q[0] - 2 * self.lam * q[0] * q[1],
                -q[1] - self.lam * (q[0] * q[0] - q[1] * q[1])]

    def H(self, q, v):
        return ((v[0] * v[0] + v[1] * v[1]) / 2 + (q[0] * q[0] + q[1] * q[1]) / 2
                + self.lam * (q[0] * q[0] * q[1] - q[1] * q[1] * q[1] / 3))


class HenonHeilesForced:
    """The non-autonomous Henon-Heiles system printed in Sec. 3 (the user
    function example): q1'' = -q1 - 2 (lam + xi sin t) q1 q2,
    q2'' = -q2 - (lam + xi sin t) (q1^2 - q2^2).  xi = 0 gives HenonHeiles.
    g depends on t, so the step evaluates it at the stage times t_n + c_i h
    (Eq. IRK_FP, first line).  H is the Hamiltonian at time t; it is not
    conserved when xi != 0."""

    d = 2
    time_dependent = True

    def __init__(self, lam=1.0, xi=0.0):
        self.lam = lam
        self.xi = xi

    def g(self, q, t):
        aux = self.lam + self.xi * sin(t)
        return [-q[0] - 2 * aux * q[0] * q[1],
                -q[1] - aux * (q[0] * q[0] - q[1] * q[1])]

    def H(self, q, v, t=0.0):
        aux = self.lam + self.xi * sin(t)
        return ((v[0] * v[0] + v[1] * v[1]) / 2 + (q[0] * q[0] + q[1] * q[1]) / 2
                + aux * (q[0] * q[0] * q[1] - q[1] * q[1] * q[1] / 3))


class Harmonic:
    """Uncoupled harmonic oscillators q'' = -omega^2 q (any d)."""

    def __init__(self, omega=1.0, d=1):
        self.omega = omega
        self.d = d

    def g(self, q):
        w2 = self.omega * self.omega
        return [-(w2 * x) for x in q]

    def H(self, q, v):
        w2 = self.omega * self.omega
        acc = zero_like(q[0])
        for x, y in zip(q, v):
            acc = acc + (y * y + w2 * x * x) / 2
        return acc


class NBody:
    """Newtonian N-body problem in 3-D (Eq. Ham2 with G = 1 by default);
    positions q[3a + x]; g_a = G sum_{b != a} m_b (q_b - q_a)/|q_b - q_a|^3.

    Pinned (tests/test_oracle_rhs.py): g = -grad H / m by 60-digit central
    differences; two unequal bodies follow the closed-form Kepler orbit with
    mu = G (m_1 + m_2); Lagrange's equilateral triangle of unequal masses
    rotates rigidly with omega^2 = G M / L^3; total momentum is conserved."""

    def __init__(self, masses, G=1.0):
        self.m = list(masses)
        self.G = G
        self.n = len(self.m)
        self.d = 3 * self.n

    def g(self, q):
        n = self.n
        out = []
        for a in range(n):
            acc = [zero_like(q[0])] * 3
            for b in range(n):
                if b == a:
                    continue
                dx = [q[3 * b + k] - q[3 * a + k] for k in range(3)]
                r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]
                w = (self.G * self.m[b]) / (r2 * sqrt(r2))
                acc = [acc[k] + w * dx[k] for k in range(3)]
            out.extend(acc)
        return out

    def H(self, q, v):
        n = self.n
        kin = zero_like(q[0])
        for a in range(n):
            kin = kin + self.m[a] * (v[3 * a] * v[3 * a] + v[3 * a + 1] * v[3 * a + 1]
                                     + v[3 * a + 2] * v[3 * a + 2]) / 2
        pot = zero_like(q[0])
        for a in range(n):
            for b in range(a + 1, n):
                dx = [q[3 * b + k] - q[3 * a + k] for k in range(3)]
                r = sqrt(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2])
                pot = pot + (self.G * self.m[a] * self.m[b]) / r
        return kin - pot


class FPUT:
    """Fermi-Pasta-Ulam-Tsingou alpha chain with fixed ends q_0 = q_{n+1} = 0:
    H = sum_j v_j^2/2 + sum_{j=0}^{n} V(q_{j+1} - q_j),
    V(r) = r^2/2 + alpha r^3/3, so g_j = V'(r_j) - V'(r_{j-1}),
    r_j = q_{j+1} - q_j, V'(r) = r + alpha r^2.

    Pinned (tests/test_oracle_rhs.py): g = -grad H by 60-digit central
    differences; g equals the Fermi-Pasta-Ulam equation of motion in its
    second-difference form; for alpha = 0 the run follows the chain's
    closed-form normal modes; the energy of a mode-1 run stays bounded."""

    def __init__(self, n, alpha=0.25):
        self.d = n
        self.alpha = alpha

    def _bond(self, q, j):
        # r_j = q_{j+1} - q_j with 0-based particle storage q[0..n-1]
        n = self.d
        left = q[j - 1] if j >= 1 else zero_like(q[0])
        right = q[j] if j <= n - 1 else zero_like(q[0])
        return right - left

    def g(self, q):
        n = self.d
        out = []
        for j in range(1, n + 1):
            r_right = self._bond(q, j)      # q_{j+1} - q_j
            r_left = self._bond(q, j - 1)   # q_j - q_{j-1}
            out.append((r_right + self.alpha * r_right * r_right)
                       - (r_left + self.alpha * r_left * r_left))
        return out

    def H(self, q, v):
        n = self.d
        acc = zero_like(q[0])
        for j in range(n):
            acc = acc + v[j] * v[j] / 2
        for j in range(n + 1):
            r = self._bond(q, j)
            acc = acc + r * r / 2 + self.alpha * r * r * r / 3
        return acc


# --------------------------------------------------------------------------
# compensated addition (Sec. 5: improved summation of the update)
# --------------------------------------------------------------------------
def two_sum_add(hi, lo, x):
    """(hi, lo) + x: Knuth's TwoSum of hi and x, error folded into lo,
    then Dekker's Fast2Sum renormalisation."""
    s = hi + x
    bb = s - hi
    err = (hi - (s - bb)) + (x - bb)
    lo2 = lo + err
    hi2 = s + lo2
    lo3 = lo2 - (hi2 - s)
    return hi2, lo3


# --------------------------------------------------------------------------
# stopping rule, Eq. Delta_n / Eq. stopping
# --------------------------------------------------------------------------
def stop_test(delta, dmin, dprev):
    """One component's share of Eq. stopping at sweep k.

    delta = Delta^[k]; dmin = min(Delta^[1..k-2]) (+inf when empty);
    dprev = Delta^[k-1] (+inf at k = 1).  Returns (cond, dmin', dprev') where
    cond is "Delta^[k] == 0 or min(Delta^[1..k-2]) <= min(Delta^[k-1], Delta^[k])"
    and (dmin', dprev') is the bookkeeping for sweep k + 1.
    """
    cond = (delta == 0) or (dmin <= min(dprev, delta))
    return cond, min(dmin, dprev), delta


# --------------------------------------------------------------------------
# the step
# --------------------------------------------------------------------------
def stage_times(t, h, c):
    """t_n + c_i h for i = 1..s (Eq. IRK_FP, first line), h c_i rounded first."""
    return [t + h * c[i] for i in range(S)]


class State:
    """Trajectory state: compensated positions/velocities and the previous
    step's increments R (used by the extrapolated initial guess)."""

    def __init__(self, q, v, q_lo=None, v_lo=None, r_prev=None, t=None, t_lo=None):
        d = len(q)
        zero = zero_like(q[0])
        self.q = list(q)
        self.v = list(v)
        self.q_lo = list(q_lo) if q_lo is not None else [zero] * d
        self.v_lo = list(v_lo) if v_lo is not None else [zero] * d
        self.r_prev = ([list(r) for r in r_prev] if r_prev is not None
                       else [[zero] * d for _ in range(S)])
        # time t_n as a compensated pair (only read by time-dependent g)
        zt = Decimal(0) if isinstance(value(q[0]), Decimal) else 0.0
        self.t = t if t is not None else zt
        self.t_lo = t_lo if t_lo is not None else zero_like(self.t)

    def copy(self):
        return State(self.q, self.v, self.q_lo, self.v_lo, self.r_prev, self.t, self.t_lo)


def step(state: State, h, tab: dict, rhs, kmax: int = KMAX, diag: dict | None = None):
    """Advance ``state`` by one IRKGL16 step of size h.

    Returns (new_state, k, status).  ``tab`` is ``coeffs.fp64_tables()``
    (or a table of another scalar type with the same keys).  When ``diag`` is
    a dict it receives the initial guess "Q0" and the last stage values "Q".
    """
    c, b, mu, eta, nu = tab["c"], tab["b"], tab["mu"], tab["eta"], tab["nu"]
    q, v = state.q, state.v
    d = len(q)
    rp = state.r_prev

    # --- init, Eq. IRK_init2 ---------------------------------------------
    V = []
    for i in range(S):
        row = []
        for l in range(d):
            acc = nu[i][0] * rp[0][l]
            for j in range(1, S):
                acc = acc + nu[i][j] * rp[j][l]
            row.append(v[l] + acc)
        V.append(row)
    Lq = [[h * (b[i] * V[i][l]) for l in range(d)] for i in range(S)]
    Q = []
    for i in range(S):
        row = []
        for l in range(d):
            acc = mu[i][0] * Lq[0][l]
            for j in range(1, S):
                acc = acc + mu[i][j] * Lq[j][l]
            row.append(q[l] + acc)
        Q.append(row)
    if diag is not None:
        diag["Q0"] = [list(r) for r in Q]

    # stage times t_n + c_i h of a time-dependent g (Eq. IRK_FP, first
    # line): h c_i rounded, then added to the hi part of t_n
    timed = getattr(rhs, "time_dependent", False)
    tau = stage_times(state.t, h, c) if timed else None

    # --- fixed-point sweeps, Eq. IRK_FP2 + stopping rule ------------------
    inf = float("inf")
    dmin = [inf] * d    # min(Delta^[1..k-2])
    dprev = [inf] * d   # Delta^[k-1]
    k = 0
    while True:
        k += 1
        if timed:
            G = [rhs.g(Q[i], tau[i]) for i in range(S)]
        else:
            G = [rhs.g(Q[i]) for i in range(S)]
        R = [[h * (b[i] * G[i][l]) for l in range(d)] for i in range(S)]
        Qn = []
        for i in range(S):
            row = []
            for l in range(d):
                acc = c[i] * v[l]
                for j in range(S):
                    acc = acc + eta[i][j] * R[j][l]
                row.append(q[l] + h * acc)
            Qn.append(row)
        finite = all(_isfinite(Qn[i][l]) for i in range(S) for l in range(d))
        if not finite:
            return state.copy(), k, NONFINITE
        stop = True
        for l in range(d):
            delta = 0.0
            for i in range(S):
                a = abs(value(Qn[i][l]) - value(Q[i][l]))
                if a > delta:
                    delta = a
            cond, dmin[l], dprev[l] = stop_test(delta, dmin[l], dprev[l])
            stop = stop and cond
        Q = Qn
        if diag is not None:
            diag["Q"] = Q
        if stop:
            break
        if k >= kmax:
            return state.copy(), k, MAXITER

    # --- update, Eq. qnvn2 with compensated sums --------------------------
    new = State(state.q, state.v, state.q_lo, state.v_lo, R, state.t, state.t_lo)
    for l in range(d):
        sR = R[0][l]
        for i in range(1, S):
            sR = sR + R[i][l]
        scR = c[0] * R[0][l]
        for i in range(1, S):
            scR = scR + c[i] * R[i][l]
        vh, vl = two_sum_add(state.v[l], state.v_lo[l], sR)
        dq = h * vh + (h * vl - h * scR)
        qh, ql = two_sum_add(state.q[l], state.q_lo[l], dq)
        new.q[l], new.q_lo[l], new.v[l], new.v_lo[l] = qh, ql, vh, vl
    # t_{n+1} = t_n + h, compensated like the state
    new.t, new.t_lo = two_sum_add(state.t, state.t_lo, h)
    return new, k, OK


def integrate(q0, v0, h, nsteps, tab, rhs, kmax=KMAX, record=None, t0=None):
    """Run ``nsteps`` steps from (q0, v0) at time t0 (default 0) with Rprev = 0.

    Returns a dict with the final state, per-step iteration counts, the
    status, steps completed and max_n |(H_n - H_0)/H_0| (Eq. DHglobmax,
    evaluated on the hi parts; 0 for a time-dependent g, whose H is not
    conserved).  ``record`` (a list) receives (q, v) after every step when
    given.
    """
    st = State(q0, v0, t=t0)
    timed = getattr(rhs, "time_dependent", False)
    H0 = None if timed else rhs.H(st.q, st.v)
    dmax = 0.0
    iters = []
    status = OK
    n = 0
    for n in range(1, nsteps + 1):
        st2, k, status = step(st, h, tab, rhs, kmax)
        iters.append(k)
        if status != OK:
            n -= 1
            break
        st = st2
        if not timed:
            Hn = rhs.H(st.q, st.v)
            dH = abs(value((Hn - H0) / H0))
            if dH > dmax:
                dmax = dH
        if record is not None:
            record.append((list(st.q), list(st.v)))
    return {"state": st, "iters": iters, "status": status, "steps": n, "dH_max": dmax}
