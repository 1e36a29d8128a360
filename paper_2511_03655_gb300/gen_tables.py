"""Generate csrc/irkgl_tables.h: the FP64 IRKGL16 tables used by the kernels.

    python -m paper_2511_03655_gb300.gen_tables          # rewrite the header
    python -m paper_2511_03655_gb300.gen_tables --check  # verify it is current

Route (arXiv 2511.03655, Sec. 2.2-2.4), in 90-digit ``decimal`` arithmetic:

* Gauss nodes: zeros of the Legendre polynomial P_8, written out from its
  explicit coefficients P_n(x) = 2^-n sum_k (-1)^k C(n,k) C(2n-2k,n) x^(n-2k)
  and refined by Newton's method; c_i = (1 + x_i)/2.
* Collocation coefficients by integrating the Lagrange basis l_j on c:
  b_j = int_0^1 l_j, a_ij = int_0^{c_i} l_j (equivalent to the collocation
  conditions of Sec. 2.2); the extrapolation weights of Eq. Pol0,
  nut_ij = int_1^{1+c_i} l_j.
* alpha = A A (Eq. Qi); eta_ij = fl(alpha_ij / b_j) for j <= i and
  eta_ij = eta_ji + c_i - c_j for i < j, which makes Eq. sympl_cond_2 exact
  over the FP64 numbers (the rule printed in Sec. 2.4 carries the opposite
  sign and would violate Eq. sympl_cond_2); mu_ij = fl(a_ij / b_j) for
  j <= i, mu_ij = 1 - mu_ji for i < j (Eq. Yi2); nu_ij = fl(nut_ij / b_j)
  (Eq. IRK_init2 applies nu to L = h b F).
* W = A nut diag(1/b), rounded once: the initial guess of Eq. IRK_init2,
  Q_i = q + sum_j mu_ij h b_j (v + sum_k nu_jk R_k), equals
  q + h (c_i v + sum_k W_ik R_k) in exact arithmetic, so the kernels form
  it with one 8x8 mixing instead of two.

Every value is rounded once with Python's correctly rounded float().
"""
from __future__ import annotations

import argparse
import os
import sys
from decimal import Decimal, localcontext
from fractions import Fraction
from math import comb

S = 8
SMALL_S = (2, 4, 6)
PREC = 90
HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "csrc", "irkgl_tables.h")


def _legendre_coeffs(n):
    """Monomial coefficients (highest degree first) of P_n, exact rationals."""
    co = [Fraction(0)] * (n + 1)
    for k in range(n // 2 + 1):
        co[2 * k] = Fraction((-1) ** k * comb(n, k) * comb(2 * n - 2 * k, n), 2 ** n)
    return co


def _horner(co, x):
    p = Decimal(0)
    dp = Decimal(0)
    for a in co:
        dp = dp * x + p
        p = p * x + Decimal(a.numerator) / Decimal(a.denominator)
    return p, dp


def gauss_nodes(s: int = S):
    co = _legendre_coeffs(s)
    xs = []
    with localcontext() as ctx:
        ctx.prec = PREC
        for i in range(s):
            # Chebyshev-Gauss points as starting values (distinct, interlaced)
            import math
            x = Decimal(repr(-math.cos(math.pi * (i + 0.5) / s)))
            for _ in range(100):
                p, dp = _horner(co, x)
                step = p / dp
                x -= step
                if abs(step) < Decimal(10) ** (-(PREC - 4)):
                    break
            xs.append(x)
        xs.sort()
        return [(1 + x) / 2 for x in xs]


def _basis_integrals(c, lo, hi):
    """M[i][j] = int_{lo_i}^{hi_i} l_j(u) du."""
    n = len(c)
    out = [[Decimal(0)] * n for _ in range(n)]
    for j in range(n):
        poly = [Decimal(1)]  # lowest degree first
        den = Decimal(1)
        for m in range(n):
            if m == j:
                continue
            nxt = [Decimal(0)] * (len(poly) + 1)
            for p, a in enumerate(poly):
                nxt[p + 1] += a
                nxt[p] -= a * c[m]
            poly = nxt
            den *= c[j] - c[m]
        prim = [Decimal(0)] + [a / (p + 1) for p, a in enumerate(poly)]

        def F(u):
            acc = Decimal(0)
            for a in reversed(prim):
                acc = acc * u + a
            return acc

        for i in range(n):
            out[i][j] = (F(hi[i]) - F(lo[i])) / den
    return out


def tables(S: int = S):
    """FP64 tables of the S-stage method (S = 8: IRKGL16)."""
    with localcontext() as ctx:
        ctx.prec = PREC
        c = gauss_nodes(S)
        zeros = [Decimal(0)] * S
        ones = [Decimal(1)] * S
        b = _basis_integrals(c, zeros, ones)[0]
        A = _basis_integrals(c, zeros, c)
        nut = _basis_integrals(c, ones, [1 + x for x in c])
        alpha = [[sum(A[i][k] * A[k][j] for k in range(S)) for j in range(S)] for i in range(S)]
        W = [[sum(A[i][j] * nut[j][k] for j in range(S)) / b[k] for k in range(S)] for i in range(S)]
        cf = [float(x) for x in c]
        bf = [float(x) for x in b]
        mu = [[0.0] * S for _ in range(S)]
        eta = [[0.0] * S for _ in range(S)]
        for i in range(S):
            for j in range(i + 1):
                mu[i][j] = float(A[i][j] / b[j])
                eta[i][j] = float(alpha[i][j] / b[j])
        nu = [[float(nut[i][j] / b[j]) for j in range(S)] for i in range(S)]
        Wf = [[float(W[i][k]) for k in range(S)] for i in range(S)]
    for i in range(S):
        for j in range(i + 1, S):
            mu[i][j] = 1.0 - mu[j][i]
            e = Fraction(eta[j][i]) + Fraction(cf[i]) - Fraction(cf[j])
            eta[i][j] = float(e)
            assert Fraction(eta[i][j]) == e, "eta upper triangle not representable"
    return {"c": cf, "b": bf, "mu": mu, "eta": eta, "nu": nu, "W": Wf}


def split_tables():
    """Drift/kick weights of symmetric compositions of Strang steps with
    weights gamma (a_1 = gamma_1/2, a_j = (gamma_{j-1} + gamma_j)/2,
    a_{s+1} = gamma_s/2, b_j = gamma_j).  Suzuki's fourth-order weights:
    p = 1/(4 - 4^(1/3)) four times around 1 - 4p."""
    out = {}
    with localcontext() as ctx:
        ctx.prec = PREC
        cube_root_4 = Decimal(4) ** (Decimal(1) / Decimal(3))
        p = Decimal(1) / (Decimal(4) - cube_root_4)
        for name, g in (("STRANG", [Decimal(1)]), ("SUZ90", [p, p, 1 - 4 * p, p, p])):
            a = [g[0] / 2] + [(g[j - 1] + g[j]) / 2 for j in range(1, len(g))] + [g[-1] / 2]
            out[name] = ([float(x) for x in a], [float(x) for x in g])
    return out


ETA_SHIFT = 63   # eta_ij = +-n_ij * 2^-63, n_ij exact (|eta| in [2^-11, 1))
W_SHIFT = 50     # W_ij ~ +-w_ij * 2^-50, w_ij = round(|W_ij| 2^50) (only seeds the guess)
MU_SHIFT = 62    # mu_ij = +-n_ij * 2^-62, n_ij exact (|mu| in [2^-8, 1.09): one bit less than eta)
NU_SHIFT = 47    # nu_ij ~ +-n_ij * 2^-47 rounded (|nu| up to 3.7e4; only seeds the guess)
R_BIAS = 61      # fixed-point R values are offset by 2^61 to make them non-negative


def int_tables(t):
    """Integer forms for the fixed-point mixing: magnitudes, signs and the
    per-row correction sum_j (+-n_ij) 2^R_BIAS that removes the offset.

    rbias is the correction for rows whose signs are only known at run time
    (one stage row per lane): there a negative coefficient multiplies the
    two's complement 2^64 - r'_j of the operand instead of going to a second
    accumulator, which adds n_ij 2^64 per negative entry; rbias_i =
    bias_i + 2^64 sum_{j: eta_ij < 0} n_ij, taken mod 2^128."""
    out = {}
    for name, shift, exact in (("ETA", ETA_SHIFT, True), ("W", W_SHIFT, False),
                               ("MU", MU_SHIFT, True), ("NU", NU_SHIFT, False)):
        mags, negs, bias, rbias = [], [], [], []
        key = {"ETA": "eta", "W": "W", "MU": "mu", "NU": "nu"}[name]
        for i in range(S):
            row_sum = 0
            neg_sum = 0
            for j in range(S):
                x = Fraction(t[key][i][j]) * (1 << shift)
                if exact:
                    assert x.denominator == 1, f"{key} is not on the 2^-{shift} grid"
                    m = abs(x.numerator)
                else:
                    m = abs(round(x))
                assert m < (1 << 63)
                neg = x < 0
                mags.append(m)
                negs.append(1 if neg else 0)
                row_sum += -m if neg else m
                neg_sum += m if neg else 0
            bias.append(row_sum * (1 << R_BIAS))
            rbias.append(row_sum * (1 << R_BIAS) + (neg_sum << 64))
        out[name] = (mags, negs, bias, rbias)
    return out


SINCOS_TERMS = 11   # Taylor terms of sin and cos on a quarter period (last term below 2^-62)
SINCOS_SHIFT = 62   # coefficient scale


def dec_pi() -> Decimal:
    """pi by Machin's formula, pi = 16 atan(1/5) - 4 atan(1/239), to PREC digits."""
    with localcontext() as ctx:
        ctx.prec = PREC + 10

        def atan_inv(k):
            x = Decimal(k)
            term = 1 / x
            total, n, sign = term, 1, -1
            while True:
                term /= x * x
                t = term / (2 * n + 1)
                if t < Decimal(10) ** (-(PREC + 5)):
                    return total
                total += sign * t
                sign, n = -sign, n + 1

        return +(16 * atan_inv(5) - 4 * atan_inv(239))


def sincos_tables():
    """Integer constants of the fixed-point sine and cosine: 2/pi rounded to
    128 bits, and the Taylor coefficients of sin(pi/2 f) / f and cos(pi/2 f)
    in powers of z = f^2, (-1)^k (pi/2)^(2k+1)/(2k+1)! and (-1)^k
    (pi/2)^(2k)/(2k)!, rounded to 2^-62 (|f| <= 1/2, so z <= 1/4 and the
    twelfth term is below 2^-62)."""
    from math import factorial
    with localcontext() as ctx:
        ctx.prec = PREC
        pi = dec_pi()
        two_over_pi = int(((2 / pi) * (Decimal(2) ** 128)).to_integral_value())
        hp = pi / 2
        scale = Decimal(2) ** SINCOS_SHIFT
        sin_c = [int((((-1) ** k) * hp ** (2 * k + 1) / factorial(2 * k + 1) * scale).to_integral_value())
                 for k in range(SINCOS_TERMS)]
        cos_c = [int((((-1) ** k) * hp ** (2 * k) / factorial(2 * k) * scale).to_integral_value())
                 for k in range(SINCOS_TERMS)]
    return two_over_pi, sin_c, cos_c


def _render_sincos() -> str:
    two_over_pi, sin_c, cos_c = sincos_tables()
    m64 = (1 << 64) - 1
    lines = ["", "// Fixed-point sine and cosine (see gen_tables.sincos_tables): 2/pi * 2^128 as",
             "// two 64-bit words; Taylor coefficients of sin(pi/2 f)/f and cos(pi/2 f) in z = f^2,",
             f"// scaled by 2^{SINCOS_SHIFT}, constant term first.",
             f"#define IRKGL_SINCOS_TERMS {SINCOS_TERMS}",
             f"#define IRKGL_TWO_OVER_PI_HI 0x{two_over_pi >> 64:016x}ULL",
             f"#define IRKGL_TWO_OVER_PI_LO 0x{two_over_pi & m64:016x}ULL"]
    for name, co in (("SIN", sin_c), ("COS", cos_c)):
        lines.append(f"__host__ __device__ constexpr long long irkgl_{name.lower()}_coef(int k) {{")
        lines.append(f"  constexpr long long t[{SINCOS_TERMS}] = {{")
        lines.append("    " + ",\n    ".join(f"{x}LL" if x != -(1 << 63) else "(-9223372036854775807LL - 1)"
                                           for x in co).replace("\\n", "\n") + "};")
        lines.append("  return t[k];\n}")
    return "\n".join(lines) + "\n"


def _render_int(t) -> str:
    it = int_tables(t)
    lines = ["", "// Integer forms for the fixed-point mixing (see gen_tables.int_tables):",
             f"// |ETA_ij| * 2^{ETA_SHIFT} (exact), round(|W_ij| * 2^{W_SHIFT}); signs; per-row",
             f"// corrections sum_j (+-m_ij) 2^{R_BIAS} as 128-bit two's complement words;",
             f"// |MU_ij| * 2^{MU_SHIFT} (exact) and round(|NU_ij| * 2^{NU_SHIFT}) for the first-order form.",
             f"#define IRKGL_ETA_SHIFT {ETA_SHIFT}", f"#define IRKGL_W_SHIFT {W_SHIFT}",
             f"#define IRKGL_MU_SHIFT {MU_SHIFT}", f"#define IRKGL_NU_SHIFT {NU_SHIFT}",
             f"#define IRKGL_R_BIAS {R_BIAS}"]
    for name in ("ETA", "W", "MU", "NU"):
        mags, negs, bias, rbias = it[name]
        lines.append(f"__host__ __device__ constexpr unsigned long long irkgl_{name.lower()}_mag(int k) {{")
        lines.append("  constexpr unsigned long long t[64] = {")
        lines.append("    " + ",\n    ".join(", ".join(f"0x{m:016x}ull" for m in mags[r * 8:(r + 1) * 8]) for r in range(8)).replace("\\n", "\n") + "};")
        lines.append("  return t[k];\n}")
        negmask = sum(1 << k for k, v in enumerate(negs) if v)
        lines.append(f"__host__ __device__ constexpr bool irkgl_{name.lower()}_neg(int k) {{ return (0x{negmask:016x}ull >> k) & 1ull; }}")
        for fn, rows in (("bias", bias), ("rbias", rbias)):
            words = []
            for b in rows:
                v = b % (1 << 128)
                words.append([(v >> (32 * w)) & 0xffffffff for w in range(4)])
            lines.append(f"__host__ __device__ constexpr unsigned irkgl_{name.lower()}_{fn}(int i, int w) {{")
            lines.append("  constexpr unsigned t[32] = {")
            lines.append("    " + ",\n    ".join(", ".join(f"0x{x:08x}u" for x in ws) for ws in words).replace("\\n", "\n") + "};")
            lines.append("  return t[i * 4 + w];\n}")
    return "\n".join(lines) + "\n"


def render(t) -> str:
    def arr1(name, v):
        return f"static const double {name}[8] = {{\n  " + ",\n  ".join(float.hex(x) for x in v) + "};\n"

    def arrn(name, v):
        return f"static const double {name}[{len(v)}] = {{\n  " + ",\n  ".join(float.hex(x) for x in v) + "};\n"

    def arr2(name, m):
        rows = ",\n  ".join(", ".join(float.hex(x) for x in row) for row in m)
        return f"static const double {name}[64] = {{\n  {rows}}};\n"

    out = ["/* Generated by paper_2511_03655_gb300/gen_tables.py -- do not edit.",
           " * IRKGL16 FP64 tables (arXiv 2511.03655 Sec. 2.2-2.4), row-major [i*8+j]:",
           " * c, b: nodes and weights; MU (Eq. Yi2); ETA (Eq. Qi2, Eq. sympl_cond_2 exact);",
           " * NU (Eq. Pol0, scaled by 1/b); W = A nut diag(1/b) (fused initial guess). */",
           "#pragma once", ""]
    out.append(arr1("IRKGL_TAB_C", t["c"]))
    out.append(arr1("IRKGL_TAB_B", t["b"]))
    out.append(arr2("IRKGL_TAB_MU", t["mu"]))
    out.append(arr2("IRKGL_TAB_ETA", t["eta"]))
    out.append(arr2("IRKGL_TAB_NU", t["nu"]))
    out.append(arr2("IRKGL_TAB_W", t["W"]))
    out.append("// s-stage variants (s = 2, 4, 6) for the first-order form: c, b [s]; MU, NU")
    out.append("// [s*s], row-major [i*s+j], built by the same route as the 8-stage tables.")
    for ns in SMALL_S:
        ts = tables(ns)
        out.append(arrn(f"IRKGL_TAB{ns}_C", ts["c"]))
        out.append(arrn(f"IRKGL_TAB{ns}_B", ts["b"]))
        out.append(arrn(f"IRKGL_TAB{ns}_MU", [x for row in ts["mu"] for x in row]))
        out.append(arrn(f"IRKGL_TAB{ns}_NU", [x for row in ts["nu"] for x in row]))
    out.append("// Explicit splitting baselines (Sec. 4, Eq. high_order_splitting): drift weights a[s+1],")
    out.append("// kick weights b[s]; Strang (s = 1) and Suzuki's fourth-order composition (s = 5).")
    for name, (a, b) in split_tables().items():
        out.append(arrn(f"IRKGL_SPLIT_{name}_A", a))
        out.append(arrn(f"IRKGL_SPLIT_{name}_B", b))
    return "\n".join(out) + _render_int(t) + _render_sincos()


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--check", action="store_true")
    a = ap.parse_args(argv)
    text = render(tables())
    if a.check:
        with open(HEADER) as f:
            ok = f.read() == text
        print("irkgl_tables.h is", "current" if ok else "STALE")
        return 0 if ok else 1
    with open(HEADER, "w") as f:
        f.write(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
