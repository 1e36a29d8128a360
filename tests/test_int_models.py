"""Models, in Python integers, of the integer-pipe elementary functions of
the device code (x^(-3/2), x^(-1/2), 1/x, sin and cos), step for step, with
the seeds' FP32 reciprocal (square) roots taken correctly rounded: their
worst errors against high-precision decimals bound the design (the device
seed is within an FP32 ulp, inside the |e| < 2^-21 the series assume).  The
device functions themselves are tested on the GPU against the same decimals
(tests/test_gpu_rinv.py).  Host-only; no oracle and no CUDA."""
import random
import struct
from decimal import Decimal, getcontext

import numpy as np

M64 = (1 << 64) - 1


def dbits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def bdbl(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b & M64))[0]


def fbits(x) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def ulp(x: float) -> float:
    return bdbl(dbits(abs(x)) + 1) - abs(x)


def round_top64(hi: int, biased: int, sign: int = 0) -> float:
    lz = 64 - hi.bit_length()
    mant = (hi << lz) & M64
    m53 = mant >> 11
    bits = ((biased - lz - 1) << 52) + m53
    bits += ((mant >> 10) & 1) & ((1 if mant & 0x3FF else 0) | (m53 & 1))
    return bdbl(bits | (sign << 63))


def seed_rsqrt(x: float):
    bx = dbits(x)
    E = (bx >> 52) & 0x7FF
    X = (bx & ((1 << 52) - 1)) | (1 << 52)
    Eu = E - 1023
    par = Eu & 1
    half = (Eu - par) // 2
    xf = np.float32(struct.unpack("<f", struct.pack("<I", ((127 + par) << 23) | ((bx >> 29) & 0x7FFFFF)))[0])
    yb = fbits(np.float32(1.0) / np.sqrt(xf))
    f = (yb >> 23) - 127 - 23 - half
    return E, X, f, (yb & 0x7FFFFF) | 0x800000


def rinv3_model(x: float) -> float:
    E, X, f, Yf = seed_rsqrt(x)
    Y2 = Yf * Yf
    sh = (1075 - E) - 2 * f - 56
    assert 41 <= sh <= 44
    D = (1 << 56) - ((X * Y2) >> sh)
    Dq = D >> 8
    T = ((3 * D) >> 1) + ((15 * Dq * Dq) >> 43)
    M = ((1 << 56) + T) << 7
    C = (Y2 * Yf) >> 8
    return round_top64((C * M) >> 64, 3 * f + 72 + 1023)


def rinv1_model(x: float) -> float:
    E, X, f, Yf = seed_rsqrt(x)
    sh = (1075 - E) - 2 * f - 56
    D = (1 << 56) - ((X * Yf * Yf) >> sh)
    Dq = D >> 8
    T = (D >> 1) + ((3 * Dq * Dq) >> 43)
    M = ((1 << 56) + T) << 7
    return round_top64(((Yf << 40) * M) >> 64, f + 24 + 1023)


def rcp_model(x: float) -> float:
    bx = dbits(x)
    E = (bx >> 52) & 0x7FF
    X = (bx & ((1 << 52) - 1)) | (1 << 52)
    xf = np.float32(struct.unpack("<f", struct.pack("<I", (127 << 23) | ((bx >> 29) & 0x7FFFFF)))[0])
    yb = fbits(np.float32(1.0) / xf)
    f = (yb >> 23) - 127 - 23 - (E - 1023)
    Yf = (yb & 0x7FFFFF) | 0x800000
    sh = (1075 - E) - f - 56
    assert 19 <= sh <= 20
    D = (1 << 56) - ((X * Yf) >> sh)
    Dq = D >> 8
    T = D + ((Dq * Dq) >> 40)
    M = ((1 << 56) + T) << 7
    return round_top64(((Yf << 40) * M) >> 64, f + 24 + 1023, bx >> 63)


def sincos_model(x: float):
    from paper_2511_03655_gb300 import gen_tables
    two_over_pi, sin_c, cos_c = gen_tables.sincos_tables()
    bx = dbits(x)
    E = (bx >> 52) & 0x7FF
    assert 993 <= E <= 1028
    T = (bx & ((1 << 52) - 1)) | (1 << 52)
    F = (T * two_over_pi) >> (1083 - E)          # t 2^120
    FH, FL = F >> 64, F & M64
    n = (FH + (1 << 55)) >> 56
    fr = ((FH - (n << 56)) << 64) + FL            # (t - n) 2^120, signed
    fneg = fr < 0
    fa = -fr if fneg else fr
    lz = 128 - fa.bit_length()
    m = (fa << lz) >> 64
    ef = 64 - lz - 120
    Z = ((fa >> 56) ** 2) >> 64
    sp, cp = sin_c[-1], cos_c[-1]
    for k in range(len(sin_c) - 2, -1, -1):
        sp = sin_c[k] + ((sp * Z) >> 64)
        cp = cos_c[k] + ((cp * Z) >> 64)
    sr = round_top64((m * sp) >> 64, ef + 2 + 63 + 1023) * (-1 if fneg else 1)
    cr = round_top64(cp, -62 + 63 + 1023)
    q = n & 3
    s, c = (cr, sr) if q & 1 else (sr, cr)
    if q in (1, 2):
        c = -c
    if q >= 2:
        s = -s
    return (-s if bx >> 63 else s), c


def _dec_pi():
    def atan_inv(k):
        t = Decimal(1) / k
        tot, n, sg = t, 1, -1
        while True:
            t /= k * k
            u = t / (2 * n + 1)
            if u < Decimal(10) ** -70:
                return tot
            tot += sg * u
            sg, n = -sg, n + 1
    return 16 * atan_inv(5) - 4 * atan_inv(239)


def _err(got: float, exact: Decimal) -> float:
    return float(abs(Decimal(got) - exact)) / ulp(float(exact))


def test_reciprocal_root_models():
    getcontext().prec = 60
    rng = random.Random(7)
    w3 = w1 = wr = 0.0
    for i in range(20000):
        x = 2.0 ** rng.uniform(-600, 600) * (1 + rng.random())
        d = Decimal(x)
        w3 = max(w3, _err(rinv3_model(x), 1 / (d * d.sqrt())))
        w1 = max(w1, _err(rinv1_model(x), 1 / d.sqrt()))
        xs = x if i % 2 else -x
        wr = max(wr, _err(rcp_model(xs), 1 / Decimal(xs)))
    assert w3 <= 0.7 and w1 <= 0.7 and wr <= 0.65, (w3, w1, wr)


def test_sincos_model():
    getcontext().prec = 70
    pi = _dec_pi()
    rng = random.Random(8)
    worst = 0.0
    xs = [rng.uniform(-63.9, 63.9) for _ in range(3000)] + [k * np.pi / 2 for k in range(1, 40)]
    for x in xs:
        d = Decimal(x)
        d -= (d / (2 * pi)).to_integral_value() * 2 * pi
        es = ec = Decimal(0)
        term, n = d, 1
        while abs(term) > Decimal(10) ** -66:
            es += term
            term = -term * d * d / ((n + 1) * (n + 2))
            n += 2
        term, n = Decimal(1), 0
        while abs(term) > Decimal(10) ** -66:
            ec += term
            term = -term * d * d / ((n + 1) * (n + 2))
            n += 2
        s, c = sincos_model(float(x))
        worst = max(worst, _err(s, es), _err(c, ec))
    assert worst <= 0.51, worst
