"""The device reciprocal roots against 50-digit decimal arithmetic.

x^(-3/2) (the force factor of the Kepler and N-body right-hand sides),
x^(-1/2) (the potential) and 1/x (the Schwarzschild terms) are evaluated
without FP64 arithmetic, from an FP32 seed and integer products; sin and cos
of the Schwarzschild right-hand side in fixed point.  All must be within one
unit in the last place over the whole normal range, and the special
operands must give the IEEE limits."""
from decimal import Decimal, getcontext

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    return torch, irkgl


def ulp(x: float) -> float:
    return float(np.spacing(np.float64(abs(x))))


def exact(x: float, p: str) -> Decimal:
    getcontext().prec = 50
    d = Decimal(x)
    return 1 / (d * d.sqrt()) if p == "3" else 1 / d.sqrt()


def test_rinv_normal_range(lib):
    torch, irkgl = lib
    rng = np.random.default_rng(21)
    x = np.concatenate([
        2.0 ** rng.uniform(-60, 60, 20000),        # the physical range
        2.0 ** rng.uniform(-680, 680, 4000),       # the rest of the normal results
        2.0 ** np.arange(-40, 41, dtype=np.float64),  # powers of two (seed boundaries)
        np.nextafter(2.0 ** np.arange(-40, 41, dtype=np.float64), 0.0),
        2.0 ** rng.uniform(-700, -682, 200),       # x^(-3/2) above the range -> Inf / FP64 form
        2.0 ** rng.uniform(682, 700, 200),         # x^(-3/2) subnormal or zero
    ])
    out = irkgl.irkgl_diag_rinv(torch.tensor(x, device="cuda")).cpu().numpy()[:, :2]
    worst3 = worst1 = 0.0
    for xi, y3, y1 in zip(x, out[:, 0], out[:, 1]):
        e3 = exact(float(xi), "3")
        if e3 < Decimal("1.7976931348623157e308"):
            if e3 >= Decimal("2.2250738585072014e-308"):
                worst3 = max(worst3, float(abs(Decimal(float(y3)) - e3)) / ulp(float(e3)))
            else:   # subnormal range: absolute error within one unit of the smallest subnormal
                assert abs(Decimal(float(y3)) - e3) <= Decimal(5e-324), xi
        else:
            assert y3 == np.inf, xi
        e1 = exact(float(xi), "1")
        worst1 = max(worst1, float(abs(Decimal(float(y1)) - e1)) / ulp(float(e1)))
    assert worst3 <= 1.0, worst3
    assert worst1 <= 1.0, worst1


def test_reciprocal(lib):
    torch, irkgl = lib
    rng = np.random.default_rng(22)
    mag = np.concatenate([2.0 ** rng.uniform(-60, 60, 20000), 2.0 ** rng.uniform(-1021, 1021, 4000),
                          2.0 ** np.arange(-40, 41, dtype=np.float64),
                          np.nextafter(2.0 ** np.arange(-40, 41, dtype=np.float64), 0.0),
                          2.0 ** rng.uniform(1022, 1023.9, 100)])   # subnormal results
    x = mag * np.where(rng.uniform(size=mag.size) < 0.5, -1.0, 1.0)
    out = irkgl.irkgl_diag_rinv(torch.tensor(x, device="cuda")).cpu().numpy()[:, 2]
    getcontext().prec = 50
    worst = 0.0
    for xi, y in zip(x, out):
        e = 1 / Decimal(float(xi))
        if abs(e) >= Decimal("2.2250738585072014e-308"):
            worst = max(worst, float(abs(Decimal(float(y)) - e)) / ulp(float(e)))
        else:
            assert abs(Decimal(float(y)) - e) <= Decimal(5e-324), xi
    assert worst <= 1.0, worst
    sp = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 5e-324, -1e-310])
    r = irkgl.irkgl_diag_rinv(torch.tensor(sp, device="cuda")).cpu().numpy()[:, 2]
    assert r[0] == np.inf and r[1] == -np.inf and r[2] == 0.0 and r[3] == 0.0 and np.isnan(r[4])
    assert r[5] == np.inf and r[6] == -np.inf   # 1/x overflows for these subnormals


def test_rinv_special_operands(lib):
    torch, irkgl = lib
    x = np.array([0.0, -0.0, 5e-324, 1e-310, np.inf, -1.0, -np.inf, np.nan])
    out = irkgl.irkgl_diag_rinv(torch.tensor(x, device="cuda")).cpu().numpy()
    r3, r1 = out[:, 0], out[:, 1]
    assert r3[0] == np.inf and r3[1] == np.inf and r3[2] == np.inf and r3[3] == np.inf
    assert r3[4] == 0.0 and np.isnan(r3[5]) and np.isnan(r3[6]) and np.isnan(r3[7])
    assert r1[0] == np.inf and r1[1] == -np.inf and r1[4] == 0.0
    assert np.isnan(r1[5]) and np.isnan(r1[6]) and np.isnan(r1[7])
    for k in (2, 3):   # positive subnormals: finite x^(-1/2), within one ulp
        e = exact(float(x[k]), "1")
        assert float(abs(Decimal(float(r1[k])) - e)) <= ulp(float(e))


def _dec_sin_cos(x: float):
    """sin and cos by Taylor series in 60-digit decimals after reduction by
    2 pi (pi from Machin's formula, computed here)."""
    getcontext().prec = 70

    def atan_inv(k):
        t = Decimal(1) / k
        tot, n, sg = t, 1, -1
        while True:
            t /= k * k
            u = t / (2 * n + 1)
            if u < Decimal(10) ** -68:
                return tot
            tot += sg * u
            sg, n = -sg, n + 1

    pi = 16 * atan_inv(5) - 4 * atan_inv(239)
    d = Decimal(x)
    d -= (d / (2 * pi)).to_integral_value() * 2 * pi
    s = c = Decimal(0)
    term, n = d, 1
    while abs(term) > Decimal(10) ** -66:
        s += term
        term = -term * d * d / ((n + 1) * (n + 2))
        n += 2
    term, n = Decimal(1), 0
    while abs(term) > Decimal(10) ** -66:
        c += term
        term = -term * d * d / ((n + 1) * (n + 2))
        n += 2
    return s, c


def test_fixed_point_sincos(lib):
    """sin and cos of the Schwarzschild right-hand side (fixed-point for
    2^-30 <= |x| < 64, the FP64 sincos elsewhere) within one ulp of the
    60-digit values, including arguments next to multiples of pi/2."""
    torch, irkgl = lib
    rng = np.random.default_rng(23)
    hp = np.pi / 2
    x = np.concatenate([
        rng.uniform(-64, 64, 6000),
        2.0 ** rng.uniform(-30, 6, 2000) * np.where(rng.uniform(size=2000) < 0.5, -1.0, 1.0),
        np.array([k * hp for k in range(1, 40)]),                    # the FP64 multiples of pi/2
        np.nextafter(np.array([k * hp for k in range(1, 40)]), 0.0),
        np.array([1e-12, 3e-10, 100.0, -1e3, 0.0, -0.0]),           # outside: the FP64 sincos
    ])
    out = irkgl.irkgl_diag_sincos(torch.tensor(x, device="cuda")).cpu().numpy()
    worst = 0.0
    for xi, (s, c) in zip(x, out):
        es, ec = _dec_sin_cos(float(xi))
        for got, ex in ((s, es), (c, ec)):
            if ex == 0:
                assert got == 0.0
                continue
            worst = max(worst, float(abs(Decimal(float(got)) - ex)) / ulp(float(ex)))
    assert worst <= 1.0, worst
    sp = irkgl.irkgl_diag_sincos(torch.tensor([np.inf, np.nan], dtype=torch.float64, device="cuda")).cpu().numpy()
    assert np.isnan(sp).all()
