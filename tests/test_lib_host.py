"""Host-side checks of libirkgl.so that need no GPU: it builds, loads, exports
every function include/irkgl.h declares, its default tables equal the
oracle's (two independent derivations), and argument validation rejects
bad input before any device work."""
import os
import re
import subprocess

import pytest

from oracle import coeffs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    return irkgl.load()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^(?:int|void|const char\*)\s+(irkgl_\w+)\s*\(", txt, re.M))
    return names


def test_header_declares_the_api():
    names = declared_functions()
    for n in ("irkgl_default_coeffs", "irkgl_create", "irkgl_step", "irkgl_integrate",
              "irkgl_integrate_host", "irkgl_destroy", "irkgl_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2511_03655_gb300 import build
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(irkgl_\w+)", out))
    missing = declared_functions() - exported
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(lib, n)


def test_default_tables_equal_oracle_tables(lib):
    from paper_2511_03655_gb300 import irkgl
    got = irkgl.irkgl_default_coeffs()
    ref = coeffs.fp64_tables()
    for k in ("c", "b", "mu", "eta", "nu"):
        assert got[k] == ref[k], k


def test_generated_header_is_current():
    from paper_2511_03655_gb300 import gen_tables
    assert gen_tables.main(["--check"]) == 0


def test_fused_init_matrix_matches_paper_init():
    """W = A nut diag(1/b) reproduces the two-stage guess of Eq. IRK_init2
    (mu, nu in FP64) to rounding: sum_j mu_ij b_j nu_jk ~ W_ik."""
    from paper_2511_03655_gb300 import gen_tables
    t = gen_tables.tables()
    for i in range(8):
        for k in range(8):
            two_stage = sum(t["mu"][i][j] * t["b"][j] * t["nu"][j][k] for j in range(8))
            assert abs(two_stage - t["W"][i][k]) <= 1e-12 * max(1.0, abs(t["W"][i][k]))


def test_create_rejects_bad_arguments(lib):
    import ctypes

    from paper_2511_03655_gb300 import irkgl
    arr = (ctypes.c_double * 1)(1.0)
    ctx = ctypes.c_void_p()
    f = irkgl.irkgl_rhs(irkgl.RHS_KEPLER, ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), 1)
    # Kepler requires dim == 2, h must be finite and nonzero; rejected before touching CUDA
    assert lib.irkgl_create(ctypes.byref(ctx), f, 3, 0.1, None) == irkgl.ERR_INVALID
    assert lib.irkgl_create(ctypes.byref(ctx), f, 2, 0.0, None) == irkgl.ERR_INVALID
    assert lib.irkgl_create(ctypes.byref(ctx), f, 2, float("nan"), None) == irkgl.ERR_INVALID
    bad = irkgl.irkgl_rhs(99, ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), 1)
    assert lib.irkgl_create(ctypes.byref(ctx), bad, 2, 0.1, None) == irkgl.ERR_INVALID
    assert lib.irkgl_create(None, f, 2, 0.1, None) == irkgl.ERR_INVALID
    assert lib.irkgl_default_coeffs(None) == irkgl.ERR_INVALID
    assert lib.irkgl_set_option(None, 1, 2) == irkgl.ERR_INVALID
    assert irkgl.irkgl_strerror(irkgl.ERR_UNSUPPORTED).startswith("no compiled kernel")


def test_workload_generator_is_deterministic():
    import numpy as np

    from paper_2511_03655_gb300 import workloads
    a = workloads.kepler_ensemble(batch=1000)
    b = workloads.kepler_ensemble(batch=1000)
    assert np.array_equal(a["e"], b["e"])
    assert a["e"].min() >= 0 and a["e"].max() < 0.9
    # splitmix64 reference values (seed 0): first outputs of the published generator
    assert int(workloads.splitmix64(0, 1)[0]) == 0xE220A8397B1DCDAF
    assert np.all(a["nsteps"] == 100 * np.rint(200 + 100 * a["e"]).astype(np.int64))


def test_runtime_row_constants():
    """The row constants of the runtime-row fixed-point form: with a negative
    coefficient applied to the two's complement 2^64 - r' of the operand,
    sum_j n_ij q_j - rbias_i equals sum_j (+-n_ij) r_j mod 2^128, the exact
    scaled sum (and the two-accumulator form's P - N - bias_i), for random
    operands r_j in (-2^61, 2^61), offset r' = r + 2^61."""
    import random

    from paper_2511_03655_gb300 import gen_tables
    it = gen_tables.int_tables(gen_tables.tables())
    M = 1 << 128
    rnd = random.Random(5)
    for name in ("ETA", "W", "MU", "NU"):
        mags, negs, bias, rbias = it[name]
        for _ in range(200):
            r = [rnd.randrange(-(1 << 61) + 1, 1 << 61) for _ in range(8)]
            if _ == 0:
                r = [(1 << 61) - 1, -(1 << 61) + 1] * 4   # extremes
            rp = [x + (1 << gen_tables.R_BIAS) for x in r]
            for i in range(8):
                n = mags[i * 8:(i + 1) * 8]
                s = negs[i * 8:(i + 1) * 8]
                exact = sum((-m if ng else m) * x for m, ng, x in zip(n, s, r))
                assert abs(exact) < (1 << 127)
                acc = sum(m * ((1 << 64) - x if ng else x) for m, ng, x in zip(n, s, rp)) % M
                assert (acc - rbias[i]) % M == exact % M, (name, i)
                pos = sum(m * x for m, ng, x in zip(n, s, rp) if not ng)
                neg = sum(m * x for m, ng, x in zip(n, s, rp) if ng)
                assert (pos - neg - bias[i]) % M == exact % M


def test_sincos_constants():
    """The generated fixed-point sine/cosine constants against the math
    library: 2/pi to 128 bits, and the Taylor polynomials of sin(pi/2 f)/f
    and cos(pi/2 f) in z = f^2 on the quarter period."""
    import math
    from fractions import Fraction

    from paper_2511_03655_gb300 import gen_tables
    two_over_pi, sin_c, cos_c = gen_tables.sincos_tables()
    assert abs(Fraction(two_over_pi, 1 << 128) - Fraction(2 / math.pi)) < Fraction(1, 1 << 52)
    scale = Fraction(1, 1 << gen_tables.SINCOS_SHIFT)
    for f in (0.5, 0.37, -0.21, 1e-3, 2.0 ** -20):
        z = Fraction(f) ** 2
        S = sum(Fraction(c) * scale * z ** k for k, c in enumerate(sin_c))
        C = sum(Fraction(c) * scale * z ** k for k, c in enumerate(cos_c))
        # the library's argument pi/2 f is rounded, hence a few units of 1e-16
        s_ref, c_ref = math.sin(math.pi / 2 * f), math.cos(math.pi / 2 * f)
        assert abs(float(Fraction(f) * S) - s_ref) <= 4e-16 * abs(s_ref)
        assert abs(float(C) - c_ref) <= 4e-16


def test_instance_record_matches_the_c_struct():
    """The numpy record the serving loop packs instance descriptors with has
    the C struct's size and field offsets (irkgl_instance, 40 bytes)."""
    import ctypes

    from paper_2511_03655_gb300 import irkgl
    assert irkgl.INSTANCE_DTYPE.itemsize == ctypes.sizeof(irkgl.irkgl_instance) == 40
    for name, _ in irkgl.irkgl_instance._fields_:
        assert irkgl.INSTANCE_DTYPE.fields[name][1] == getattr(irkgl.irkgl_instance, name).offset
    w = {"kind": [2, 3], "dim": [9, 17], "offset": [0, 9], "param_offset": [0, 4], "nparams": [4, 1],
         "h": [0.01, 0.25], "nsteps": [7, 11]}
    rec = irkgl.instances_array(w)
    arr = (irkgl.irkgl_instance * 2)(*[irkgl.irkgl_instance(*(w[f][k] for f, _ in irkgl.irkgl_instance._fields_))
                                       for k in range(2)])
    assert rec.tobytes() == bytes(arr)
