"""ctypes binding to the C form of the oracle (``irkgl_oracle.c``).

Test infrastructure only (see ``oracle/__init__.py``).  The shared object is
compiled on demand with the host C compiler, ``-O2 -ffp-contract=off`` and
no fast-math, so every floating-point operation is rounded separately, as in
``oracle/irkgl.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

from . import coeffs

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "irkgl_oracle.c")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "liborc.so")

KEPLER, NBODY, FPUT, HENON_HEILES, HARMONIC, HH_FORCED = 1, 2, 3, 4, 5, 6
SCHWARZSCHILD, HARMONIC1 = 7, 8  # first-order (mu form), D = 4 and 2
DIM1 = {SCHWARZSCHILD: 4, HARMONIC1: 2}
_lock = threading.Lock()
_lib = None


class OrcTab(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double * 8), ("b", ctypes.c_double * 8),
                ("mu", ctypes.c_double * 64), ("eta", ctypes.c_double * 64),
                ("nu", ctypes.c_double * 64)]


def build(force: bool = False) -> str:
    """Compile irkgl_oracle.c into oracle/_build/liborc.so (if stale)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-pthread", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.POINTER
            L.orc_run.restype = ctypes.c_int
            L.orc_run.argtypes = [
                P(OrcTab), ctypes.c_int, P(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                P(ctypes.c_longlong), ctypes.c_int, P(ctypes.c_int), ctypes.c_int,
                P(ctypes.c_longlong), P(ctypes.c_double), P(ctypes.c_int),
                P(ctypes.c_longlong), ctypes.c_int]
            L.orc_run_t.restype = ctypes.c_int
            L.orc_run_t.argtypes = (L.orc_run.argtypes[:11] + [P(ctypes.c_double), P(ctypes.c_double)]
                                    + L.orc_run.argtypes[11:])
            L.orc_run1.restype = ctypes.c_int
            L.orc_run1.argtypes = [
                P(OrcTab), ctypes.c_int, ctypes.c_int, P(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double),
                P(ctypes.c_longlong), ctypes.c_int, P(ctypes.c_int), ctypes.c_int,
                P(ctypes.c_longlong), P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_longlong)]
            L.orc_hamiltonian1.restype = ctypes.c_double
            L.orc_hamiltonian1.argtypes = [ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double)]
            L.orc_split.restype = ctypes.c_int
            L.orc_split.argtypes = [
                P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int, ctypes.c_int, P(ctypes.c_double),
                ctypes.c_int, ctypes.c_int, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_longlong),
                ctypes.c_int, P(ctypes.c_double), P(ctypes.c_int), P(ctypes.c_longlong)]
            L.orc_hamiltonian.restype = ctypes.c_double
            L.orc_hamiltonian.argtypes = [ctypes.c_int, P(ctypes.c_double), ctypes.c_int,
                                          P(ctypes.c_double), P(ctypes.c_double)]
            _lib = L
    return _lib


def table(tab: dict | None = None) -> OrcTab:
    """C table of an s-stage scheme (s <= 8): c, b [s]; mu, eta, nu packed
    row-major with stride s (s = 8: the IRKGL16 layout [i*8+j])."""
    tab = tab or coeffs.fp64_tables()
    s = len(tab["c"])
    t = OrcTab()
    for i in range(s):
        t.c[i] = tab["c"][i]
        t.b[i] = tab["b"][i]
        for j in range(s):
            t.mu[i * s + j] = tab["mu"][i][j]
            t.eta[i * s + j] = tab["eta"][i][j]
            t.nu[i * s + j] = tab["nu"][i][j]
    return t


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def run(kind: int, params, q, v, h, nsteps, *, q_lo=None, v_lo=None, r_prev=None,
        t0=None, t_lo=None, iters_len: int = 0, kmax: int = 100, nthreads: int = 1,
        tab: dict | None = None):
    """Advance a batch with the C oracle.

    q, v: (batch, d) float64.  params: (P,) shared or (batch, P) per
    trajectory.  h: scalar or (batch,).  nsteps: int or (batch,).  t0, t_lo:
    scalar or (batch,) start time as a compensated pair (default 0; read
    only by a time-dependent g).  Returns a dict of numpy arrays: q, v, q_lo,
    v_lo, r_prev (batch, 8, d), t, t_lo, iters (batch, iters_len),
    iters_total, dH_max, status, steps.
    """
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    if q.ndim == 1:
        q, v = q[None, :], v[None, :]
    batch, d = q.shape
    q_lo = (np.zeros_like(q) if q_lo is None
            else np.array(q_lo, dtype=np.float64, order="C", copy=True).reshape(batch, d))
    v_lo = (np.zeros_like(q) if v_lo is None
            else np.array(v_lo, dtype=np.float64, order="C", copy=True).reshape(batch, d))
    r_prev = (np.zeros((batch, 8, d)) if r_prev is None
              else np.array(r_prev, dtype=np.float64, order="C", copy=True).reshape(batch, 8, d))
    params = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    pstride = params.shape[-1] if params.ndim == 2 else 0
    hh = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (batch,)))
    ns = np.ascontiguousarray(np.broadcast_to(np.asarray(nsteps, dtype=np.int64), (batch,)))
    iters = np.zeros((batch, max(iters_len, 1)), dtype=np.int32)
    tot = np.zeros(batch, dtype=np.int64)
    dH = np.zeros(batch, dtype=np.float64)
    st = np.zeros(batch, dtype=np.int32)
    steps = np.zeros(batch, dtype=np.int64)
    th = np.array(np.broadcast_to(np.asarray(0.0 if t0 is None else t0, dtype=np.float64), (batch,)))
    tl = np.array(np.broadcast_to(np.asarray(0.0 if t_lo is None else t_lo, dtype=np.float64), (batch,)))
    t = table(tab)
    rc = lib().orc_run_t(ctypes.byref(t), kind, _ptr(params, ctypes.c_double), pstride, d, batch,
                       _ptr(q, ctypes.c_double), _ptr(v, ctypes.c_double),
                       _ptr(q_lo, ctypes.c_double), _ptr(v_lo, ctypes.c_double),
                       _ptr(r_prev, ctypes.c_double), _ptr(th, ctypes.c_double),
                       _ptr(tl, ctypes.c_double), _ptr(hh, ctypes.c_double),
                       _ptr(ns, ctypes.c_longlong), kmax,
                       _ptr(iters, ctypes.c_int) if iters_len > 0 else None, iters_len,
                       _ptr(tot, ctypes.c_longlong), _ptr(dH, ctypes.c_double),
                       _ptr(st, ctypes.c_int), _ptr(steps, ctypes.c_longlong), nthreads)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return {"q": q, "v": v, "q_lo": q_lo, "v_lo": v_lo, "r_prev": r_prev, "t": th, "t_lo": tl,
            "iters": iters[:, :iters_len], "iters_total": tot, "dH_max": dH,
            "status": st, "steps": steps}


def hamiltonian(kind: int, params, q, v) -> float:
    params = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    q = np.ascontiguousarray(np.asarray(q, dtype=np.float64))
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float64))
    return lib().orc_hamiltonian(kind, _ptr(params, ctypes.c_double), q.shape[-1],
                                 _ptr(q, ctypes.c_double), _ptr(v, ctypes.c_double))


def run1(kind: int, params, y, h, nsteps, *, y_lo=None, l_prev=None, iters_len: int = 0,
         kmax: int = 100, tab: dict | None = None, stages: int = 8):
    """Advance a batch of first-order trajectories with the C oracle
    (SCHWARZSCHILD: y = (r, theta, p_r, p_theta); HARMONIC1: y = (q, p)),
    s-stage scheme (stages = s; tab defaults to coeffs.fp64_tables(s)).
    y: (batch, D).  params: (P,) shared or (batch, P).  Returns y, y_lo,
    l_prev (batch, s, D), iters, iters_total, dH_max, status, steps."""
    D = DIM1[kind]
    tab = tab or coeffs.fp64_tables(stages)
    ns = len(tab["c"])
    y = np.array(y, dtype=np.float64, order="C", copy=True).reshape(-1, D)
    batch = y.shape[0]
    y_lo = (np.zeros_like(y) if y_lo is None
            else np.array(y_lo, dtype=np.float64, order="C", copy=True).reshape(batch, D))
    l_prev = (np.zeros((batch, ns, D)) if l_prev is None
              else np.array(l_prev, dtype=np.float64, order="C", copy=True).reshape(batch, ns, D))
    params = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    pstride = params.shape[-1] if params.ndim == 2 else 0
    hh = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (batch,)))
    nst = np.ascontiguousarray(np.broadcast_to(np.asarray(nsteps, dtype=np.int64), (batch,)))
    iters = np.zeros((batch, max(iters_len, 1)), dtype=np.int32)
    tot = np.zeros(batch, dtype=np.int64)
    dH = np.zeros(batch, dtype=np.float64)
    st = np.zeros(batch, dtype=np.int32)
    steps = np.zeros(batch, dtype=np.int64)
    t = table(tab)
    rc = lib().orc_run1(ctypes.byref(t), ns, kind, _ptr(params, ctypes.c_double), pstride, batch,
                        _ptr(y, ctypes.c_double), _ptr(y_lo, ctypes.c_double),
                        _ptr(l_prev, ctypes.c_double), _ptr(hh, ctypes.c_double),
                        _ptr(nst, ctypes.c_longlong), kmax,
                        _ptr(iters, ctypes.c_int) if iters_len > 0 else None, iters_len,
                        _ptr(tot, ctypes.c_longlong), _ptr(dH, ctypes.c_double),
                        _ptr(st, ctypes.c_int), _ptr(steps, ctypes.c_longlong))
    if rc != 0:
        raise ValueError(f"orc_run1 failed ({rc})")
    return {"y": y, "y_lo": y_lo, "l_prev": l_prev, "iters": iters[:, :iters_len],
            "iters_total": tot, "dH_max": dH, "status": st, "steps": steps}


def hamiltonian1(kind: int, params, y) -> float:
    params = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
    return lib().orc_hamiltonian1(kind, _ptr(params, ctypes.c_double), _ptr(y, ctypes.c_double))


def run_split(scheme: str, kind: int, params, q, v, h, nsteps, *, q_lo=None, v_lo=None, local=False):
    """Explicit splitting baseline (oracle/splitting.py) in C: scheme
    "strang" or "suz90", second-order kinds.  Returns q, v, q_lo, v_lo,
    dH_max, status, steps."""
    from . import splitting
    a, b = splitting.coefficients(scheme)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    q = np.array(q, dtype=np.float64, order="C", copy=True)
    v = np.array(v, dtype=np.float64, order="C", copy=True)
    if q.ndim == 1:
        q, v = q[None, :], v[None, :]
    batch, d = q.shape
    q_lo = np.zeros_like(q) if q_lo is None else np.array(q_lo, dtype=np.float64, order="C", copy=True).reshape(batch, d)
    v_lo = np.zeros_like(q) if v_lo is None else np.array(v_lo, dtype=np.float64, order="C", copy=True).reshape(batch, d)
    params = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    pstride = params.shape[-1] if params.ndim == 2 else 0
    hh = np.ascontiguousarray(np.broadcast_to(np.asarray(h, dtype=np.float64), (batch,)))
    ns = np.ascontiguousarray(np.broadcast_to(np.asarray(nsteps, dtype=np.int64), (batch,)))
    dH = np.zeros(batch)
    st = np.zeros(batch, dtype=np.int32)
    steps = np.zeros(batch, dtype=np.int64)
    rc = lib().orc_split(_ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double), len(b), kind,
                         _ptr(params, ctypes.c_double), pstride, d, batch, _ptr(q, ctypes.c_double),
                         _ptr(v, ctypes.c_double), _ptr(q_lo, ctypes.c_double), _ptr(v_lo, ctypes.c_double),
                         _ptr(hh, ctypes.c_double), _ptr(ns, ctypes.c_longlong), int(bool(local)),
                         _ptr(dH, ctypes.c_double), _ptr(st, ctypes.c_int), _ptr(steps, ctypes.c_longlong))
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return {"q": q, "v": v, "q_lo": q_lo, "v_lo": v_lo, "dH_max": dH, "status": st, "steps": steps}
