"""Python binding of libirkgl.so (include/irkgl.h): argument marshalling only.

Every step of the integration runs in the library's CUDA kernels; this
module only turns torch tensors (device memory, streams) into the plain
pointers and sizes of the C-ABI.  It raises if the library is not built or
cannot be loaded: there is no CPU fallback.

The functions below keep the C names (``irkgl_create``, ``irkgl_step``,
``irkgl_integrate``, ...); ``Integrator`` is a small convenience wrapper.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

OK = 0
ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_UNSUPPORTED = -1, -2, -3, -4
STATUS_OK, STATUS_MAXITER, STATUS_NONFINITE = 0, 1, 2
RHS_KEPLER, RHS_NBODY, RHS_FPUT, RHS_HENON_HEILES, RHS_HARMONIC = 1, 2, 3, 4, 5
RHS_HENON_HEILES_FORCED = 6  # g(t, q): lambda + xi sin t (params = [lambda, xi])
RHS_SCHWARZSCHILD, RHS_HARMONIC1 = 7, 8  # first-order kinds (dim = D): the irkgl_*1 calls
OPT_LANES_PER_TRAJ, OPT_KMAX, OPT_MONITOR_EVERY, OPT_BLOCK_THREADS, OPT_GRID_BLOCKS = 1, 2, 3, 4, 5
OPT_WIDE_TEAM = 6
OPT_MONITOR_LOCAL = 7
OPT_STAGES = 9
OPT_TILE_LAYOUT = 10  # 0 auto, 1 stage split, 2 component split (d = 2 kinds)
SPLIT_STRANG, SPLIT_SUZ90 = 1, 2
OPT_MIX = 8

EXPORTS = ("irkgl_default_coeffs", "irkgl_create", "irkgl_set_option", "irkgl_step",
           "irkgl_integrate", "irkgl_integrate_host", "irkgl_destroy", "irkgl_strerror",
           "irkgl_last_cuda_error", "irkgl_get_tile", "irkgl_probe_fp64_fma",
           "irkgl_integrate_noalloc", "irkgl_integrate_ragged", "irkgl_advance",
           "irkgl_advance_multi", "irkgl_advance_ragged", "irkgl_diag_fixed_mix",
           "irkgl_diag_fixed_mix_rows", "irkgl_diag_rinv", "irkgl_diag_sincos")
NOALLOC_MAX_PARAMS = 63

_P = ctypes.c_void_p


class IrkglError(RuntimeError):
    pass


class irkgl_rhs(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("params", ctypes.POINTER(ctypes.c_double)),
                ("nparams", ctypes.c_int)]


class irkgl_coeffs(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double * 8), ("b", ctypes.c_double * 8),
                ("mu", ctypes.c_double * 64), ("eta", ctypes.c_double * 64),
                ("nu", ctypes.c_double * 64)]


class irkgl_instance(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("dim", ctypes.c_int), ("offset", ctypes.c_longlong),
                ("param_offset", ctypes.c_int), ("nparams", ctypes.c_int), ("h", ctypes.c_double),
                ("nsteps", ctypes.c_longlong)]


class irkgl_outputs(ctypes.Structure):
    _fields_ = [("q", _P), ("v", _P), ("q_lo", _P), ("v_lo", _P), ("r_prev", _P),
                ("dH_max", _P), ("iters", _P), ("steps", _P), ("status", _P)]


class irkgl_outputs1(ctypes.Structure):
    _fields_ = [("y", _P), ("y_lo", _P), ("l_prev", _P), ("dH_max", _P), ("iters", _P),
                ("steps", _P), ("status", _P)]


_lib = None


def load(path: str | None = None, build_if_missing: bool = False):
    """Load libirkgl.so (in-tree build).  Raises IrkglError if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build()
        else:
            raise IrkglError(f"{path} is missing: run __graft_entry__.build() or "
                             "python -m paper_2511_03655_gb300.build")
    L = ctypes.CDLL(path)
    L.irkgl_default_coeffs.argtypes = [ctypes.POINTER(irkgl_coeffs)]
    L.irkgl_create.argtypes = [ctypes.POINTER(_P), irkgl_rhs, ctypes.c_int, ctypes.c_double,
                               ctypes.POINTER(irkgl_coeffs)]
    L.irkgl_set_option.argtypes = [_P, ctypes.c_int, ctypes.c_longlong]
    L.irkgl_step.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P]
    L.irkgl_integrate.argtypes = [_P, _P, _P, ctypes.c_int, _P, ctypes.c_longlong, _P, _P,
                                  ctypes.POINTER(irkgl_outputs), _P]
    L.irkgl_integrate_host.argtypes = L.irkgl_integrate.argtypes
    L.irkgl_split_integrate.argtypes = [_P, ctypes.c_int, _P, _P, ctypes.c_int, _P, ctypes.c_longlong, _P,
                                        ctypes.POINTER(irkgl_outputs), _P]
    L.irkgl_integrate1.argtypes = [_P, _P, ctypes.c_int, _P, ctypes.c_longlong, _P, _P,
                                   ctypes.POINTER(irkgl_outputs1), _P]
    L.irkgl_advance1.argtypes = [_P, _P, _P, _P, _P, _P, _P, ctypes.c_int, _P, _P, _P, ctypes.c_int, _P]
    L.irkgl_destroy.argtypes = [_P]
    L.irkgl_destroy.restype = None
    L.irkgl_strerror.argtypes = [ctypes.c_int]
    L.irkgl_strerror.restype = ctypes.c_char_p
    L.irkgl_last_cuda_error.argtypes = []
    L.irkgl_last_cuda_error.restype = ctypes.c_char_p
    L.irkgl_get_tile.argtypes = [_P]
    L.irkgl_get_layout.argtypes = [_P]
    L.irkgl_probe_fp64_fma.argtypes = [_P, ctypes.POINTER(ctypes.c_longlong), _P]
    L.irkgl_advance.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int, _P, _P, _P,
                                ctypes.c_int, _P]
    L.irkgl_advance_t.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int, _P]
    L.irkgl_diag_fixed_mix.argtypes = [_P, _P, ctypes.c_int, _P]
    L.irkgl_diag_fixed_mix_rows.argtypes = [_P, _P, ctypes.c_int, _P]
    L.irkgl_diag_rinv.argtypes = [_P, _P, ctypes.c_int, _P]
    L.irkgl_diag_sincos.argtypes = [_P, _P, ctypes.c_int, _P]
    L.irkgl_advance_ragged.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P, _P,
                                       _P, _P, ctypes.c_int, _P, _P, _P, _P, _P]
    L.irkgl_advance_multi.argtypes = [_P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int, _P, _P,
                                      _P, _P, _P, ctypes.c_int, _P]
    L.irkgl_integrate_ragged.argtypes = [_P, _P, ctypes.c_int, ctypes.c_int, _P, _P, _P, _P,
                                         ctypes.POINTER(irkgl_outputs), _P]
    L.irkgl_integrate_noalloc.argtypes = [irkgl_rhs, ctypes.c_int, ctypes.c_double, _P, _P,
                                          ctypes.c_int, _P, ctypes.c_longlong, _P, _P,
                                          ctypes.POINTER(irkgl_outputs), _P]
    for name in ("irkgl_default_coeffs", "irkgl_create", "irkgl_set_option", "irkgl_step",
                 "irkgl_integrate", "irkgl_integrate_host", "irkgl_get_tile",
                 "irkgl_probe_fp64_fma", "irkgl_integrate_noalloc", "irkgl_integrate_ragged",
                 "irkgl_advance", "irkgl_advance_multi", "irkgl_advance_ragged",
                 "irkgl_diag_fixed_mix", "irkgl_diag_fixed_mix_rows", "irkgl_diag_rinv",
                 "irkgl_diag_sincos"):
        getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc < 0:
        L = load()
        msg = L.irkgl_strerror(rc).decode()
        if rc == ERR_CUDA:
            msg += ": " + L.irkgl_last_cuda_error().decode()
        raise IrkglError(f"libirkgl error {rc}: {msg}")
    return rc


def _ptr(t: torch.Tensor | None, dtype, shape=None, name="array", device=True):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if device and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not device and t.is_cuda:
        raise ValueError(f"{name} must be a host tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return _P(t.data_ptr())


def _stream(stream) -> _P:
    if stream is None:
        stream = torch.cuda.current_stream()
    return _P(stream.cuda_stream)


# ---------------------------------------------------------------- C names
def irkgl_default_coeffs() -> dict:
    c = irkgl_coeffs()
    _check(load().irkgl_default_coeffs(ctypes.byref(c)))
    return {"c": list(c.c), "b": list(c.b),
            "mu": [list(c.mu[i * 8:(i + 1) * 8]) for i in range(8)],
            "eta": [list(c.eta[i * 8:(i + 1) * 8]) for i in range(8)],
            "nu": [list(c.nu[i * 8:(i + 1) * 8]) for i in range(8)]}


def irkgl_create(kind: int, params, dim: int, h: float, coeffs: dict | None = None) -> int:
    L = load()
    arr = (ctypes.c_double * len(params))(*[float(x) for x in params])
    f = irkgl_rhs(kind, ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), len(params))
    ctx = _P()
    cref = None
    if coeffs is not None:
        cref = irkgl_coeffs()
        for i in range(8):
            cref.c[i] = coeffs["c"][i]
            cref.b[i] = coeffs["b"][i]
            for j in range(8):
                cref.mu[i * 8 + j] = coeffs["mu"][i][j]
                cref.eta[i * 8 + j] = coeffs["eta"][i][j]
                cref.nu[i * 8 + j] = coeffs["nu"][i][j]
        cref = ctypes.byref(cref)
    _check(L.irkgl_create(ctypes.byref(ctx), f, dim, float(h), cref))
    return ctx.value


def irkgl_set_option(ctx: int, option: int, value: int):
    _check(load().irkgl_set_option(_P(ctx), option, int(value)))


def irkgl_get_tile(ctx: int) -> int:
    return _check(load().irkgl_get_tile(_P(ctx)))


def irkgl_probe_fp64_fma(scratch: torch.Tensor, stream=None) -> int:
    """Launch the FP64 FMA throughput probe; returns the FMA count issued."""
    n = ctypes.c_longlong(0)
    _check(load().irkgl_probe_fp64_fma(_ptr(scratch, torch.float64, None, "scratch"),
                                       ctypes.byref(n), _stream(stream)))
    return n.value


def irkgl_diag_fixed_mix(R: torch.Tensor, stream=None) -> torch.Tensor:
    """Fixed-point mixing of columns R [n, 8] -> [n, 8, 2] (eta rows, W rows)."""
    n = R.shape[0]
    out = torch.empty((n, 8, 2), dtype=torch.float64, device=R.device)
    _check(load().irkgl_diag_fixed_mix(_ptr(R, torch.float64, (n, 8), "R"),
                                       _ptr(out, torch.float64, (n, 8, 2), "out"), n, _stream(stream)))
    return out


def irkgl_diag_fixed_mix_rows(R: torch.Tensor, stream=None) -> torch.Tensor:
    """The same sums by the runtime-row form (rows spread over lanes)."""
    n = R.shape[0]
    out = torch.empty((n, 8, 2), dtype=torch.float64, device=R.device)
    _check(load().irkgl_diag_fixed_mix_rows(_ptr(R, torch.float64, (n, 8), "R"),
                                            _ptr(out, torch.float64, (n, 8, 2), "out"), n, _stream(stream)))
    return out


def irkgl_diag_rinv(x: torch.Tensor, stream=None) -> torch.Tensor:
    """x^(-3/2), x^(-1/2) and 1/x as the right-hand sides evaluate them: [n] -> [n, 3]."""
    n = x.shape[0]
    out = torch.empty((n, 3), dtype=torch.float64, device=x.device)
    _check(load().irkgl_diag_rinv(_ptr(x, torch.float64, (n,), "x"),
                                  _ptr(out, torch.float64, (n, 3), "out"), n, _stream(stream)))
    return out


def irkgl_diag_sincos(x: torch.Tensor, stream=None) -> torch.Tensor:
    """(sin x, cos x) as the Schwarzschild right-hand side evaluates them: [n] -> [n, 2]."""
    n = x.shape[0]
    out = torch.empty((n, 2), dtype=torch.float64, device=x.device)
    _check(load().irkgl_diag_sincos(_ptr(x, torch.float64, (n,), "x"),
                                    _ptr(out, torch.float64, (n, 2), "out"), n, _stream(stream)))
    return out


def irkgl_destroy(ctx: int):
    load().irkgl_destroy(_P(ctx))


def irkgl_strerror(code: int) -> str:
    return load().irkgl_strerror(code).decode()


def irkgl_step(ctx: int, dim: int, q, v, q_lo=None, v_lo=None, r_prev=None, h=None,
               nsteps: int = 1, iters=None, status=None, stream=None):
    """Advance in place (device tensors): q, v [B, dim]; q_lo, v_lo [B, dim];
    r_prev [B, 8, dim]; h [B]; iters int32 [B, nsteps]; status int32 [B]."""
    B = q.shape[0]
    f64, i32 = torch.float64, torch.int32
    _check(load().irkgl_step(
        _P(ctx), _ptr(q, f64, (B, dim), "q"), _ptr(v, f64, (B, dim), "v"),
        _ptr(q_lo, f64, (B, dim), "q_lo"), _ptr(v_lo, f64, (B, dim), "v_lo"),
        _ptr(r_prev, f64, (B, 8, dim), "r_prev"), _ptr(h, f64, (B,), "h"),
        B, int(nsteps), _ptr(iters, i32, (B, nsteps), "iters"), _ptr(status, i32, (B,), "status"),
        _stream(stream)))


def irkgl_advance(ctx: int, dim: int, q, v, q_lo, v_lo, r_prev, nsteps, h=None, H0=None,
                  h0_init: bool = False, dH_max=None, iters=None, status=None, stream=None):
    """Continue device-resident trajectories by nsteps[b] steps each (int64 [B])."""
    B = q.shape[0]
    f64 = torch.float64
    _check(load().irkgl_advance(
        _P(ctx), _ptr(q, f64, (B, dim), "q"), _ptr(v, f64, (B, dim), "v"),
        _ptr(q_lo, f64, (B, dim), "q_lo"), _ptr(v_lo, f64, (B, dim), "v_lo"),
        _ptr(r_prev, f64, (B, 8, dim), "r_prev"), _ptr(h, f64, (B,), "h"),
        _ptr(nsteps, torch.int64, (B,), "nsteps"), _ptr(H0, f64, (B,), "H0"), int(bool(h0_init)),
        _ptr(dH_max, f64, (B,), "dH_max"), _ptr(iters, torch.int64, (B,), "iters"),
        _ptr(status, torch.int32, (B,), "status"), B, _stream(stream)))


def irkgl_advance_t(ctx: int, dim: int, q, v, q_lo, v_lo, r_prev, t, nsteps, t_lo=None, h=None,
                    iters=None, status=None, stream=None):
    """Continue trajectories of a time-dependent right-hand side by nsteps[b]
    steps each, carrying the time t (float64 [B], and its compensation part
    t_lo) in place."""
    B = q.shape[0]
    f64 = torch.float64
    _check(load().irkgl_advance_t(
        _P(ctx), _ptr(q, f64, (B, dim), "q"), _ptr(v, f64, (B, dim), "v"),
        _ptr(q_lo, f64, (B, dim), "q_lo"), _ptr(v_lo, f64, (B, dim), "v_lo"),
        _ptr(r_prev, f64, (B, 8, dim), "r_prev"), _ptr(t, f64, (B,), "t"),
        _ptr(t_lo, f64, (B,), "t_lo"), _ptr(h, f64, (B,), "h"),
        _ptr(nsteps, torch.int64, (B,), "nsteps"), _ptr(iters, torch.int64, (B,), "iters"),
        _ptr(status, torch.int32, (B,), "status"), B, _stream(stream)))


@dataclass
class Outputs:
    q: torch.Tensor
    v: torch.Tensor
    q_lo: torch.Tensor | None = None
    v_lo: torch.Tensor | None = None
    r_prev: torch.Tensor | None = None
    dH_max: torch.Tensor | None = None
    iters: torch.Tensor | None = None
    steps: torch.Tensor | None = None
    status: torch.Tensor | None = None

    @staticmethod
    def allocate(batch: int, dim: int, device="cuda", full: bool = True, pin: bool = False):
        kw = dict(device=device)
        if pin:
            kw["pin_memory"] = True
        z = lambda shape, dt: torch.empty(shape, dtype=dt, **kw)  # noqa: E731
        o = Outputs(q=z((batch, dim), torch.float64), v=z((batch, dim), torch.float64))
        if full:
            o.q_lo = z((batch, dim), torch.float64)
            o.v_lo = z((batch, dim), torch.float64)
            o.r_prev = z((batch, 8, dim), torch.float64)
            o.dH_max = z((batch,), torch.float64)
            o.iters = z((batch,), torch.int64)
            o.steps = z((batch,), torch.int64)
            o.status = z((batch,), torch.int32)
        return o

    def _struct(self, batch, dim, device=True):
        f64, i64, i32 = torch.float64, torch.int64, torch.int32
        return irkgl_outputs(
            _ptr(self.q, f64, (batch, dim), "out.q", device), _ptr(self.v, f64, (batch, dim), "out.v", device),
            _ptr(self.q_lo, f64, (batch, dim), "out.q_lo", device),
            _ptr(self.v_lo, f64, (batch, dim), "out.v_lo", device),
            _ptr(self.r_prev, f64, (batch, 8, dim), "out.r_prev", device),
            _ptr(self.dH_max, f64, (batch,), "out.dH_max", device),
            _ptr(self.iters, i64, (batch,), "out.iters", device),
            _ptr(self.steps, i64, (batch,), "out.steps", device),
            _ptr(self.status, i32, (batch,), "out.status", device))


def irkgl_integrate(ctx: int, dim: int, q0, v0, out: Outputs, nsteps=None, nsteps_all: int = 0,
                    h=None, order=None, stream=None):
    """Device tensors: q0, v0 [B, dim]; nsteps int64 [B] (or nsteps_all);
    h [B]; order int32 [B]."""
    B = q0.shape[0]
    f64 = torch.float64
    st = out._struct(B, dim)
    _check(load().irkgl_integrate(
        _P(ctx), _ptr(q0, f64, (B, dim), "q0"), _ptr(v0, f64, (B, dim), "v0"), B,
        _ptr(nsteps, torch.int64, (B,), "nsteps"), int(nsteps_all), _ptr(h, f64, (B,), "h"),
        _ptr(order, torch.int32, (B,), "order"), ctypes.byref(st), _stream(stream)))


def irkgl_split_integrate(ctx: int, dim: int, scheme: int, q0, v0, out: Outputs, nsteps=None,
                          nsteps_all: int = 0, h=None, stream=None):
    """Explicit splitting baseline (SPLIT_STRANG / SPLIT_SUZ90) on the context's
    right-hand side; device tensors as in irkgl_integrate; out.iters = g evaluations."""
    B = q0.shape[0]
    f64 = torch.float64
    st = out._struct(B, dim)
    _check(load().irkgl_split_integrate(
        _P(ctx), int(scheme), _ptr(q0, f64, (B, dim), "q0"), _ptr(v0, f64, (B, dim), "v0"), B,
        _ptr(nsteps, torch.int64, (B,), "nsteps"), int(nsteps_all), _ptr(h, f64, (B,), "h"),
        ctypes.byref(st), _stream(stream)))


def irkgl_integrate_host(ctx: int, dim: int, q0, v0, out: Outputs, nsteps=None,
                         nsteps_all: int = 0, h=None, order=None, stream=None):
    """Host (CPU, ideally pinned) tensors; synchronous; copies inside the call."""
    B = q0.shape[0]
    f64 = torch.float64
    st = out._struct(B, dim, device=False)
    _check(load().irkgl_integrate_host(
        _P(ctx), _ptr(q0, f64, (B, dim), "q0", False), _ptr(v0, f64, (B, dim), "v0", False), B,
        _ptr(nsteps, torch.int64, (B,), "nsteps", False), int(nsteps_all),
        _ptr(h, f64, (B,), "h", False), _ptr(order, torch.int32, (B,), "order", False),
        ctypes.byref(st), _stream(stream)))


# irkgl_instance as a numpy record (the C struct's natural alignment, 40 bytes)
INSTANCE_DTYPE = np.dtype({"names": ["kind", "dim", "offset", "param_offset", "nparams", "h", "nsteps"],
                           "formats": [np.int32, np.int32, np.int64, np.int32, np.int32, np.float64,
                                       np.int64],
                           "offsets": [0, 4, 8, 16, 20, 24, 32], "itemsize": 40})


def instances_array(w: dict) -> np.ndarray:
    """A ragged batch description (arrays kind, dim, offset, param_offset,
    nparams, h, nsteps) as irkgl_instance records (numpy, host)."""
    n = len(w["kind"])
    rec = np.zeros(n, dtype=INSTANCE_DTYPE)
    for name in INSTANCE_DTYPE.names:
        rec[name] = np.asarray(w[name])
    return rec


def instances_tensor(w: dict, device) -> torch.Tensor:
    """Pack a ragged batch description (arrays kind, dim, offset, param_offset,
    nparams, h, nsteps) into a device byte tensor of irkgl_instance records."""
    raw = torch.from_numpy(instances_array(w).view(np.uint8).copy())
    if torch.device(device).type == "cuda":
        return raw.pin_memory().to(device, non_blocking=True)
    return raw.to(device)


@dataclass
class RaggedOutputs:
    q: torch.Tensor
    v: torch.Tensor
    q_lo: torch.Tensor | None = None
    v_lo: torch.Tensor | None = None
    r_prev: torch.Tensor | None = None
    dH_max: torch.Tensor | None = None
    iters: torch.Tensor | None = None
    steps: torch.Tensor | None = None
    status: torch.Tensor | None = None

    @staticmethod
    def allocate(total_dim: int, ninst: int, device="cuda"):
        f = dict(dtype=torch.float64, device=device)
        return RaggedOutputs(q=torch.empty(total_dim, **f), v=torch.empty(total_dim, **f),
                             q_lo=torch.empty(total_dim, **f), v_lo=torch.empty(total_dim, **f),
                             r_prev=torch.empty(8 * total_dim, **f),
                             dH_max=torch.empty(ninst, **f),
                             iters=torch.empty(ninst, dtype=torch.int64, device=device),
                             steps=torch.empty(ninst, dtype=torch.int64, device=device),
                             status=torch.empty(ninst, dtype=torch.int32, device=device))

    def _struct(self):
        f64, i64, i32 = torch.float64, torch.int64, torch.int32
        return irkgl_outputs(_ptr(self.q, f64, None, "out.q"), _ptr(self.v, f64, None, "out.v"),
                             _ptr(self.q_lo, f64, None, "out.q_lo"), _ptr(self.v_lo, f64, None, "out.v_lo"),
                             _ptr(self.r_prev, f64, None, "out.r_prev"),
                             _ptr(self.dH_max, f64, None, "out.dH_max"),
                             _ptr(self.iters, i64, None, "out.iters"), _ptr(self.steps, i64, None, "out.steps"),
                             _ptr(self.status, i32, None, "out.status"))


@dataclass
class Outputs1:
    """Outputs of the first-order calls (device tensors, [B, D] / [B])."""
    y: torch.Tensor
    y_lo: torch.Tensor | None = None
    l_prev: torch.Tensor | None = None
    dH_max: torch.Tensor | None = None
    iters: torch.Tensor | None = None
    steps: torch.Tensor | None = None
    status: torch.Tensor | None = None

    @staticmethod
    def allocate(batch: int, D: int, device="cuda", stages: int = 8):
        f = dict(dtype=torch.float64, device=device)
        return Outputs1(y=torch.empty((batch, D), **f), y_lo=torch.empty((batch, D), **f),
                        l_prev=torch.empty((batch, stages, D), **f), dH_max=torch.empty(batch, **f),
                        iters=torch.empty(batch, dtype=torch.int64, device=device),
                        steps=torch.empty(batch, dtype=torch.int64, device=device),
                        status=torch.empty(batch, dtype=torch.int32, device=device))

    def _struct(self, batch, D, stages=8):
        f64, i64, i32 = torch.float64, torch.int64, torch.int32
        return irkgl_outputs1(_ptr(self.y, f64, (batch, D), "out.y"), _ptr(self.y_lo, f64, (batch, D), "out.y_lo"),
                              _ptr(self.l_prev, f64, (batch, stages, D), "out.l_prev"),
                              _ptr(self.dH_max, f64, (batch,), "out.dH_max"),
                              _ptr(self.iters, i64, (batch,), "out.iters"),
                              _ptr(self.steps, i64, (batch,), "out.steps"),
                              _ptr(self.status, i32, (batch,), "out.status"))


def irkgl_integrate1(ctx: int, D: int, y0, out: Outputs1, nsteps=None, nsteps_all: int = 0, h=None,
                     order=None, stream=None, stages: int = 8):
    """First-order kinds: y0 [B, D] device; nsteps int64 [B] (or nsteps_all); h [B]; order int32 [B].
    `stages` is the context's IRKGL_OPT_STAGES (out.l_prev is [B, stages, D])."""
    B = y0.shape[0]
    st = out._struct(B, D, stages)
    _check(load().irkgl_integrate1(
        _P(ctx), _ptr(y0, torch.float64, (B, D), "y0"), B, _ptr(nsteps, torch.int64, (B,), "nsteps"),
        int(nsteps_all), _ptr(h, torch.float64, (B,), "h"), _ptr(order, torch.int32, (B,), "order"),
        ctypes.byref(st), _stream(stream)))


def irkgl_advance1(ctx: int, D: int, y, y_lo, l_prev, nsteps, h=None, H0=None, h0_init: bool = False,
                   dH_max=None, iters=None, status=None, stream=None, stages: int = 8):
    """Continue first-order trajectories in place (y, y_lo [B, D], l_prev [B, stages, D])."""
    B = y.shape[0]
    f64 = torch.float64
    _check(load().irkgl_advance1(
        _P(ctx), _ptr(y, f64, (B, D), "y"), _ptr(y_lo, f64, (B, D), "y_lo"),
        _ptr(l_prev, f64, (B, stages, D), "l_prev"), _ptr(h, f64, (B,), "h"),
        _ptr(nsteps, torch.int64, (B,), "nsteps"), _ptr(H0, f64, (B,), "H0"), int(bool(h0_init)),
        _ptr(dH_max, f64, (B,), "dH_max"), _ptr(iters, torch.int64, (B,), "iters"),
        _ptr(status, torch.int32, (B,), "status"), B, _stream(stream)))


def irkgl_integrate_ragged(ctx: int, inst: torch.Tensor, ninst: int, dmax: int, params, q0, v0,
                           out: RaggedOutputs, order=None, stream=None):
    """Ragged batch (device tensors): inst from instances_tensor(); packed
    params, q0, v0; order int32 [ninst] or None."""
    f64 = torch.float64
    st = out._struct()
    _check(load().irkgl_integrate_ragged(
        _P(ctx), _ptr(inst, torch.uint8, None, "inst"), int(ninst), int(dmax),
        _ptr(params, f64, None, "params"), _ptr(q0, f64, None, "q0"), _ptr(v0, f64, None, "v0"),
        _ptr(order, torch.int32, (ninst,), "order"), ctypes.byref(st), _stream(stream)))


def irkgl_advance_ragged(ctx: int, inst: torch.Tensor, ninst: int, dmax: int, params, q, v, q_lo,
                         v_lo, r_prev, nsteps, H0=None, h0_init: bool = False, dH_max=None,
                         iters=None, status=None, order=None, stream=None):
    """Continue a ragged batch in place (packed device tensors); nsteps int64
    [ninst]; order int32 [ninst] (-1 entries skipped) or None."""
    f64 = torch.float64
    _check(load().irkgl_advance_ragged(
        _P(ctx), _ptr(inst, torch.uint8, None, "inst"), int(ninst), int(dmax),
        _ptr(params, f64, None, "params"), _ptr(q, f64, None, "q"), _ptr(v, f64, None, "v"),
        _ptr(q_lo, f64, None, "q_lo"), _ptr(v_lo, f64, None, "v_lo"),
        _ptr(r_prev, f64, None, "r_prev"), _ptr(nsteps, torch.int64, (ninst,), "nsteps"),
        _ptr(H0, f64, (ninst,), "H0"), int(bool(h0_init)), _ptr(dH_max, f64, (ninst,), "dH_max"),
        _ptr(iters, torch.int64, (ninst,), "iters"), _ptr(status, torch.int32, (ninst,), "status"),
        _ptr(order, torch.int32, (ninst,), "order"), _stream(stream)))


def irkgl_advance_multi(ctx: int, dim: int, q, v, q_lo, v_lo, r_prev, nsteps, h=None, params=None,
                        param_stride: int = 0, order=None, H0=None, dH_max=None, iters=None,
                        status=None, stream=None):
    """Continue trajectories of many requests of one kind and dimension in
    place (device tensors [B, dim], r_prev [B, 8, dim]); params [B, stride]
    per trajectory or None; order int32 [B] (-1 entries skipped) or None; a
    NaN entry of H0 is computed at that trajectory's first step."""
    B = q.shape[0]
    f64 = torch.float64
    P = int(param_stride)
    _check(load().irkgl_advance_multi(
        _P(ctx), _ptr(q, f64, (B, dim), "q"), _ptr(v, f64, (B, dim), "v"),
        _ptr(q_lo, f64, (B, dim), "q_lo"), _ptr(v_lo, f64, (B, dim), "v_lo"),
        _ptr(r_prev, f64, (B, 8, dim), "r_prev"), _ptr(h, f64, (B,), "h"),
        _ptr(nsteps, torch.int64, (B,), "nsteps"),
        _ptr(params, f64, (B, P) if params is not None else None, "params"), P,
        _ptr(order, torch.int32, (B,), "order"), _ptr(H0, f64, (B,), "H0"),
        _ptr(dH_max, f64, (B,), "dH_max"), _ptr(iters, torch.int64, (B,), "iters"),
        _ptr(status, torch.int32, (B,), "status"), B, _stream(stream)))


def irkgl_integrate_noalloc(kind: int, params, dim: int, h: float, q0, v0, out: Outputs,
                            nsteps=None, nsteps_all: int = 0, h_per_traj=None, order=None,
                            stream=None) -> int:
    """Context-free integration that allocates nothing on the device (see
    irkgl.h).  Device tensors as for irkgl_integrate; returns the C code
    (raises on errors other than IRKGL_ERR_INVALID, which is returned so
    callers can see the capacity check)."""
    B = q0.shape[0]
    f64 = torch.float64
    arr = (ctypes.c_double * len(params))(*[float(x) for x in params])
    f = irkgl_rhs(kind, ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), len(params))
    st = out._struct(B, dim)
    rc = load().irkgl_integrate_noalloc(
        f, dim, float(h), _ptr(q0, f64, (B, dim), "q0"), _ptr(v0, f64, (B, dim), "v0"), B,
        _ptr(nsteps, torch.int64, (B,), "nsteps"), int(nsteps_all),
        _ptr(h_per_traj, f64, (B,), "h_per_traj"), _ptr(order, torch.int32, (B,), "order"),
        ctypes.byref(st), _stream(stream))
    if rc != ERR_INVALID:
        _check(rc)
    return rc


class Integrator:
    """Owns one irkgl context (right-hand side, dimension, default step)."""

    def __init__(self, kind: int, params, dim: int, h: float, coeffs: dict | None = None,
                 lanes_per_traj: int = 0, kmax: int = 100, monitor_every: int = 1,
                 block_threads: int = 128, mix: int = 0, stages: int = 8, layout: int = 0):
        self.dim = dim
        self.stages = stages
        self.ctx = irkgl_create(kind, params, dim, h, coeffs)
        self.set(OPT_STAGES, stages)
        self.set(OPT_MIX, mix)
        self.set(OPT_TILE_LAYOUT, layout)
        self.set(OPT_LANES_PER_TRAJ, lanes_per_traj)
        self.set(OPT_KMAX, kmax)
        self.set(OPT_MONITOR_EVERY, monitor_every)
        self.set(OPT_BLOCK_THREADS, block_threads)

    def set(self, option, value):
        irkgl_set_option(self.ctx, option, value)

    @property
    def tile(self) -> int:
        return irkgl_get_tile(self.ctx)

    @property
    def layout(self) -> str:
        """The tile layout calls run: "stage split", "component split", or
        "reproducible" (one thread per trajectory, mix = 2)."""
        return {1: "stage split", 2: "component split",
                3: "reproducible"}[load().irkgl_get_layout(_P(self.ctx))]

    def step(self, *args, **kw):
        return irkgl_step(self.ctx, self.dim, *args, **kw)

    def advance(self, *args, **kw):
        return irkgl_advance(self.ctx, self.dim, *args, **kw)

    def advance_t(self, *args, **kw):
        return irkgl_advance_t(self.ctx, self.dim, *args, **kw)

    def integrate(self, q0, v0, out=None, **kw) -> Outputs:
        out = out or Outputs.allocate(q0.shape[0], self.dim, device=q0.device)
        irkgl_integrate(self.ctx, self.dim, q0, v0, out, **kw)
        return out

    def integrate1(self, y0, out=None, **kw) -> Outputs1:
        out = out or Outputs1.allocate(y0.shape[0], self.dim, device=y0.device, stages=self.stages)
        irkgl_integrate1(self.ctx, self.dim, y0, out, stages=self.stages, **kw)
        return out

    def advance1(self, *args, **kw):
        return irkgl_advance1(self.ctx, self.dim, *args, stages=self.stages, **kw)

    def split_integrate(self, scheme, q0, v0, out=None, **kw) -> Outputs:
        out = out or Outputs.allocate(q0.shape[0], self.dim, device=q0.device)
        irkgl_split_integrate(self.ctx, self.dim, scheme, q0, v0, out, **kw)
        return out

    def integrate_host(self, q0, v0, out=None, **kw) -> Outputs:
        out = out or Outputs.allocate(q0.shape[0], self.dim, device="cpu")
        irkgl_integrate_host(self.ctx, self.dim, q0, v0, out, **kw)
        return out

    def close(self):
        if self.ctx:
            irkgl_destroy(self.ctx)
            self.ctx = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
