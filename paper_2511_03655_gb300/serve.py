"""Continuous-batching request loop over the IRKGL16 library.

Integration requests (a batch of initial states of one system, a step size
and a horizon) arrive over time.  The server

  * admits a waiting request as soon as its device-memory footprint fits the
    budget (states stay resident on the device until the request finishes);
  * advances every admitted request in chunks of steps: on each tick, a
    request whose previous chunk has completed gets its next chunk launched
    on its own CUDA stream (``irkgl_advance`` for right-hand sides with a
    compiled register kernel, ``irkgl_advance_ragged`` on the wide kernel
    otherwise), so the work of many requests overlaps on the GPU and new
    requests start without waiting for long ones to finish;
  * copies a request's result to the host when its last chunk completes and
    frees its memory.

A chunked run gives the same bits as one uninterrupted launch (the
continuation carries the compensated state, R_prev, H_0 and the running
maxima), so a request's result does not depend on what it was mixed with.

The loop never blocks on the device except when a request finishes: inputs
go up from pinned host buffers with asynchronous copies on the request's
stream, and library contexts (each holds the work counter of one launch in
flight) come from a pool and are destroyed only when the server closes,
since freeing device memory synchronizes the device.

``run_plain`` is the comparator: the plain per-request GPU form, one request
at a time in arrival order, each integrated by one launch.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import irkgl

KIND_IDS = {"kepler": irkgl.RHS_KEPLER, "nbody": irkgl.RHS_NBODY, "fput": irkgl.RHS_FPUT,
            "henon_heiles": irkgl.RHS_HENON_HEILES, "harmonic": irkgl.RHS_HARMONIC}


@dataclass
class Request:
    rid: int
    kind: str
    params: list
    dim: int
    q0: np.ndarray          # [B, d]
    v0: np.ndarray          # [B, d]
    h: float | np.ndarray   # one step, or one per trajectory [B]
    nsteps: int
    arrival: float = 0.0    # seconds after the start of the run
    # filled by the server
    q: np.ndarray | None = None
    v: np.ndarray | None = None
    dH_max: np.ndarray | None = None
    iters: np.ndarray | None = None
    status: np.ndarray | None = None
    t_admit: float = math.nan
    t_done: float = math.nan

    @property
    def batch(self) -> int:
        return self.q0.shape[0]

    @property
    def traj_steps(self) -> int:
        return self.batch * self.nsteps

    def device_bytes(self) -> int:
        B, d = self.batch, self.dim
        return B * d * 8 * (2 + 2 + 8) + B * (8 * 5 + 4) + B * 48


def make_requests(descs: list[dict]) -> list[Request]:
    return [Request(**d) for d in descs]


def register_kernel_available(kind: str, params, dim: int) -> bool:
    """True if the batched register kernel is compiled for (kind, dim)."""
    try:
        ctx = irkgl.irkgl_create(KIND_IDS[kind], params, dim, 0.1)
    except irkgl.IrkglError:
        return False
    try:
        return irkgl.irkgl_get_tile(ctx) > 0
    finally:
        irkgl.irkgl_destroy(ctx)


# Register tiles whose fixed-point form is slower on GB300: the N-body tile
# spreads the stage rows over eight lanes, and the integer chains then cost
# occupancy (measured 3.9e7 vs 4.9e7 trajectory-steps/s on the 6-body ensemble).
FP64_MIX_FASTER = {"nbody"}


def new_context(kind: str, params, dim: int, h: float, mix: int) -> int:
    """A context for the register kernel of (kind, dim): with the fixed-point
    stage mixing when mix = 1, a kernel with it is compiled and it is the
    faster form, else with the FP64 mixing. The choice depends only on
    (kind, dim, mix), so the server and run_plain integrate a request with
    the same kernel."""
    ctx = irkgl.irkgl_create(KIND_IDS[kind], params, dim, h)
    if mix and kind not in FP64_MIX_FASTER:
        irkgl.irkgl_set_option(ctx, irkgl.OPT_MIX, 1)
        if irkgl.irkgl_get_tile(ctx) <= 0:
            irkgl.irkgl_set_option(ctx, irkgl.OPT_MIX, 0)
    return ctx


def new_wide_context(mix: int) -> int:
    """A context for the wide kernel (the kinds come per instance)."""
    ctx = irkgl.irkgl_create(irkgl.RHS_HARMONIC, [1.0], 1, 1.0)
    irkgl.irkgl_set_option(ctx, irkgl.OPT_MIX, 1 if mix else 0)
    return ctx


@dataclass
class _Active:
    req: Request
    stream: torch.cuda.Stream
    ctx: int
    wide: bool
    q: torch.Tensor
    v: torch.Tensor
    qlo: torch.Tensor
    vlo: torch.Tensor
    rp: torch.Tensor
    h: torch.Tensor | None
    H0: torch.Tensor
    dH: torch.Tensor
    it: torch.Tensor
    st: torch.Tensor
    ns: torch.Tensor
    inst: torch.Tensor | None = None
    params_dev: torch.Tensor | None = None
    ckey: tuple = ()
    remaining: int = 0
    started: bool = False
    event: torch.cuda.Event | None = None
    nbytes: int = 0
    chunks: int = 0


@dataclass
class ServeStats:
    latencies: list = field(default_factory=list)
    queueing: list = field(default_factory=list)
    traj_steps: int = 0
    makespan: float = 0.0
    launches: int = 0
    peak_bytes: int = 0
    max_concurrent: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.array([math.nan])
        qd = np.array(self.queueing) if self.queueing else np.array([math.nan])
        return {"requests": len(self.latencies), "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
                "p50_queueing_s": float(np.percentile(qd, 50)),
                "throughput_traj_steps_s": self.traj_steps / self.makespan if self.makespan > 0 else math.nan,
                "makespan_s": self.makespan, "gpu_launches": self.launches,
                "peak_device_bytes": self.peak_bytes, "max_concurrent_requests": self.max_concurrent}


def estimated_flops(req: Request) -> float:
    """Work estimate of a request (FP64 flops, about three sweeps per step):
    the per-step and per-sweep counts of the kernel that will run it."""
    from . import ragged
    kind = KIND_IDS[req.kind]
    if kind == irkgl.RHS_KEPLER:
        per_step = 413 + 3 * 424
    else:
        per_step = ragged.flops_per_step(kind, req.dim) + 3 * ragged.flops_per_sweep(kind, req.dim)
    return float(req.batch) * req.nsteps * per_step


class Server:
    """policy "fifo" admits waiting requests in arrival order; "sjf" admits
    the one with the least estimated work first (shortest job first), which
    lowers the median latency when many requests wait; max_active caps how
    many requests share the GPU at once. mix = 1 runs the fixed-point stage
    mixing wherever a kernel with it is compiled (``new_context``)."""

    def __init__(self, mem_budget_bytes: int = 8 << 30, nstreams: int = 16,
                 chunk_traj_steps: float = 4e5, max_active: int = 512, device=None,
                 policy: str = "fifo", mix: int = 1):
        if policy not in ("fifo", "sjf"):
            raise ValueError(policy)
        self.policy = policy
        self.mix = 1 if mix else 0
        self.budget = int(mem_budget_bytes)
        self.device = device or torch.device("cuda")
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(nstreams)]
        self.chunk_traj_steps = chunk_traj_steps
        self.max_active = max_active
        self._next_stream = 0
        self._route_cache: dict = {}
        self._pool: dict = {}  # (kind, params, dim, wide) -> free contexts

    def _take_ctx(self, key, make):
        free = self._pool.get(key)
        return free.pop() if free else make()

    def _give_ctx(self, key, ctx):
        self._pool.setdefault(key, []).append(ctx)

    def close(self):
        for ctxs in self._pool.values():
            for c in ctxs:
                irkgl.irkgl_destroy(c)
        self._pool = {}

    # ---------------------------------------------------------------- admission
    def _admit(self, req: Request, now: float) -> _Active:
        dev = self.device
        stream = self.streams[self._next_stream % len(self.streams)]
        self._next_stream += 1
        key = (req.kind, req.dim)
        if key not in self._route_cache:
            self._route_cache[key] = not register_kernel_available(req.kind, req.params, req.dim)
        wide = self._route_cache[key]
        B, d = req.batch, req.dim
        f64 = dict(dtype=torch.float64, device=dev)
        def up(x):
            # pinned staging + asynchronous copy on the request's stream
            h = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).pin_memory()
            return h.to(dev, non_blocking=True)

        with torch.cuda.stream(stream):
            a = _Active(req=req, stream=stream, ctx=0, wide=wide,
                        q=up(req.q0).reshape(B, d),
                        v=up(req.v0).reshape(B, d),
                        qlo=torch.zeros((B, d), **f64), vlo=torch.zeros((B, d), **f64),
                        rp=torch.zeros((B, 8, d), **f64), h=None,
                        H0=torch.zeros(B, **f64), dH=torch.zeros(B, **f64),
                        it=torch.zeros(B, dtype=torch.int64, device=dev),
                        st=torch.zeros(B, dtype=torch.int32, device=dev),
                        ns=torch.zeros(B, dtype=torch.int64, device=dev))
            hb = np.broadcast_to(np.asarray(req.h, dtype=np.float64), (B,))
            a.h = up(hb)
            h_first = float(hb[0])
            if wide:
                a.ckey = ("wide",)
                a.ctx = self._take_ctx(a.ckey, lambda: new_wide_context(self.mix))
                w = {"kind": np.full(B, KIND_IDS[req.kind], np.int32), "dim": np.full(B, d, np.int32),
                     "offset": np.arange(B, dtype=np.int64) * d, "param_offset": np.zeros(B, np.int32),
                     "nparams": np.full(B, len(req.params), np.int32), "h": hb,
                     "nsteps": np.zeros(B, np.int64)}
                a.inst = irkgl.instances_tensor(w, dev)
                a.params_dev = up(np.asarray(req.params, dtype=np.float64))
            else:
                # the step size comes per trajectory (a.h), so contexts of the
                # same system are interchangeable
                a.ckey = (req.kind, tuple(float(x) for x in req.params), d)
                a.ctx = self._take_ctx(a.ckey, lambda: new_context(req.kind, req.params, d, h_first,
                                                                  self.mix))
        a.remaining = req.nsteps
        a.nbytes = req.device_bytes()
        req.t_admit = now
        return a

    def _launch_chunk(self, a: _Active):
        req = a.req
        k = int(max(16, min(a.remaining, self.chunk_traj_steps / max(req.batch, 1))))
        k = min(k, a.remaining)
        with torch.cuda.stream(a.stream):
            a.ns.fill_(k)
            if a.wide:
                irkgl.irkgl_advance_ragged(a.ctx, a.inst, req.batch, req.dim, a.params_dev,
                                           a.q, a.v, a.qlo, a.vlo, a.rp, a.ns, H0=a.H0,
                                           h0_init=not a.started, dH_max=a.dH, iters=a.it,
                                           status=a.st, stream=a.stream)
            else:
                irkgl.irkgl_advance(a.ctx, req.dim, a.q, a.v, a.qlo, a.vlo, a.rp, a.ns, h=a.h, H0=a.H0,
                                    h0_init=not a.started, dH_max=a.dH, iters=a.it, status=a.st,
                                    stream=a.stream)
            a.event = torch.cuda.Event()
            a.event.record(a.stream)
        a.started = True
        a.remaining -= k
        a.chunks += 1

    def _finish(self, a: _Active, now: float):
        req = a.req
        with torch.cuda.stream(a.stream):
            req.q = a.q.cpu().numpy()
            req.v = a.v.cpu().numpy()
            req.dH_max = a.dH.cpu().numpy()
            req.iters = a.it.cpu().numpy()
            req.status = a.st.cpu().numpy()
        self._give_ctx(a.ckey, a.ctx)
        req.t_done = now

    # ---------------------------------------------------------------- the loop
    def run(self, requests: list[Request], time_scale: float = 1.0) -> ServeStats:
        """Serve `requests` (arrival times in seconds, scaled by time_scale) to
        completion; returns latency / throughput statistics."""
        stats = ServeStats()
        pending = sorted(requests, key=lambda r: r.arrival)
        waiting: list[Request] = []
        active: list[_Active] = []
        used = 0
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        i = 0
        while i < len(pending) or waiting or active:
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival * time_scale <= now:
                waiting.append(pending[i])
                i += 1
            # admit in arrival order while memory and slots allow
            while waiting and len(active) < self.max_active:
                j = 0
                if self.policy == "sjf":
                    j = min(range(len(waiting)), key=lambda x: estimated_flops(waiting[x]))
                req = waiting[j]
                if used + req.device_bytes() > self.budget and active:
                    break
                waiting.pop(j)
                a = self._admit(req, now)
                used += a.nbytes
                active.append(a)
            stats.peak_bytes = max(stats.peak_bytes, used)
            stats.max_concurrent = max(stats.max_concurrent, len(active))
            progressed = False
            still = []
            for a in active:
                if a.event is not None and not a.event.query():
                    still.append(a)
                    continue
                if a.remaining > 0:
                    self._launch_chunk(a)
                    stats.launches += 1
                    progressed = True
                    still.append(a)
                else:
                    a.stream.synchronize()
                    t = time.perf_counter() - t0
                    self._finish(a, t)
                    used -= a.nbytes
                    stats.latencies.append(t - a.req.arrival * time_scale)
                    stats.queueing.append(a.req.t_admit - a.req.arrival * time_scale)
                    stats.traj_steps += a.req.traj_steps
                    progressed = True
            active = still
            if not progressed:
                time.sleep(50e-6)
        torch.cuda.synchronize(self.device)
        stats.makespan = time.perf_counter() - t0
        return stats


def run_plain(requests: list[Request], time_scale: float = 1.0, device=None, mix: int = 1) -> ServeStats:
    """The plain per-request GPU form: one request at a time, in arrival order,
    each integrated by one launch on the default stream."""
    device = device or torch.device("cuda")
    stats = ServeStats()
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    for req in sorted(requests, key=lambda r: r.arrival):
        now = time.perf_counter() - t0
        if req.arrival * time_scale > now:
            time.sleep(req.arrival * time_scale - now)
        req.t_admit = time.perf_counter() - t0
        B, d = req.batch, req.dim
        q0 = torch.tensor(req.q0, dtype=torch.float64, device=device).reshape(B, d).contiguous()
        v0 = torch.tensor(req.v0, dtype=torch.float64, device=device).reshape(B, d).contiguous()
        hb = np.ascontiguousarray(np.broadcast_to(np.asarray(req.h, dtype=np.float64), (B,)))
        if register_kernel_available(req.kind, req.params, d):
            ctx = new_context(req.kind, req.params, d, float(hb[0]), mix)
            out = irkgl.Outputs.allocate(B, d, device=device)
            irkgl.irkgl_integrate(ctx, d, q0, v0, out, nsteps_all=req.nsteps,
                                  h=torch.tensor(hb, dtype=torch.float64, device=device))
            irkgl.irkgl_destroy(ctx)
            req.q, req.v = out.q.cpu().numpy(), out.v.cpu().numpy()
            req.dH_max, req.iters, req.status = (out.dH_max.cpu().numpy(), out.iters.cpu().numpy(),
                                                 out.status.cpu().numpy())
        else:
            ctx = new_wide_context(mix)
            w = {"kind": np.full(B, KIND_IDS[req.kind], np.int32), "dim": np.full(B, d, np.int32),
                 "offset": np.arange(B, dtype=np.int64) * d, "param_offset": np.zeros(B, np.int32),
                 "nparams": np.full(B, len(req.params), np.int32), "h": hb,
                 "nsteps": np.full(B, req.nsteps, np.int64)}
            out = irkgl.RaggedOutputs.allocate(B * d, B, device=device)
            irkgl.irkgl_integrate_ragged(ctx, irkgl.instances_tensor(w, device), B, d,
                                         torch.tensor(np.asarray(req.params, dtype=np.float64), device=device),
                                         q0.reshape(-1), v0.reshape(-1), out)
            irkgl.irkgl_destroy(ctx)
            req.q, req.v = out.q.cpu().numpy().reshape(B, d), out.v.cpu().numpy().reshape(B, d)
            req.dH_max, req.iters, req.status = (out.dH_max.cpu().numpy(), out.iters.cpu().numpy(),
                                                 out.status.cpu().numpy())
        stats.launches += 1
        t = time.perf_counter() - t0
        req.t_done = t
        stats.latencies.append(t - req.arrival * time_scale)
        stats.queueing.append(req.t_admit - req.arrival * time_scale)
        stats.traj_steps += req.traj_steps
    stats.makespan = time.perf_counter() - t0
    return stats
