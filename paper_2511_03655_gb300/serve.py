"""Continuous-batching request loop over the IRKGL16 library.

Integration requests (a batch of initial states of one system, a step size
and a horizon) arrive over time.  The server keeps every admitted request's
state in the shared device arrays of one *pool* per kernel class:

  * a register pool per (right-hand side, dimension) that has a compiled
    register kernel (Kepler, the N-body tiles up to six bodies): arrays of
    trajectory slots advanced by ``irkgl_advance_multi``, each slot with its
    own parameters;
  * a wide pool per size bucket of the wide kernel (N-body by body count,
    FPUT chains by length): packed component arrays and instance
    descriptors advanced by ``irkgl_advance_ragged``.

A request is admitted as soon as its pool has room for it (the device-memory
budget is the pools' capacity), its initial states are copied up from
pinned host memory, and it joins its pool's next launch.  Every pool runs
its own tick loop on its own CUDA stream: when the pool's previous launch
has completed, finished requests are copied out and their slots freed,
waiting requests are admitted into the free slots, and ONE launch advances
every admitted request of the pool by up to K steps (K sized so that a tick
takes a few milliseconds).  So the number of launches per tick is the number
of busy pools, independent of the number of requests, and a request that
arrives while others run starts at the next tick of its pool.

A trajectory's bits do not depend on what it shares a launch with or on how
its steps are split over ticks: the continuation carries the compensated
state, R_prev, H_0 (computed at the trajectory's first step: its H0 entry
starts as NaN), the running maxima and a final status.  The pool of a
request depends only on its kind and dimension, and each wide pool has a
fixed team size, so a result is the same alone and in the mix.

``run_plain`` is the comparator: the plain per-request GPU form, one request
at a time in arrival order, each integrated by one launch.
"""
from __future__ import annotations

import bisect
import functools
import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import irkgl, ragged

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
        """Device memory of the request's state in a pool: q, v and their
        compensation parts, R_prev, and the per-trajectory scalars."""
        B, d = self.batch, self.dim
        return B * d * 8 * (2 + 2 + 8) + B * (8 * 5 + 4 + 4 + 40) + 8 * len(self.params) * B


def make_requests(descs: list[dict]) -> list[Request]:
    return [Request(**d) for d in descs]


_REGISTER_CACHE: dict = {}


def register_kernel_available(kind: str, params, dim: int) -> bool:
    """True if the batched register kernel is compiled for (kind, dim)."""
    key = (kind, dim)
    if key not in _REGISTER_CACHE:
        try:
            ctx = irkgl.irkgl_create(KIND_IDS[kind], params, dim, 0.1)
        except irkgl.IrkglError:
            _REGISTER_CACHE[key] = False
        else:
            try:
                _REGISTER_CACHE[key] = irkgl.irkgl_get_tile(ctx) > 0
            finally:
                irkgl.irkgl_destroy(ctx)
    return _REGISTER_CACHE[key]


# Register tiles whose fixed-point form is slower on GB300: the N-body tile
# spreads the stage rows over eight lanes, and the integer chains then cost
# occupancy (measured 3.9e7 vs 4.9e7 trajectory-steps/s on the 6-body ensemble).
FP64_MIX_FASTER = {"nbody"}


def new_context(kind: str, params, dim: int, h: float, mix: int) -> int:
    """A context for the register kernel of (kind, dim): with the fixed-point
    stage mixing when mix = 1, a kernel with it is compiled and it is the
    faster form, else with the FP64 mixing; mix = 2 is the reproducible form,
    which every register (kind, dim) has (an error otherwise, never a
    silent fallback). The choice depends only on (kind, dim, mix), so the
    server and run_plain integrate a request with the same kernel."""
    ctx = irkgl.irkgl_create(KIND_IDS[kind], params, dim, h)
    if mix == 2:
        irkgl.irkgl_set_option(ctx, irkgl.OPT_MIX, 2)
        if irkgl.irkgl_get_tile(ctx) <= 0:
            irkgl.irkgl_destroy(ctx)
            raise irkgl.IrkglError(f"no reproducible kernel for {kind} d={dim}")
        return ctx
    if mix and kind not in FP64_MIX_FASTER:
        irkgl.irkgl_set_option(ctx, irkgl.OPT_MIX, 1)
        if irkgl.irkgl_get_tile(ctx) <= 0:
            irkgl.irkgl_set_option(ctx, irkgl.OPT_MIX, 0)
    return ctx


def new_wide_context(mix: int, team: int = 0) -> int:
    """A context for the wide kernel (the kinds come per instance)."""
    ctx = irkgl.irkgl_create(irkgl.RHS_HARMONIC, [1.0], 1, 1.0)
    irkgl.irkgl_set_option(ctx, irkgl.OPT_MIX, mix if mix in (0, 2) else 1)
    if team:
        irkgl.irkgl_set_option(ctx, irkgl.OPT_WIDE_TEAM, team)
    return ctx


@functools.lru_cache(maxsize=None)
def wide_team(label: str) -> int:
    """Team size of a wide pool: the autotuner's tile table entry for the
    size bucket, else 256 (the library default)."""
    from . import autotune
    tab = autotune.load_table()
    tiles = (tab or {}).get("tiles", {}).get("wide", {})
    if label in tiles:
        return int(tiles[label]["team"])
    return 256


def pool_key(req: Request) -> tuple:
    """The kernel class a request runs in: ("register", kind, dim) or
    ("wide", size bucket)."""
    if register_kernel_available(req.kind, req.params, req.dim):
        return ("register", req.kind, req.dim)
    return ("wide", ragged.bucket_label(KIND_IDS[req.kind], req.dim))


def estimated_flops(req: Request) -> float:
    """Work estimate of a request (FP64 flops, about three sweeps per step):
    the per-step and per-sweep counts of the kernel that will run it."""
    kind = KIND_IDS[req.kind]
    if kind == irkgl.RHS_KEPLER:
        per_step = 413 + 3 * 424
    else:
        per_step = ragged.flops_per_step(kind, req.dim) + 3 * ragged.flops_per_sweep(kind, req.dim)
    return float(req.batch) * req.nsteps * per_step


def algorithmic_flops(req: Request) -> float:
    """Algorithmic FP64 flops of a served request from its sweep totals
    (the kernels' per-step and per-sweep counts)."""
    kind = KIND_IDS[req.kind]
    sweeps = float(np.asarray(req.iters).sum()) if req.iters is not None else 0.0
    steps = float(req.batch) * req.nsteps
    if kind == irkgl.RHS_KEPLER:
        return 413.0 * steps + 424.0 * sweeps
    if kind == irkgl.RHS_NBODY and req.dim == 18:
        return 3882.0 * steps + 6456.0 * sweeps
    return ragged.flops_per_step(kind, req.dim) * steps + ragged.flops_per_sweep(kind, req.dim) * sweeps


# --------------------------------------------------------------------------
# pools
# --------------------------------------------------------------------------
class _Ranges:
    """First-fit allocation of contiguous ranges of [0, capacity)."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.free = [(0, self.capacity)] if capacity > 0 else []   # sorted, coalesced
        self.used: dict = {}

    def alloc(self, n: int):
        if n <= 0:
            return 0
        for k, (s, length) in enumerate(self.free):
            if length >= n:
                if length == n:
                    del self.free[k]
                else:
                    self.free[k] = (s + n, length - n)
                self.used[s] = n
                return s
        return None

    def release(self, s: int):
        n = self.used.pop(s, 0)
        if n <= 0:
            return
        k = bisect.bisect_left(self.free, (s, 0))
        self.free.insert(k, (s, n))
        # merge with the right, then the left neighbour
        if k + 1 < len(self.free) and self.free[k][0] + self.free[k][1] == self.free[k + 1][0]:
            self.free[k] = (s, self.free[k][1] + self.free[k + 1][1])
            del self.free[k + 1]
        if k > 0 and self.free[k - 1][0] + self.free[k - 1][1] == self.free[k][0]:
            self.free[k - 1] = (self.free[k - 1][0], self.free[k - 1][1] + self.free[k][1])
            del self.free[k]

    def high_water(self) -> int:
        return max((s + n for s, n in self.used.items()), default=0)


@dataclass
class _Member:
    req: Request
    slot: int              # first trajectory slot (register) / instance (wide)
    comp: int = 0          # first packed component (wide)
    par: int = 0           # first packed parameter (wide)
    remaining: int = 0
    k: int = 0             # steps of the launch in flight
    done_event: torch.cuda.Event | None = None
    host: dict | None = None


class _Pool:
    """Shared device arrays of the requests of one kernel class, advanced by
    one launch per tick on the pool's own stream."""

    def __init__(self, key, mix, device, capacity_bytes, target_tick_s):
        self.key = key
        self.mix = mix
        self.device = device
        self.capacity_bytes = int(capacity_bytes)
        self.target = target_tick_s
        self.stream = torch.cuda.Stream(device=device)
        self.members: list[_Member] = []
        self.waiting: list[Request] = []
        self.event: torch.cuda.Event | None = None  # end of the launch in flight
        self.launch_events: list = []              # (start, end, traj-steps) per launch
        self.K = 16                                # steps per tick, adapted to the target
        self._rated = 0                            # launches whose time has set K
        self._k_of_launch: list = []               # largest k of each launch
        self._traj_last = 0                        # trajectories of the last launch
        self.ctx = 0
        self.allocated = False

    def idle(self) -> bool:
        return self.event is None or self.event.query()

    def settle(self):
        """After the launch in flight: size the next tick from the time per
        step of the last one (K steps take about `target` seconds, whatever
        the batch: a pool holding one long trajectory gets short ticks too,
        so requests that arrive behind it wait one tick at most), and return
        the members whose horizon is reached."""
        if self._rated < len(self.launch_events):
            a, b, _ = self.launch_events[-1]
            k_last = self._k_of_launch[-1]
            if b.query():
                self._rated = len(self.launch_events)
                dt = a.elapsed_time(b) * 1e-3
                if dt > 0 and k_last > 0:
                    want = k_last * self.target / dt
                    self.K = int(max(1, min(1 << 20, k_last * 4, max(k_last / 4, want))))
        finished = [m for m in self.members if m.remaining == 0 and m.k >= 0]
        return finished

    def launch(self) -> int:
        live = [m for m in self.members if m.remaining > 0]
        if not live:
            return 0
        # K was measured on the last launch's trajectories: when more joined
        # since, a step may take proportionally longer, so shorten the tick
        traj = sum(m.req.batch for m in live)
        K = self.K
        if self._traj_last and traj > self._traj_last:
            K = max(1, int(K * self._traj_last / traj))
        self._traj_last = traj
        for m in live:
            m.k = min(m.remaining, K)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(self.stream):
            self._upload_tick(live)
            start.record(self.stream)
            self._launch(live)
            end.record(self.stream)
        self.launch_events.append((start, end, sum(m.k * m.req.batch for m in live)))
        self._k_of_launch.append(max(m.k for m in live))
        for m in live:
            m.remaining -= m.k
        self.event = end
        return 1


class _RegisterPool(_Pool):
    """Trajectory slots of one (kind, dim) on the register kernel."""

    def __init__(self, key, req: Request, mix, device, capacity_bytes, target_tick_s):
        super().__init__(key, mix, device, capacity_bytes, target_tick_s)
        self.kind, self.dim = req.kind, req.dim
        self.P = len(req.params)
        d = self.dim
        self.slot_bytes = 8 * (12 * d + self.P + 4) + 8 + 4 + 4 + 8
        self.cap = max(1, self.capacity_bytes // self.slot_bytes)
        self.slots = _Ranges(self.cap)
        self.ctx = new_context(req.kind, req.params, d, 0.1, mix)

    def _allocate(self):
        S, d, dev = self.cap, self.dim, self.device
        f64 = dict(dtype=torch.float64, device=dev)
        with torch.cuda.stream(self.stream):
            self.q = torch.zeros((S, d), **f64)
            self.v = torch.zeros((S, d), **f64)
            self.ql = torch.zeros((S, d), **f64)
            self.vl = torch.zeros((S, d), **f64)
            self.rp = torch.zeros((S, 8, d), **f64)
            self.params = torch.zeros((S, self.P), **f64)
            self.h = torch.ones(S, **f64)
            self.H0 = torch.zeros(S, **f64)
            self.dH = torch.zeros(S, **f64)
            self.it = torch.zeros(S, dtype=torch.int64, device=dev)
            self.st = torch.zeros(S, dtype=torch.int32, device=dev)
            self.ns = torch.zeros(S, dtype=torch.int64, device=dev)
            self.order = torch.full((S,), -1, dtype=torch.int32, device=dev)
        self.ns_host = torch.zeros(S, dtype=torch.int64, pin_memory=True)
        self.order_host = torch.full((S,), -1, dtype=torch.int32, pin_memory=True)
        self.allocated = True

    def fits(self, req: Request) -> bool:
        return req.batch <= self.cap

    def admit(self, req: Request):
        if not self.allocated:
            self._allocate()
        B = req.batch
        s = self.slots.alloc(B)
        if s is None:
            return None
        sl = slice(s, s + B)
        hb = np.broadcast_to(np.asarray(req.h, dtype=np.float64), (B,))
        pin = lambda x: torch.from_numpy(np.array(x, dtype=np.float64, copy=True)).pin_memory()  # noqa: E731
        with torch.cuda.stream(self.stream):
            self.q[sl].copy_(pin(req.q0).reshape(B, self.dim), non_blocking=True)
            self.v[sl].copy_(pin(req.v0).reshape(B, self.dim), non_blocking=True)
            self.params[sl].copy_(pin(np.broadcast_to(np.asarray(req.params, np.float64), (B, self.P))),
                                  non_blocking=True)
            self.h[sl].copy_(pin(hb), non_blocking=True)
            for t in (self.ql[sl], self.vl[sl], self.rp[sl], self.dH[sl], self.it[sl], self.st[sl]):
                t.zero_()
            self.H0[sl].fill_(float("nan"))  # computed at the trajectory's first step
        m = _Member(req=req, slot=s, remaining=req.nsteps, k=-1 if req.nsteps > 0 else 0)
        self.members.append(m)
        return m

    def _upload_tick(self, live):
        n = 0
        ns, od = self.ns_host.numpy(), self.order_host.numpy()
        for m in live:
            B = m.req.batch
            ns[m.slot:m.slot + B] = m.k
            od[n:n + B] = np.arange(m.slot, m.slot + B, dtype=np.int32)
            n += B
        hw = self.slots.high_water()
        od[n:hw] = -1
        self.batch = hw
        self.ns[:hw].copy_(self.ns_host[:hw], non_blocking=True)
        self.order[:hw].copy_(self.order_host[:hw], non_blocking=True)

    def _launch(self, live):
        hw = self.batch
        irkgl.irkgl_advance_multi(self.ctx, self.dim, self.q[:hw], self.v[:hw], self.ql[:hw],
                                  self.vl[:hw], self.rp[:hw], self.ns[:hw], h=self.h[:hw],
                                  params=self.params[:hw], param_stride=self.P,
                                  order=self.order[:hw], H0=self.H0[:hw], dH_max=self.dH[:hw],
                                  iters=self.it[:hw], status=self.st[:hw], stream=self.stream)

    def retire(self, m: _Member):
        """Copy the member's results to pinned host memory (on the pool's
        stream, after its last launch) and free its slots."""
        B, sl = m.req.batch, slice(m.slot, m.slot + m.req.batch)
        with torch.cuda.stream(self.stream):
            host = {"q": torch.empty((B, self.dim), dtype=torch.float64, pin_memory=True),
                    "v": torch.empty((B, self.dim), dtype=torch.float64, pin_memory=True),
                    "dH": torch.empty(B, dtype=torch.float64, pin_memory=True),
                    "it": torch.empty(B, dtype=torch.int64, pin_memory=True),
                    "st": torch.empty(B, dtype=torch.int32, pin_memory=True)}
            host["q"].copy_(self.q[sl], non_blocking=True)
            host["v"].copy_(self.v[sl], non_blocking=True)
            host["dH"].copy_(self.dH[sl], non_blocking=True)
            host["it"].copy_(self.it[sl], non_blocking=True)
            host["st"].copy_(self.st[sl], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        m.host, m.done_event = host, ev
        self.slots.release(m.slot)
        self.members.remove(m)


class _WidePool(_Pool):
    """Packed instances of one size bucket on the wide kernel."""

    def __init__(self, key, req: Request, mix, device, capacity_bytes, target_tick_s):
        super().__init__(key, mix, device, capacity_bytes, target_tick_s)
        self.label = key[1]
        lo, hi = (int(x) for x in self.label.split(":")[1].split("-"))
        self.dmax = 3 * hi if self.label.startswith("nbody") else hi
        self.team = wide_team(self.label)
        # capacity: components (q, v, their compensation parts and R_prev: 12
        # doubles each, plus margin), instances (at most one per component of
        # the bucket's smallest size, at most 2^20), parameters (2^20 doubles)
        lo_dim = 3 * lo if self.label.startswith("nbody") else lo
        self.comp_cap = max(self.dmax, self.capacity_bytes // (12 * 8 + 8))
        self.inst_cap = int(max(64, min(self.comp_cap // max(lo_dim, 1), 1 << 20)))
        self.par_cap = 1 << 20
        self.comps = _Ranges(self.comp_cap)
        self.insts = _Ranges(self.inst_cap)
        self.pars = _Ranges(self.par_cap)
        self.ctx = new_wide_context(mix, self.team)

    def _allocate(self):
        C, I, dev = self.comp_cap, self.inst_cap, self.device
        f64 = dict(dtype=torch.float64, device=dev)
        with torch.cuda.stream(self.stream):
            self.q = torch.zeros(C, **f64)
            self.v = torch.zeros(C, **f64)
            self.ql = torch.zeros(C, **f64)
            self.vl = torch.zeros(C, **f64)
            self.rp = torch.zeros(8 * C, **f64)
            self.params = torch.zeros(self.par_cap, **f64)
            self.inst = torch.zeros(I * ragged.INSTANCE_BYTES, dtype=torch.uint8, device=dev)
            self.H0 = torch.zeros(I, **f64)
            self.dH = torch.zeros(I, **f64)
            self.it = torch.zeros(I, dtype=torch.int64, device=dev)
            self.st = torch.zeros(I, dtype=torch.int32, device=dev)
            self.ns = torch.zeros(I, dtype=torch.int64, device=dev)
            self.order = torch.full((I,), -1, dtype=torch.int32, device=dev)
        self.ns_host = torch.zeros(I, dtype=torch.int64, pin_memory=True)
        self.order_host = torch.full((I,), -1, dtype=torch.int32, pin_memory=True)
        self.allocated = True

    def fits(self, req: Request) -> bool:
        return req.batch * req.dim <= self.comp_cap and req.batch <= self.inst_cap \
            and len(req.params) <= self.par_cap

    def admit(self, req: Request):
        if not self.allocated:
            self._allocate()
        B, d, P = req.batch, req.dim, len(req.params)
        c = self.comps.alloc(B * d)
        if c is None:
            return None
        s = self.insts.alloc(B)
        if s is None:
            self.comps.release(c)
            return None
        p = self.pars.alloc(P)
        if p is None:
            self.comps.release(c)
            self.insts.release(s)
            return None
        hb = np.broadcast_to(np.asarray(req.h, dtype=np.float64), (B,))
        rec = irkgl.instances_array({
            "kind": np.full(B, KIND_IDS[req.kind], np.int32), "dim": np.full(B, d, np.int32),
            "offset": c + np.arange(B, dtype=np.int64) * d, "param_offset": np.full(B, p, np.int32),
            "nparams": np.full(B, P, np.int32), "h": hb, "nsteps": np.zeros(B, np.int64)})
        pin = lambda x: torch.from_numpy(np.array(x, dtype=np.float64, copy=True).reshape(-1)).pin_memory()  # noqa: E731
        cs, ss = slice(c, c + B * d), slice(s, s + B)
        with torch.cuda.stream(self.stream):
            self.q[cs].copy_(pin(req.q0), non_blocking=True)
            self.v[cs].copy_(pin(req.v0), non_blocking=True)
            self.params[p:p + P].copy_(pin(req.params), non_blocking=True)
            raw = torch.from_numpy(rec.view(np.uint8).copy()).pin_memory()
            self.inst[s * ragged.INSTANCE_BYTES:(s + B) * ragged.INSTANCE_BYTES].copy_(raw, non_blocking=True)
            for t in (self.ql[cs], self.vl[cs], self.rp[8 * c:8 * (c + B * d)], self.dH[ss],
                      self.it[ss], self.st[ss]):
                t.zero_()
            self.H0[ss].fill_(float("nan"))  # computed at the instance's first step
        m = _Member(req=req, slot=s, comp=c, par=p, remaining=req.nsteps, k=-1 if req.nsteps > 0 else 0)
        self.members.append(m)
        return m

    def _upload_tick(self, live):
        # costliest members first, so the persistent teams stay balanced
        live = sorted(live, key=lambda m: -(m.req.dim * m.k))
        ns, od = self.ns_host.numpy(), self.order_host.numpy()
        n = 0
        for m in live:
            B = m.req.batch
            ns[m.slot:m.slot + B] = m.k
            od[n:n + B] = np.arange(m.slot, m.slot + B, dtype=np.int32)
            n += B
        hw = self.insts.high_water()
        od[n:hw] = -1
        self.ninst = hw
        self.ns[:hw].copy_(self.ns_host[:hw], non_blocking=True)
        self.order[:hw].copy_(self.order_host[:hw], non_blocking=True)

    def _launch(self, live):
        hw = self.ninst
        irkgl.irkgl_advance_ragged(self.ctx, self.inst[:hw * ragged.INSTANCE_BYTES], hw, self.dmax,
                                   self.params, self.q, self.v, self.ql, self.vl, self.rp,
                                   self.ns[:hw], H0=self.H0[:hw], h0_init=False, dH_max=self.dH[:hw],
                                   iters=self.it[:hw], status=self.st[:hw], order=self.order[:hw],
                                   stream=self.stream)

    def retire(self, m: _Member):
        B, d = m.req.batch, m.req.dim
        cs, ss = slice(m.comp, m.comp + B * d), slice(m.slot, m.slot + B)
        with torch.cuda.stream(self.stream):
            host = {"q": torch.empty(B * d, dtype=torch.float64, pin_memory=True),
                    "v": torch.empty(B * d, dtype=torch.float64, pin_memory=True),
                    "dH": torch.empty(B, dtype=torch.float64, pin_memory=True),
                    "it": torch.empty(B, dtype=torch.int64, pin_memory=True),
                    "st": torch.empty(B, dtype=torch.int32, pin_memory=True)}
            host["q"].copy_(self.q[cs], non_blocking=True)
            host["v"].copy_(self.v[cs], non_blocking=True)
            host["dH"].copy_(self.dH[ss], non_blocking=True)
            host["it"].copy_(self.it[ss], non_blocking=True)
            host["st"].copy_(self.st[ss], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(self.stream)
        m.host, m.done_event = host, ev
        self.comps.release(m.comp)
        self.insts.release(m.slot)
        self.pars.release(m.par)
        self.members.remove(m)


# --------------------------------------------------------------------------
# statistics
# --------------------------------------------------------------------------
@dataclass
class ServeStats:
    latencies: list = field(default_factory=list)
    queueing: list = field(default_factory=list)
    traj_steps: int = 0
    flops: float = 0.0
    makespan: float = 0.0
    launches: int = 0
    ticks: int = 0
    peak_bytes: int = 0
    max_concurrent: int = 0
    gpu_busy_s: float = 0.0
    pools: int = 0

    def summary(self) -> dict:
        lat = np.array(self.latencies) if self.latencies else np.array([math.nan])
        qd = np.array(self.queueing) if self.queueing else np.array([math.nan])
        return {"requests": len(self.latencies), "p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
                "p50_queueing_s": float(np.percentile(qd, 50)),
                "throughput_traj_steps_s": self.traj_steps / self.makespan if self.makespan > 0 else math.nan,
                "flops_per_s": self.flops / self.makespan if self.makespan > 0 else math.nan,
                "makespan_s": self.makespan, "gpu_launches": self.launches,
                "launches_per_tick": self.launches / self.ticks if self.ticks else math.nan,
                "gpu_busy": self.gpu_busy_s / self.makespan if self.makespan > 0 else math.nan,
                "peak_device_bytes": self.peak_bytes, "max_concurrent_requests": self.max_concurrent,
                "pools": self.pools}


def _union_length(intervals) -> float:
    tot, end = 0.0, -math.inf
    for a, b in sorted(intervals):
        if b <= end:
            continue
        tot += b - max(a, end)
        end = b
    return tot


# --------------------------------------------------------------------------
# the server
# --------------------------------------------------------------------------
class Server:
    """policy "fifo" admits each pool's waiting requests in arrival order;
    "sjf" admits the one with the least estimated work first (shortest job
    first); max_active caps how many requests are admitted at once.
    pool_bytes is the device memory of each pool's state arrays (allocated
    when the pool's first request is admitted; a pool whose largest request
    is bigger gets that size): requests wait until their pool has room.
    mix = 1 runs the fixed-point stage mixing wherever a kernel with it is
    compiled (``new_context``); mix = 2 runs every pool in the reproducible
    form (each request's results are then those of any IEEE FP64 program of
    the method's plain sequence).  target_tick_s is the wanted duration of a
    tick: each pool sizes its steps per tick from the time per step of its
    previous tick."""

    def __init__(self, pool_bytes: int = 1 << 30, max_active: int = 1 << 20, device=None,
                 policy: str = "fifo", mix: int = 1, target_tick_s: float = 0.03):
        if policy not in ("fifo", "sjf"):
            raise ValueError(policy)
        self.policy = policy
        if mix not in (0, 1, 2):
            raise ValueError(f"mix {mix}: 0, 1 or 2")
        self.mix = mix
        self.pool_bytes = int(pool_bytes)
        self.device = device or torch.device("cuda")
        self.max_active = max_active
        self.target = target_tick_s
        self.pools: dict = {}

    def close(self):
        for p in self.pools.values():
            irkgl.irkgl_destroy(p.ctx)
        self.pools = {}

    def _pools_for(self, requests: list[Request]):
        """Create the pools the requests route to (before the clock starts),
        each large enough for its largest request."""
        need: dict = {}
        first: dict = {}
        for r in requests:
            key = pool_key(r)
            need[key] = max(need.get(key, 0), r.device_bytes())
            first.setdefault(key, r)
        for key, nbytes in need.items():
            p = self.pools.get(key)
            if p is not None and p.fits(first[key]) and p.capacity_bytes >= nbytes:
                continue
            if p is not None and not p.members:
                irkgl.irkgl_destroy(p.ctx)
            cls = _RegisterPool if key[0] == "register" else _WidePool
            self.pools[key] = cls(key, first[key], self.mix, self.device,
                                  max(self.pool_bytes, 2 * nbytes), self.target)
        for p in self.pools.values():
            if not p.allocated:
                p._allocate()  # device arrays before the clock starts

    def run(self, requests: list[Request], time_scale: float = 1.0) -> ServeStats:
        """Serve `requests` (arrival times in seconds, scaled by time_scale) to
        completion; returns latency / throughput statistics."""
        stats = ServeStats()
        pending = sorted(requests, key=lambda r: r.arrival)
        self._pools_for(pending)
        for p in self.pools.values():
            p.launch_events, p._k_of_launch, p._rated, p._traj_last = [], [], 0, 0
        finishing: list[tuple[_Pool, _Member]] = []
        active = 0
        torch.cuda.synchronize(self.device)
        ref = torch.cuda.Event(enable_timing=True)
        ref.record(torch.cuda.current_stream(self.device))
        t0 = time.perf_counter()
        i = 0
        remaining_reqs = len(pending)
        while remaining_reqs > 0:
            now = time.perf_counter() - t0
            while i < len(pending) and pending[i].arrival * time_scale <= now:
                self.pools[pool_key(pending[i])].waiting.append(pending[i])
                i += 1
            progressed = False
            launched = 0
            for p in self.pools.values():
                if not p.idle():
                    continue
                for m in p.settle():
                    p.retire(m)
                    finishing.append((p, m))
                    active -= 1
                    progressed = True
                # admission into the pool's free slots
                while p.waiting and active < self.max_active:
                    j = 0
                    if self.policy == "sjf":
                        j = min(range(len(p.waiting)), key=lambda x: estimated_flops(p.waiting[x]))
                    req = p.waiting[j]
                    if not p.fits(req):
                        raise ValueError(f"request {req.rid} ({req.kind}, d = {req.dim}, batch "
                                         f"{req.batch}) does not fit an empty pool")
                    if p.admit(req) is None:
                        break
                    p.waiting.pop(j)
                    req.t_admit = time.perf_counter() - t0
                    active += 1
                    progressed = True
                n = p.launch()
                launched += n
            stats.launches += launched
            stats.ticks += 1 if launched else 0
            progressed = progressed or launched > 0
            stats.max_concurrent = max(stats.max_concurrent, active)
            if launched:
                used = sum(r.req.device_bytes() for p in self.pools.values() for r in p.members)
                stats.peak_bytes = max(stats.peak_bytes, used)
            still = []
            for p, m in finishing:
                if m.done_event.query():
                    t = time.perf_counter() - t0
                    req = m.req
                    B, d = req.batch, req.dim
                    req.q = m.host["q"].numpy().reshape(B, d).copy()
                    req.v = m.host["v"].numpy().reshape(B, d).copy()
                    req.dH_max = m.host["dH"].numpy().copy()
                    req.iters = m.host["it"].numpy().copy()
                    req.status = m.host["st"].numpy().copy()
                    req.t_done = t
                    stats.latencies.append(t - req.arrival * time_scale)
                    stats.queueing.append(req.t_admit - req.arrival * time_scale)
                    stats.traj_steps += req.traj_steps
                    stats.flops += algorithmic_flops(req)
                    remaining_reqs -= 1
                    progressed = True
                else:
                    still.append((p, m))
            finishing = still
            if not progressed:
                time.sleep(20e-6)
        torch.cuda.synchronize(self.device)
        stats.makespan = time.perf_counter() - t0
        # device-busy time: the union of the launches' intervals on the GPU clock
        iv = []
        for p in self.pools.values():
            for a, b, _ in p.launch_events:
                iv.append((ref.elapsed_time(a) * 1e-3, ref.elapsed_time(b) * 1e-3))
        stats.gpu_busy_s = _union_length(iv)
        stats.pools = sum(1 for p in self.pools.values() if p.launch_events)
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
        key = pool_key(req)
        if key[0] == "register":
            ctx = new_context(req.kind, req.params, d, float(hb[0]), mix)
            out = irkgl.Outputs.allocate(B, d, device=device)
            irkgl.irkgl_integrate(ctx, d, q0, v0, out, nsteps_all=req.nsteps,
                                  h=torch.tensor(hb, dtype=torch.float64, device=device))
            irkgl.irkgl_destroy(ctx)
            req.q, req.v = out.q.cpu().numpy(), out.v.cpu().numpy()
            req.dH_max, req.iters, req.status = (out.dH_max.cpu().numpy(), out.iters.cpu().numpy(),
                                                 out.status.cpu().numpy())
        else:
            ctx = new_wide_context(mix, wide_team(key[1]))
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
        stats.flops += algorithmic_flops(req)
    stats.makespan = time.perf_counter() - t0
    return stats
