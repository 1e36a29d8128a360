"""Bucketed launches for ragged batches (the wide kernel, irkgl_integrate_ragged).

One launch of the wide kernel uses one team size for the whole batch, chosen
for the largest instance; a small instance on a large team leaves most of
its threads idle in the per-component work.  ``RaggedPlan`` groups the
instances into size buckets per right-hand side (N-body by body count, FPUT
by chain length), orders each bucket costliest first, and gives each bucket
its own team size: from the autotuner's tile table when one is given, else
the library's choice for the bucket's largest dimension.  ``RaggedRunner``
launches every bucket on its own CUDA stream (each launch is a persistent
grid over all SMs, so buckets overlap at their tails) and joins them.

Team shapes give bit-identical states, sweep counts and statuses (the
per-component arithmetic and the summation orders of the method do not
depend on the team size), so a bucketed run equals one launch of the whole
batch bit for bit in those; only the energy monitor's sum of H over the
team (per-warp partials) rounds differently, so dH_max agrees to roundoff.

Instance descriptors are re-ordered on the host; the packed state arrays
keep their layout (descriptors carry absolute offsets), and per-instance
outputs come back in plan order (``RaggedPlan.perm``; ``unpermute`` maps
them back to the caller's instance order).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import irkgl

# Size buckets: N-body by body count N = d/3, FPUT and harmonic by d.
NBODY_BUCKETS = ((3, 8), (9, 16), (17, 32), (33, 64), (65, 128))
CHAIN_BUCKETS = ((1, 64), (65, 128), (129, 256), (257, 512), (513, 1024), (1025, 1536))
INSTANCE_BYTES = 40  # sizeof(irkgl_instance)


def bucket_label(kind: int, dim: int) -> str:
    if kind == irkgl.RHS_NBODY:
        n = dim // 3
        for lo, hi in NBODY_BUCKETS:
            if lo <= n <= hi:
                return f"nbody:{lo}-{hi}"
    else:
        name = "fput" if kind == irkgl.RHS_FPUT else "harmonic"
        for lo, hi in CHAIN_BUCKETS:
            if lo <= dim <= hi:
                return f"{name}:{lo}-{hi}"
    raise ValueError(f"no bucket for kind {kind}, dim {dim}")


def flops_per_step(kind: int, dim: int) -> float:
    """Algorithmic FP64 flops (an FMA counts 2) per completed step, outside
    the sweeps: fused initial guess 152 d, compensated update 45 d, energy
    monitor (N-body 16 per pair + 16 per body; chains 8 d)."""
    if kind == irkgl.RHS_NBODY:
        n = dim // 3
        return 197.0 * dim + 16.0 * n * (n - 1) / 2 + 16.0 * n
    return 205.0 * dim


def flops_per_sweep(kind: int, dim: int) -> float:
    """Algorithmic FP64 flops per fixed-point sweep: g and R over the 8
    stages (N-body 31 per pair per stage; FPUT 6 per component per stage;
    harmonic 2), the eta mixing 144 d and the Delta differences 8 d."""
    if kind == irkgl.RHS_NBODY:
        n = dim // 3
        return 248.0 * n * (n - 1) / 2 + 152.0 * dim
    if kind == irkgl.RHS_FPUT:
        return 200.0 * dim
    return 168.0 * dim


def algorithmic_flops(kind, dim, steps, iters) -> float:
    """Sum over instances of flops_per_step * steps + flops_per_sweep * sweeps."""
    tot = 0.0
    for k, d, s, i in zip(kind, dim, steps, iters):
        tot += flops_per_step(int(k), int(d)) * float(s) + flops_per_sweep(int(k), int(d)) * float(i)
    return tot


@dataclass
class Bucket:
    label: str
    start: int       # first instance (plan order)
    count: int
    dmax: int
    team: int        # 0 = the library's choice for dmax


class RaggedPlan:
    """Bucketing of a ragged batch ``w`` (the dict of workloads.uneven_batch)."""

    def __init__(self, w: dict, tiles: dict | None = None):
        kinds = np.asarray(w["kind"])
        dims = np.asarray(w["dim"])
        labels = [bucket_label(int(k), int(d)) for k, d in zip(kinds, dims)]
        cost = np.array([flops_per_sweep(int(k), int(d)) for k, d in zip(kinds, dims)])
        uniq = sorted(set(labels), key=lambda s: (s.split(":")[0], int(s.split(":")[1].split("-")[0])))
        perm, buckets = [], []
        for lab in uniq:
            idx = np.array([i for i, x in enumerate(labels) if x == lab], dtype=np.int64)
            idx = idx[np.argsort(-cost[idx], kind="stable")]
            team = 0
            if tiles and lab in tiles:
                team = int(tiles[lab]["team"])
            buckets.append(Bucket(lab, len(perm), len(idx), int(dims[idx].max()), team))
            perm.extend(idx.tolist())
        # costliest buckets first: they start while the short ones fill in
        self.perm = np.array(perm, dtype=np.int64)
        self.buckets = sorted(buckets, key=lambda b: -float(cost[self.perm[b.start:b.start + b.count]].sum()))
        self.w = w

    def permuted(self) -> dict:
        """Instance arrays in plan order (packed state arrays unchanged)."""
        w, p = self.w, self.perm
        out = dict(w)
        for k in ("kind", "dim", "offset", "param_offset", "nparams", "h", "nsteps"):
            out[k] = np.asarray(w[k])[p]
        return out

    def unpermute(self, a: np.ndarray) -> np.ndarray:
        """Per-instance array in plan order -> the caller's instance order."""
        r = np.empty_like(a)
        r[self.perm] = a
        return r


class RaggedRunner:
    """Device-resident ragged batch run as bucketed launches.

    ``run(out)`` integrates every instance from (q0, v0) into ``out`` (a
    RaggedOutputs with per-instance arrays in plan order).  ``single(out)``
    is the comparator: one launch of the whole batch with one team size
    (``team`` = 0: the library's choice for the largest dimension)."""

    def __init__(self, plan: RaggedPlan, params, q0, v0, device="cuda", mix: int = 0):
        self.plan = plan
        self.mix = mix
        wp = plan.permuted()
        self.inst = irkgl.instances_tensor(wp, device)
        self.ninst = len(wp["kind"])
        self.dmax = int(np.asarray(wp["dim"]).max())
        self.params, self.q0, self.v0 = params, q0, v0
        # one context per bucket: each holds the work counter of its launch,
        # and the launches run concurrently
        self.bctx = [self._ctx(b.team) for b in plan.buckets]
        self.ctx = {}
        self.streams = [torch.cuda.Stream(device=device) for _ in plan.buckets]

    def _ctx(self, team: int) -> int:
        c = irkgl.irkgl_create(irkgl.RHS_HARMONIC, [1.0], 1, 0.1)
        irkgl.irkgl_set_option(c, irkgl.OPT_WIDE_TEAM, team)
        irkgl.irkgl_set_option(c, irkgl.OPT_MIX, self.mix)
        return c

    def launches(self) -> int:
        return len(self.plan.buckets)

    def run(self, out: irkgl.RaggedOutputs):
        cur = torch.cuda.current_stream()
        ev = torch.cuda.Event()
        ev.record(cur)
        for b, s, c in zip(self.plan.buckets, self.streams, self.bctx):
            s.wait_event(ev)
            sl = slice(b.start, b.start + b.count)
            view = irkgl.RaggedOutputs(q=out.q, v=out.v, q_lo=out.q_lo, v_lo=out.v_lo, r_prev=out.r_prev,
                                       dH_max=out.dH_max[sl], iters=out.iters[sl], steps=out.steps[sl],
                                       status=out.status[sl])
            inst = self.inst[b.start * INSTANCE_BYTES:(b.start + b.count) * INSTANCE_BYTES]
            irkgl.irkgl_integrate_ragged(c, inst, b.count, b.dmax, self.params,
                                         self.q0, self.v0, view, stream=s)
        for s in self.streams:
            done = torch.cuda.Event()
            done.record(s)
            cur.wait_event(done)

    def capture(self, out: irkgl.RaggedOutputs) -> torch.cuda.CUDAGraph:
        """Record run(out) as a CUDA graph: every bucket's counter reset and
        launch on its own stream, forked from and joined to the capturing
        stream.  graph.replay() then repeats the whole bucketed integration
        into `out` with one host call; the results are those of run(out)
        bit for bit.  Inputs and outputs stay at the addresses captured."""
        self.run(out)  # resolves each bucket's shape and shared-memory attribute first
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            self.run(out)
        return g

    def single(self, out: irkgl.RaggedOutputs, team: int = 0):
        if team not in self.ctx:
            self.ctx[team] = self._ctx(team)
        irkgl.irkgl_integrate_ragged(self.ctx[team], self.inst, self.ninst, self.dmax, self.params,
                                     self.q0, self.v0, out)

    def close(self):
        for c in list(self.ctx.values()) + self.bctx:
            irkgl.irkgl_destroy(c)
        self.ctx, self.bctx = {}, []
