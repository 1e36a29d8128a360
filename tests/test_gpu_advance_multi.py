"""The continuation calls a serving loop runs on (through the C-ABI):

  * irkgl_advance_multi: per-trajectory parameters give the bits of separate
    contexts; an H0 entry holding NaN is computed at the trajectory's first
    step (so a trajectory joining a running batch gets the bits of a fresh
    run); slots listed as -1 in `order` are not touched; a nonzero status on
    entry is final; a parameter stride below the kind's count is rejected;
  * irkgl_advance_ragged: the same H0 / order / status rules per instance;
  * the wide kernel's shape for chains longer than 1024 (c_i v formed again
    instead of stored: the same bits as the stored form) against the oracle.
"""
import ctypes

import numpy as np
import pytest

from oracle import cbind
from paper_2511_03655_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    return torch, irkgl


class Slots:
    """Device arrays of B trajectory slots of dimension d."""

    def __init__(self, torch, q0, v0, P):
        B, d = q0.shape
        f = dict(dtype=torch.float64, device="cuda")
        self.q = torch.tensor(q0, **f)
        self.v = torch.tensor(v0, **f)
        self.ql = torch.zeros((B, d), **f)
        self.vl = torch.zeros((B, d), **f)
        self.rp = torch.zeros((B, 8, d), **f)
        self.params = torch.zeros((B, P), **f)
        self.H0 = torch.full((B,), float("nan"), **f)
        self.dH = torch.zeros(B, **f)
        self.it = torch.zeros(B, dtype=torch.int64, device="cuda")
        self.st = torch.zeros(B, dtype=torch.int32, device="cuda")

    def advance(self, irkgl, ctx, d, ns, h, order=None, stride=None):
        irkgl.irkgl_advance_multi(ctx, d, self.q, self.v, self.ql, self.vl, self.rp, ns, h=h,
                                  params=self.params, param_stride=self.params.shape[1] if stride is None
                                  else stride, order=order, H0=self.H0, dH_max=self.dH,
                                  iters=self.it, status=self.st)

    def snapshot(self):
        return {k: getattr(self, k).clone() for k in ("q", "v", "ql", "vl", "rp", "H0", "dH", "it", "st")}


@pytest.mark.parametrize("mix", [0, 1])
def test_per_trajectory_params_equal_separate_contexts(lib, mix):
    torch, irkgl = lib
    w = workloads.kepler_ensemble(batch=300, periods=1)
    mus = np.array([0.8, 1.0, 1.3])[np.arange(300) % 3]
    ns = torch.full((300,), 150, dtype=torch.int64, device="cuda")
    hh = torch.tensor(w["h"], device="cuda")
    # one call, three parameter sets, split into two chunks
    s = Slots(torch, w["q0"], w["v0"], 1)
    s.params.copy_(torch.tensor(mus[:, None]))
    ctx = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.1, mix=mix)
    for k in (70, 80):
        s.advance(irkgl, ctx.ctx, 2, torch.full((300,), k, dtype=torch.int64, device="cuda"), hh)
    torch.cuda.synchronize()
    for mu in (0.8, 1.0, 1.3):
        idx = np.flatnonzero(mus == mu)
        sel = torch.tensor(idx, device="cuda")
        ig = irkgl.Integrator(irkgl.RHS_KEPLER, [mu], 2, 0.1, mix=mix)
        out = ig.integrate(torch.tensor(w["q0"][idx], device="cuda"), torch.tensor(w["v0"][idx], device="cuda"),
                           nsteps=ns[sel], h=hh[sel])
        torch.cuda.synchronize()
        assert torch.equal(out.q, s.q[sel]) and torch.equal(out.v, s.v[sel])
        assert torch.equal(out.iters, s.it[sel]) and torch.equal(out.dH_max, s.dH[sel])
        assert torch.equal(out.status, s.st[sel])
        ig.close()
    ctx.close()


def test_nbody_masses_per_trajectory(lib):
    """Two 6-body systems with different masses in one launch of the
    register kernel: each gets the bits of its own context."""
    torch, irkgl = lib
    a = workloads.nbody_ensemble(copies=40, steps=60, seed_id=3)
    b = workloads.nbody_ensemble(copies=40, steps=60, seed_id=11)
    q0 = np.concatenate([a["q0"], b["q0"]])
    v0 = np.concatenate([a["v0"], b["v0"]])
    h = np.concatenate([a["h"], b["h"]])
    s = Slots(torch, q0, v0, 7)
    s.params[:40] = torch.tensor(a["params"], dtype=torch.float64)
    s.params[40:] = torch.tensor(b["params"], dtype=torch.float64)
    ctx = irkgl.Integrator(irkgl.RHS_NBODY, a["params"], 18, 0.1)
    ns = torch.full((80,), 60, dtype=torch.int64, device="cuda")
    s.advance(irkgl, ctx.ctx, 18, ns, torch.tensor(h, device="cuda"))
    torch.cuda.synchronize()
    for w, sl in ((a, slice(0, 40)), (b, slice(40, 80))):
        ig = irkgl.Integrator(irkgl.RHS_NBODY, w["params"], 18, 0.1)
        out = ig.integrate(torch.tensor(w["q0"], device="cuda"), torch.tensor(w["v0"], device="cuda"),
                           nsteps_all=60, h=torch.tensor(w["h"], device="cuda"))
        torch.cuda.synchronize()
        assert torch.equal(out.q, s.q[sl]) and torch.equal(out.iters, s.it[sl])
        assert torch.equal(out.dH_max, s.dH[sl])
        ig.close()
    ctx.close()


def test_order_skips_slots_and_status_is_final(lib):
    torch, irkgl = lib
    w = workloads.kepler_ensemble(batch=64, periods=1)
    s = Slots(torch, w["q0"], w["v0"], 1)
    s.params.fill_(1.0)
    s.st[5] = 1  # stopped in an earlier call
    before = s.snapshot()
    order = torch.tensor([i if i % 4 else -1 for i in range(64)], dtype=torch.int32, device="cuda")
    ctx = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.1, mix=1)
    s.advance(irkgl, ctx.ctx, 2, torch.full((64,), 30, dtype=torch.int64, device="cuda"),
              torch.tensor(w["h"], device="cuda"), order=order)
    torch.cuda.synchronize()
    after = s.snapshot()
    skipped = torch.arange(0, 64, 4, device="cuda")
    for k in before:
        assert torch.equal(before[k][skipped], after[k][skipped]) or \
            (k == "H0" and torch.isnan(after[k][skipped]).all()), k
    # the failed slot is not advanced and keeps its status
    for k in ("q", "v", "it"):
        assert torch.equal(before[k][5], after[k][5]), k
    assert int(after["st"][5]) == 1
    moved = [i for i in range(64) if i % 4 and i != 5]
    assert not torch.equal(before["q"][moved], after["q"][moved])
    assert (after["it"][moved] > 0).all() and torch.isfinite(after["H0"][moved]).all()
    # parameters given with a stride below the kind's count: rejected by the library
    P = ctypes.c_void_p
    ns = torch.full((64,), 1, dtype=torch.int64, device="cuda")
    hh = torch.tensor(w["h"], device="cuda")
    rc = irkgl.load().irkgl_advance_multi(
        P(ctx.ctx), *(P(t.data_ptr()) for t in (s.q, s.v, s.ql, s.vl, s.rp, hh, ns, s.params)), 0, None,
        P(s.H0.data_ptr()), None, None, None, 64, None)
    assert rc == irkgl.ERR_INVALID
    ctx.close()


def _ragged(torch, irkgl, dims, steps, team=256, mix=1, dmax=None):
    """FPUT chains of the given lengths as one packed ragged batch."""
    qs, vs, h = [], [], []
    for n in dims:
        c = workloads.fput_chain(n)
        qs.append(c["q"])
        vs.append(c["v"])
    off = np.concatenate([[0], np.cumsum(dims)[:-1]]).astype(np.int64)
    w = {"kind": np.full(len(dims), 3, np.int32), "dim": np.array(dims, np.int32), "offset": off,
         "param_offset": np.zeros(len(dims), np.int32), "nparams": np.ones(len(dims), np.int32),
         "h": np.full(len(dims), 0.25), "nsteps": np.full(len(dims), steps, np.int64)}
    ctx = irkgl.irkgl_create(irkgl.RHS_HARMONIC, [1.0], 1, 1.0)
    irkgl.irkgl_set_option(ctx, irkgl.OPT_WIDE_TEAM, team)
    irkgl.irkgl_set_option(ctx, irkgl.OPT_MIX, mix)
    out = irkgl.RaggedOutputs.allocate(int(sum(dims)), len(dims), device="cuda")
    irkgl.irkgl_integrate_ragged(ctx, irkgl.instances_tensor(w, "cuda"), len(dims), dmax or max(dims),
                                 torch.tensor([0.25], dtype=torch.float64, device="cuda"),
                                 torch.tensor(np.concatenate(qs), device="cuda"),
                                 torch.tensor(np.concatenate(vs), device="cuda"), out)
    torch.cuda.synchronize()
    irkgl.irkgl_destroy(ctx)
    return out, qs, vs


@pytest.mark.parametrize("mix", [0, 1])
def test_long_chains_on_the_recomputing_shape(lib, mix):
    """Chains of 1025..1536 particles (D up to 3072) run on the shape that
    forms c_i v again; against the oracle over the first 10 steps, and the
    shape gives the bits of the stored-c_i v shape on a chain both take."""
    torch, irkgl = lib
    dims = [1536, 1200, 1025, 1000]
    out, qs, vs = _ragged(torch, irkgl, dims, 10, mix=mix)
    assert (out.status.cpu().numpy() == 0).all()
    off = 0
    for n, q0, v0 in zip(dims, qs, vs):
        o = cbind.run(cbind.FPUT, [0.25], q0, v0, 0.25, 10)
        g = np.concatenate([out.q[off:off + n].cpu().numpy(), out.v[off:off + n].cpu().numpy()])
        e = np.concatenate([o["q"][0], o["v"][0]])
        assert np.abs(g - e).max() / np.abs(e).max() <= 1e-13, n
        off += n
    small, _, _ = _ragged(torch, irkgl, [1000], 10, mix=mix)             # dmax 1000: c_i v stored
    big, _, _ = _ragged(torch, irkgl, [1000], 10, mix=mix, dmax=1536)    # dmax 1536: formed again
    assert torch.equal(small.q, big.q) and torch.equal(small.v, big.v)
    assert torch.equal(small.iters, big.iters)


def test_ragged_advance_nan_h0_order_and_status(lib):
    """A packed batch advanced in two calls, one instance joining at the
    second call (NaN H0), one skipped by order, one stopped: the joining
    instance gets the bits of a fresh single-call run."""
    torch, irkgl = lib
    dims = [40, 64, 33]
    fresh, qs, vs = _ragged(torch, irkgl, dims, 30, team=64)
    off = np.concatenate([[0], np.cumsum(dims)[:-1]]).astype(np.int64)
    w = {"kind": np.full(3, 3, np.int32), "dim": np.array(dims, np.int32), "offset": off,
         "param_offset": np.zeros(3, np.int32), "nparams": np.ones(3, np.int32),
         "h": np.full(3, 0.25), "nsteps": np.zeros(3, np.int64)}
    f = dict(dtype=torch.float64, device="cuda")
    C = int(sum(dims))
    q = torch.tensor(np.concatenate(qs), **f)
    v = torch.tensor(np.concatenate(vs), **f)
    ql, vl, rp = torch.zeros(C, **f), torch.zeros(C, **f), torch.zeros(8 * C, **f)
    H0 = torch.full((3,), float("nan"), **f)
    dH = torch.zeros(3, **f)
    it = torch.zeros(3, dtype=torch.int64, device="cuda")
    st = torch.zeros(3, dtype=torch.int32, device="cuda")
    st[2] = 2
    ctx = irkgl.irkgl_create(irkgl.RHS_HARMONIC, [1.0], 1, 1.0)
    irkgl.irkgl_set_option(ctx, irkgl.OPT_WIDE_TEAM, 64)
    irkgl.irkgl_set_option(ctx, irkgl.OPT_MIX, 1)
    inst = irkgl.instances_tensor(w, "cuda")
    par = torch.tensor([0.25], **f)
    q2_before = q[off[2]:off[2] + dims[2]].clone()
    # call 1: instance 0 takes 12 steps, instance 1 is not listed
    order = torch.tensor([0, -1, 2], dtype=torch.int32, device="cuda")
    ns = torch.tensor([12, 0, 30], dtype=torch.int64, device="cuda")
    irkgl.irkgl_advance_ragged(ctx, inst, 3, 64, par, q, v, ql, vl, rp, ns, H0=H0, dH_max=dH, iters=it,
                               status=st, order=order)
    assert torch.isnan(H0[1]) and not torch.isnan(H0[0])
    # call 2: instance 0 continues, instance 1 joins
    ns = torch.tensor([18, 30, 30], dtype=torch.int64, device="cuda")
    irkgl.irkgl_advance_ragged(ctx, inst, 3, 64, par, q, v, ql, vl, rp, ns, H0=H0, dH_max=dH, iters=it,
                               status=st)
    torch.cuda.synchronize()
    irkgl.irkgl_destroy(ctx)
    for k in (0, 1):
        sl = slice(int(off[k]), int(off[k]) + dims[k])
        assert torch.equal(q[sl], fresh.q[sl]) and torch.equal(v[sl], fresh.v[sl]), k
        assert int(it[k]) == int(fresh.iters[k]) and float(dH[k]) == float(fresh.dH_max[k]), k
    assert int(st[2]) == 2 and int(it[2]) == 0
    assert torch.equal(q[off[2]:off[2] + dims[2]], q2_before)
