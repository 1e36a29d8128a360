"""Autotuner: step table and tile table for this GPU, written to tuning/gb300.json.

    python -m paper_2511_03655_gb300.autotune [--quick]

Step table.  The paper sets each problem's step where the local energy
error max_n |(H_n - H_{n-1})/H_{n-1}| (Eq. DHlocmax) is about 1e-14 (its
reference step size for Table tab:overhead).  For every (kind, size bucket)
the tuner runs short pilot integrations on the GPU with the local-error
monitor over a geometric ladder of steps and keeps the largest step whose
pilots all stay at or below the target: 1e-14, or twice the roundoff floor
of H where evaluating H in FP64 alone loses more than that (the floor is
the error at the smallest step of the ladder; N-body systems with many
pair terms reach it).  N-body steps are stored as a fraction of the
innermost orbital period; FPUT steps are absolute.

Tile table.  For the batched register kernel it times every compiled
lanes-per-trajectory tile on a pilot batch of each (kind, dim); for ragged
batches it times every team size of the wide kernel on a pilot batch of
each size bucket.  The fastest wins.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time

import numpy as np
import torch

from . import irkgl, workloads

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning", "gb300.json")
TARGET_LOCAL = 1e-14
WIDE_MAX_SLOTS = {32: 2, 64: 4, 128: 4, 256: 4}  # compiled wide-kernel shapes (k_wide.cu)


def load_table(path: str = TABLE) -> dict | None:
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return None


def _ragged(descs, steps):
    """Pack single-system instance descriptions into a ragged batch dict."""
    kinds, dims, hs, params, qs, vs = [], [], [], [], [], []
    for kind, p, q, v, h in descs:
        kinds.append(kind)
        dims.append(len(q))
        hs.append(h)
        params.append(p)
        qs.append(q)
        vs.append(v)
    offsets = np.concatenate([[0], np.cumsum(dims)[:-1]]).astype(np.int64)
    pc = np.array([len(p) for p in params])
    po = np.concatenate([[0], np.cumsum(pc)[:-1]]).astype(np.int32)
    return {"kind": np.array(kinds, np.int32), "dim": np.array(dims, np.int32), "offset": offsets,
            "param_offset": po, "nparams": pc.astype(np.int32), "h": np.array(hs),
            "nsteps": np.full(len(kinds), steps, np.int64),
            "params": np.concatenate([np.asarray(p, np.float64) for p in params]),
            "q0": np.concatenate(qs), "v0": np.concatenate(vs)}


def _run_ragged(w, team=0, local=False, timed=False):
    n = len(w["kind"])
    ctx = irkgl.irkgl_create(irkgl.RHS_HARMONIC, [1.0], 1, 0.1)
    irkgl.irkgl_set_option(ctx, irkgl.OPT_WIDE_TEAM, team)
    irkgl.irkgl_set_option(ctx, irkgl.OPT_MONITOR_LOCAL, 1 if local else 0)
    inst = irkgl.instances_tensor(w, "cuda")
    out = irkgl.RaggedOutputs.allocate(len(w["q0"]), n)
    args = (ctx, inst, n, int(w["dim"].max()), torch.tensor(w["params"], device="cuda"),
            torch.tensor(w["q0"], device="cuda"), torch.tensor(w["v0"], device="cuda"), out)
    irkgl.irkgl_integrate_ragged(*args)
    torch.cuda.synchronize()
    dt = None
    if timed:
        t0 = time.perf_counter()
        irkgl.irkgl_integrate_ragged(*args)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    irkgl.irkgl_destroy(ctx)
    return out, dt


def _pilot_dH(descs, steps) -> float:
    """Largest local energy error (Eq. DHlocmax) over the pilots; inf if any failed."""
    out, _ = _run_ragged(_ragged(descs, steps), local=True)
    if not (out.status.cpu().numpy() == 0).all():
        return math.inf
    return float(out.dH_max.cpu().numpy().max())


def _choose(ladder, dH):
    """Largest step of the ladder whose local error meets the target.  The
    target is 1e-14, raised to twice the roundoff floor (the error at the
    smallest step, where truncation is far below roundoff) when evaluating
    H in FP64 already loses more than that (N-body with many pair terms)."""
    floor = dH[0]
    target = max(TARGET_LOCAL, 2.0 * floor)
    ok = [x for x, e in zip(ladder, dH) if e <= target]
    return (max(ok) if ok else ladder[0]), floor, target, bool(ok)


def step_table(quick: bool = False) -> dict:
    pilots, steps = (4, 300) if quick else (8, 1000)
    table = {"nbody": {"fraction_of_inner_period": {}, "detail": {}},
             "fput": {"by_bucket": {}, "detail": {}}}
    # N-body: fraction of the innermost period
    fracs = [0.0025, 0.0035, 0.005, 0.007, 0.01, 0.014, 0.02]
    for nb in ([4, 8, 16] if quick else [3, 6, 12, 24, 48, 64]):
        dH = []
        for f in fracs:
            descs = []
            for k in range(pilots):
                sy = workloads.nbody_system(nb, seed_id=50000 + 97 * nb + k)
                descs.append((irkgl.RHS_NBODY, [1.0] + list(sy["masses"]), sy["q"], sy["v"],
                              f * sy["period_inner"]))
            dH.append(_pilot_dH(descs, steps))
        best, floor, target, met = _choose(fracs, dH)
        table["nbody"]["fraction_of_inner_period"][str(nb)] = best
        table["nbody"]["detail"][str(nb)] = {"dH_loc": dict(zip(map(str, fracs), dH)),
                                             "roundoff_floor": floor, "target": target, "met": met}
    # FPUT: absolute step per size bucket
    hs = [0.1, 0.15, 0.2, 0.3, 0.4, 0.5, 0.7, 1.0]
    for n in ([16, 128] if quick else [16, 32, 64, 128, 256, 512]):
        c = workloads.fput_chain(n)
        dH = []
        for h in hs:
            descs = [(irkgl.RHS_FPUT, c["params"], c["q"] * (1 + 1e-3 * k), c["v"], h)
                     for k in range(pilots)]
            dH.append(_pilot_dH(descs, steps))
        best, floor, target, met = _choose(hs, dH)
        table["fput"]["by_bucket"][str(n)] = best
        table["fput"]["detail"][str(n)] = {"dH_loc": dict(zip(map(str, hs), dH)),
                                           "roundoff_floor": floor, "target": target, "met": met}
    return table


def tile_table(quick: bool = False) -> dict:
    res = {"register": {}, "wide": {}}
    # register kernel, Kepler d = 2 (the ensemble)
    w = workloads.kepler_ensemble(batch=16384 if quick else 65536, periods=2)
    q0, v0 = torch.tensor(w["q0"], device="cuda"), torch.tensor(w["v0"], device="cuda")
    ns, hh = torch.tensor(w["nsteps"], device="cuda"), torch.tensor(w["h"], device="cuda")
    od = torch.tensor(workloads.similarity_order(w["e"]), device="cuda")
    times = {}
    for lpt in (1, 2, 4, 8):
        integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, lanes_per_traj=lpt)
        out = integ.integrate(q0, v0, nsteps=ns, h=hh, order=od)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        integ.integrate(q0, v0, out=out, nsteps=ns, h=hh, order=od)
        torch.cuda.synchronize()
        times[lpt] = time.perf_counter() - t0
        integ.close()
    res["register"]["kepler/2"] = {"lanes_per_traj": min(times, key=times.get),
                                   "seconds": {str(k): v for k, v in times.items()}}
    # wide kernel: team size per size bucket of a ragged batch (the buckets of
    # ragged.RaggedPlan); each bucket's pilot instances are timed alone
    from . import ragged
    wb = workloads.uneven_batch(ninst=256 if quick else 1024, steps=40 if quick else 100)
    plan = ragged.RaggedPlan(wb)
    wp = plan.permuted()
    params = torch.tensor(wb["params"], device="cuda")
    q0, v0 = torch.tensor(wb["q0"], device="cuda"), torch.tensor(wb["v0"], device="cuda")
    inst_all = irkgl.instances_tensor(wp, "cuda")
    out = irkgl.RaggedOutputs.allocate(len(wb["q0"]), len(wp["kind"]))
    for b in plan.buckets:
        inst = inst_all[b.start * ragged.INSTANCE_BYTES:(b.start + b.count) * ragged.INSTANCE_BYTES]
        tt = {}
        for team in (32, 64, 128, 256):
            if team * WIDE_MAX_SLOTS[team] < b.dmax:
                continue
            ctx = irkgl.irkgl_create(irkgl.RHS_HARMONIC, [1.0], 1, 0.1)
            irkgl.irkgl_set_option(ctx, irkgl.OPT_WIDE_TEAM, team)
            view = irkgl.RaggedOutputs(q=out.q, v=out.v, q_lo=out.q_lo, v_lo=out.v_lo, r_prev=out.r_prev,
                                       dH_max=out.dH_max[b.start:b.start + b.count],
                                       iters=out.iters[b.start:b.start + b.count],
                                       steps=out.steps[b.start:b.start + b.count],
                                       status=out.status[b.start:b.start + b.count])
            try:
                irkgl.irkgl_integrate_ragged(ctx, inst, b.count, b.dmax, params, q0, v0, view)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                irkgl.irkgl_integrate_ragged(ctx, inst, b.count, b.dmax, params, q0, v0, view)
                torch.cuda.synchronize()
                tt[team] = time.perf_counter() - t0
            except irkgl.IrkglError:
                pass  # shape not available for this dimension (shared memory)
            finally:
                irkgl.irkgl_destroy(ctx)
        res["wide"][b.label] = {"team": min(tt, key=tt.get), "seconds": {str(k): v for k, v in tt.items()},
                                "pilot_instances": b.count}
    return res


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--out", default=TABLE)
    a = ap.parse_args(argv)
    irkgl.load()
    t0 = time.time()
    table = {"device": torch.cuda.get_device_name(), "target_local_dH": TARGET_LOCAL,
             "step_table": step_table(a.quick), "tiles": tile_table(a.quick),
             "seconds": None}
    table["seconds"] = time.time() - t0
    os.makedirs(os.path.dirname(a.out), exist_ok=True)
    with open(a.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps(table, indent=1, sort_keys=True))


if __name__ == "__main__":
    main()
