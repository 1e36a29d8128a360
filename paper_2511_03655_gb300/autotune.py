"""Autotuner: step table and tile table for this GPU, written to tuning/gb300.json.

    python -m paper_2511_03655_gb300.autotune [--quick]

Step table.  The paper sets each problem's step where the local energy
error max_n |(H_n - H_{n-1})/H_{n-1}| (Eq. DHlocmax) is about 1e-14 (its
reference step size for Table tab:overhead).  For every (kind, size bucket)
the tuner runs short pilot integrations on the GPU with the local-error
monitor over a geometric ladder of steps and keeps the largest step whose
pilots all stay at or below 1e-14.  N-body steps are stored as a fraction
of the innermost orbital period; FPUT steps are absolute.

Tile table.  For the batched register kernel it times every compiled
lanes-per-trajectory tile on a pilot batch of each (kind, dim); for ragged
batches it times every team size of the wide kernel on a pilot batch of
each size bucket.  The fastest wins.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np
import torch

from . import irkgl, workloads

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning", "gb300.json")
TARGET_LOCAL = 1e-14


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


def step_table(quick: bool = False) -> dict:
    pilots, steps = (4, 300) if quick else (8, 1000)
    table = {"nbody": {"fraction_of_inner_period": {}}, "fput": {"by_bucket": {}}}
    # N-body: fraction of the innermost period
    fracs = [0.0025, 0.0035, 0.005, 0.007, 0.01]
    for nb in ([4, 8, 16] if quick else [3, 6, 12, 24, 48, 64]):
        best = fracs[0]
        for f in fracs:
            descs = []
            for k in range(pilots):
                s = workloads.nbody_system(nb, seed_id=50000 + 97 * nb + k)
                descs.append((irkgl.RHS_NBODY, [1.0] + list(s["masses"]), s["q"], s["v"],
                              f * s["period_inner"]))
            out, _ = _run_ragged(_ragged(descs, steps), local=True)
            ok = (out.status.cpu().numpy() == 0).all() and out.dH_max.cpu().numpy().max() <= TARGET_LOCAL
            if ok:
                best = f
        table["nbody"]["fraction_of_inner_period"][str(nb)] = best
    # FPUT: absolute step per size bucket
    hs = [0.1, 0.15, 0.2, 0.3, 0.4, 0.5]
    for n in ([16, 128] if quick else [16, 32, 64, 128, 256, 512]):
        best = hs[0]
        for h in hs:
            c = workloads.fput_chain(n)
            descs = [(irkgl.RHS_FPUT, c["params"], c["q"] * (1 + 1e-3 * k), c["v"], h)
                     for k in range(pilots)]
            out, _ = _run_ragged(_ragged(descs, steps), local=True)
            ok = (out.status.cpu().numpy() == 0).all() and out.dH_max.cpu().numpy().max() <= TARGET_LOCAL
            if ok:
                best = h
        table["fput"]["by_bucket"][str(n)] = best
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
    # wide kernel: team size per size bucket of a ragged batch
    for label, kw in (("nbody<=64", dict(nmax_body=64, nmax_chain=8)),
                      ("fput<=512", dict(nmax_body=3, nmax_chain=512))):
        wb = workloads.uneven_batch(ninst=64 if quick else 256, steps=100, **kw)
        wb = {k: (v[wb["kind"] == (2 if label.startswith("nbody") else 3)]
                  if isinstance(v, np.ndarray) and len(v) == len(wb["kind"]) else v)
              for k, v in wb.items()}
        # re-pack after filtering
        descs = []
        for k in range(len(wb["kind"])):
            o, d = int(wb["offset"][k]), int(wb["dim"][k])
            po, pn = int(wb["param_offset"][k]), int(wb["nparams"][k])
            descs.append((int(wb["kind"][k]), wb["params"][po:po + pn], wb["q0"][o:o + d],
                          wb["v0"][o:o + d], float(wb["h"][k])))
        rb = _ragged(descs, 100)
        tt = {}
        for team in (32, 64, 128, 256):
            if team * (2 if team in (32, 256) else 4) < int(rb["dim"].max()):
                continue
            _, dt = _run_ragged(rb, team=team, timed=True)
            tt[team] = dt
        res["wide"][label] = {"team": min(tt, key=tt.get), "seconds": {str(k): v for k, v in tt.items()}}
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
