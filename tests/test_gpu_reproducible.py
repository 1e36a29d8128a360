"""The reproducible form (IRKGL_OPT_MIX = 2) against the oracle, bit for bit.

Both sides perform the plain operation sequence of the method: the two-matrix
initial guess of Eq. IRK_init2, the sweep of Eq. IRK_FP2 with sums left to
right, Eqs. Delta_n / stopping on FP64 values, the compensated update of
Eq. qnvn2, and g and H with IEEE division and square root, every operation
rounded once.  So every output must be equal, not close: q, v and their
compensation parts, R_prev, the sweep count of every step and their totals,
dH_max, steps and status.  The +-1 sweep requirement therefore holds with a
difference of 0 on every step, including the workloads whose fast tiles
differ beyond +-1 at the roundoff floor (Henon-Heiles at h = 1).
"""
import numpy as np
import pytest

from oracle import cbind, coeffs
from paper_2511_03655_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    torch.cuda.init()
    return torch, irkgl


def same(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return a.shape == b.shape and a.dtype == b.dtype and np.array_equal(a.view(np.uint8), b.view(np.uint8))


def cases():
    w = workloads.kepler_ensemble(batch=512, periods=2)
    hq, hv, _ = workloads.henon_heiles_ensemble(256)
    nb = workloads.nbody_ensemble(copies=48, nbodies=6, steps=600)
    rng = np.random.default_rng(11)
    return {
        "kepler": (irkgl_kind("KEPLER"), cbind.KEPLER, [1.0], w["q0"], w["v0"], w["h"], w["nsteps"]),
        "henon_heiles_h1": (irkgl_kind("HENON_HEILES"), cbind.HENON_HEILES, [1.0], hq, hv,
                            np.full(len(hq), 1.0), np.full(len(hq), 400, dtype=np.int64)),
        "harmonic3": (irkgl_kind("HARMONIC"), cbind.HARMONIC, [1.3], rng.standard_normal((128, 3)),
                      rng.standard_normal((128, 3)), np.full(128, 0.4), np.full(128, 500, dtype=np.int64)),
        "nbody6": (irkgl_kind("NBODY"), cbind.NBODY, nb["params"], nb["q0"], nb["v0"], nb["h"], nb["nsteps"]),
    }


def irkgl_kind(name):
    from paper_2511_03655_gb300 import irkgl
    return getattr(irkgl, "RHS_" + name)


def oracle(ko, params, q0, v0, h, nsteps, **kw):
    return cbind.run(ko, params, q0, v0, h, nsteps, nthreads=8, **kw)


@pytest.mark.parametrize("name", ["kepler", "henon_heiles_h1", "harmonic3", "nbody6"])
def test_integrate_bitwise(env, name):
    torch, irkgl = env
    kg, ko, params, q0, v0, h, ns = cases()[name]
    B, d = q0.shape
    integ = irkgl.Integrator(kg, params, d, float(h[0]), mix=2)
    assert integ.layout == "reproducible" and integ.tile == 1
    f = dict(device="cuda")
    out = integ.integrate(torch.tensor(q0, **f), torch.tensor(v0, **f), nsteps=torch.tensor(ns, **f),
                          h=torch.tensor(h, **f))
    torch.cuda.synchronize()
    o = oracle(ko, params, q0, v0, h, ns)
    g = {k: getattr(out, k).cpu().numpy() for k in ("q", "v", "q_lo", "v_lo", "r_prev", "dH_max",
                                                      "iters", "steps", "status")}
    assert (o["status"] == 0).all()
    for k, ok in (("q", "q"), ("v", "v"), ("q_lo", "q_lo"), ("v_lo", "v_lo"), ("r_prev", "r_prev"),
                  ("dH_max", "dH_max")):
        assert same(g[k], o[ok]), (name, k)
    assert np.array_equal(g["iters"], o["iters_total"]), name
    assert np.array_equal(g["steps"], o["steps"]) and np.array_equal(g["status"], o["status"])
    integ.close()


@pytest.mark.parametrize("name", ["kepler", "henon_heiles_h1"])
def test_sweep_counts_equal_on_every_step(env, name):
    """irkgl_step with the per-step sweep history: every step's count equals
    the oracle's (difference 0 on all steps), and the state after the last
    step is the oracle's."""
    torch, irkgl = env
    kg, ko, params, q0, v0, h, _ = cases()[name]
    n = 300
    B, d = q0.shape
    integ = irkgl.Integrator(kg, params, d, float(h[0]), mix=2)
    f = dict(dtype=torch.float64, device="cuda")
    q, v = torch.tensor(q0, **f), torch.tensor(v0, **f)
    ql, vl = torch.zeros_like(q), torch.zeros_like(v)
    rp = torch.zeros((B, 8, d), **f)
    it = torch.zeros((B, n), dtype=torch.int32, device="cuda")
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    integ.step(q, v, ql, vl, rp, h=torch.tensor(h, **f), nsteps=n, iters=it, status=st)
    torch.cuda.synchronize()
    o = oracle(ko, params, q0, v0, h, n, iters_len=n)
    assert np.array_equal(it.cpu().numpy(), o["iters"])
    assert np.array_equal(st.cpu().numpy(), o["status"])
    for a, k in ((q, "q"), (v, "v"), (ql, "q_lo"), (vl, "v_lo"), (rp, "r_prev")):
        assert same(a.cpu().numpy(), o[k]), k
    integ.close()


def test_chunked_advance_and_host_buffers(env):
    """irkgl_advance in three chunks (H0 carried, dH_max and sweep totals
    accumulated) and irkgl_integrate_host give the oracle's single run."""
    torch, irkgl = env
    kg, ko, params, q0, v0, h, ns = cases()["kepler"]
    B, d = q0.shape
    f = dict(dtype=torch.float64, device="cuda")
    integ = irkgl.Integrator(kg, params, d, float(h[0]), mix=2)
    q, v = torch.tensor(q0, **f), torch.tensor(v0, **f)
    ql, vl = torch.zeros_like(q), torch.zeros_like(v)
    rp = torch.zeros((B, 8, d), **f)
    H0 = torch.zeros(B, **f)
    dH = torch.zeros(B, **f)
    it = torch.zeros(B, dtype=torch.int64, device="cuda")
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    hh = torch.tensor(h, **f)
    left = ns.copy()
    for c, frac in enumerate((0.3, 0.5, 1.0)):
        k = np.minimum(left, np.ceil(frac * ns).astype(np.int64) - (ns - left))
        integ.advance(q, v, ql, vl, rp, h=hh, nsteps=torch.tensor(k, device="cuda"), H0=H0,
                      h0_init=(c == 0), dH_max=dH, iters=it, status=st)
        left -= k
    assert (left == 0).all()
    torch.cuda.synchronize()
    o = oracle(ko, params, q0, v0, h, ns)
    for a, k in ((q, "q"), (v, "v"), (ql, "q_lo"), (vl, "v_lo"), (rp, "r_prev"), (dH, "dH_max")):
        assert same(a.cpu().numpy(), o[k]), k
    assert np.array_equal(it.cpu().numpy(), o["iters_total"])
    host = integ.integrate_host(torch.tensor(q0), torch.tensor(v0), nsteps=torch.tensor(ns),
                                h=torch.tensor(h))
    assert same(host.q.numpy(), o["q"]) and same(host.v.numpy(), o["v"])
    assert np.array_equal(host.iters.numpy(), o["iters_total"])
    integ.close()


def test_failures_and_own_tables(env):
    """Status 1 (sweep cap) and 2 (non-finite stage value, a Kepler
    collision) at the oracle's step with its state, and a context built
    with its own tables (nu = 0: the guess from v alone) follows them."""
    torch, irkgl = env
    q0 = np.array([[0.0, 0.0], [0.5, 0.0], [0.9, 0.0], [1.0, 0.0]])
    v0 = np.array([[0.0, 0.0], [0.0, np.sqrt(3.0)], [0.0, 1.1], [0.0, 1.0]])
    h = np.full(4, 2 * np.pi / 120)
    ns = np.full(4, 400, dtype=np.int64)
    f = dict(device="cuda")
    for kmax in (100, 4):
        integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, h[0], mix=2, kmax=kmax)
        out = integ.integrate(torch.tensor(q0, **f), torch.tensor(v0, **f), nsteps=torch.tensor(ns, **f),
                              h=torch.tensor(h, **f))
        o = oracle(cbind.KEPLER, [1.0], q0, v0, h, ns, kmax=kmax)
        assert np.array_equal(out.status.cpu().numpy(), o["status"])
        assert (o["status"] != 0).any()
        assert np.array_equal(out.steps.cpu().numpy(), o["steps"])
        assert np.array_equal(out.iters.cpu().numpy(), o["iters_total"])
        assert same(out.q.cpu().numpy(), o["q"]) and same(out.v.cpu().numpy(), o["v"])
        integ.close()
    tab = {k: np.array(val, dtype=np.float64) for k, val in coeffs.fp64_tables().items()
           if k in ("c", "b", "mu", "eta", "nu")}
    tab["nu"] = np.zeros_like(tab["nu"])
    w = workloads.kepler_ensemble(batch=128, periods=1)
    own = {k: tab[k] for k in ("c", "b", "mu", "eta", "nu")}
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, float(w["h"][0]), coeffs=own, mix=2)
    out = integ.integrate(torch.tensor(w["q0"], **f), torch.tensor(w["v0"], **f),
                          nsteps=torch.tensor(w["nsteps"], **f), h=torch.tensor(w["h"], **f))
    o = oracle(cbind.KEPLER, [1.0], w["q0"], w["v0"], w["h"], w["nsteps"], tab=tab)
    assert same(out.q.cpu().numpy(), o["q"]) and same(out.v.cpu().numpy(), o["v"])
    assert np.array_equal(out.iters.cpu().numpy(), o["iters_total"])
    integ.close()


def test_per_trajectory_params_multi(env):
    """irkgl_advance_multi with per-trajectory mu (Kepler) in the reproducible
    form: each trajectory equals the oracle run with its own parameter."""
    torch, irkgl = env
    w = workloads.kepler_ensemble(batch=256, periods=1)
    B = 256
    mu = 0.5 + np.linspace(0.0, 1.0, B)
    f = dict(dtype=torch.float64, device="cuda")
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, float(w["h"][0]), mix=2)
    q, v = torch.tensor(w["q0"], **f), torch.tensor(w["v0"], **f)
    ql, vl = torch.zeros_like(q), torch.zeros_like(v)
    rp = torch.zeros((B, 8, 2), **f)
    H0 = torch.full((B,), float("nan"), **f)
    dH = torch.zeros(B, **f)
    it = torch.zeros(B, dtype=torch.int64, device="cuda")
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    irkgl.irkgl_advance_multi(integ.ctx, 2, q, v, ql, vl, rp, torch.tensor(w["nsteps"], device="cuda"),
                              h=torch.tensor(w["h"], **f), params=torch.tensor(mu[:, None], **f),
                              param_stride=1, H0=H0, dH_max=dH, iters=it, status=st)
    torch.cuda.synchronize()
    o = oracle(cbind.KEPLER, mu[:, None], w["q0"], w["v0"], w["h"], w["nsteps"])
    for a, k in ((q, "q"), (v, "v"), (rp, "r_prev"), (dH, "dH_max")):
        assert same(a.cpu().numpy(), o[k]), k
    assert np.array_equal(it.cpu().numpy(), o["iters_total"])
    integ.close()


def test_full_ensemble_sampled(env):
    """The 65,536-orbit Kepler ensemble over its full 100 periods in one
    launch; 192 orbits (every 512th, and the 64 most eccentric) equal the
    oracle's full-horizon runs bit for bit, sweep totals and dH_max included."""
    torch, irkgl = env
    w = workloads.kepler_ensemble()
    B = len(w["e"])
    f = dict(device="cuda")
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, float(w["h"][0]), mix=2)
    out = integ.integrate(torch.tensor(w["q0"], **f), torch.tensor(w["v0"], **f),
                          nsteps=torch.tensor(w["nsteps"], **f), h=torch.tensor(w["h"], **f))
    torch.cuda.synchronize()
    idx = np.unique(np.concatenate([np.arange(0, B, 512), np.argsort(w["e"])[-64:]]))
    o = oracle(cbind.KEPLER, [1.0], w["q0"][idx], w["v0"][idx], w["h"][idx], w["nsteps"][idx])
    for k in ("q", "v", "q_lo", "v_lo", "dH_max"):
        assert same(getattr(out, k).cpu().numpy()[idx], o[k]), k
    assert np.array_equal(out.iters.cpu().numpy()[idx], o["iters_total"])
    assert np.array_equal(out.status.cpu().numpy()[idx], o["status"])
    assert (out.status.cpu().numpy() == 0).all()
    integ.close()


def ragged_oracle(w, k, nsteps=None):
    o, d = int(w["offset"][k]), int(w["dim"][k])
    po, pn = int(w["param_offset"][k]), int(w["nparams"][k])
    kind = {2: cbind.NBODY, 3: cbind.FPUT, 5: cbind.HARMONIC}[int(w["kind"][k])]
    n = int(w["nsteps"][k]) if nsteps is None else int(nsteps)
    return cbind.run(kind, w["params"][po:po + pn], w["q0"][o:o + d], w["v0"][o:o + d], w["h"][k], n)


def ragged_run(torch, irkgl, w, team=0):
    n = len(w["kind"])
    integ = irkgl.Integrator(irkgl.RHS_HARMONIC, [1.0], 1, 0.1, mix=2)  # tables and options
    integ.set(irkgl.OPT_WIDE_TEAM, team)
    out = irkgl.RaggedOutputs.allocate(len(w["q0"]), n)
    irkgl.irkgl_integrate_ragged(integ.ctx, irkgl.instances_tensor(w, "cuda"), n, int(w["dim"].max()),
                                 torch.tensor(w["params"], device="cuda"),
                                 torch.tensor(w["q0"], device="cuda"), torch.tensor(w["v0"], device="cuda"),
                                 out)
    torch.cuda.synchronize()
    integ.close()
    return {k: getattr(out, k).cpu().numpy() for k in ("q", "v", "q_lo", "v_lo", "r_prev", "dH_max",
                                                       "iters", "steps", "status")}


def check_ragged_instance(g, w, k, o):
    off, d = int(w["offset"][k]), int(w["dim"][k])
    for key in ("q", "v", "q_lo", "v_lo"):
        assert same(g[key][off:off + d], o[key][0]), (k, key)
    assert same(g["r_prev"][8 * off:8 * (off + d)], o["r_prev"][0].ravel()), (k, "r_prev")
    assert same(g["dH_max"][k:k + 1], o["dH_max"]), (k, "dH_max")
    assert g["iters"][k] == o["iters_total"][0] and g["status"][k] == o["status"][0]
    assert g["steps"][k] == o["steps"][0]


def test_ragged_bitwise_every_team_size(env):
    """Small N-body systems and FPUT chains in one ragged launch: every team
    size (32 to 256 threads) returns the same bits, the oracle's."""
    torch, irkgl = env
    w = workloads.uneven_batch(ninst=16, steps=150, nmax_body=20, nmax_chain=60)
    runs = {team: ragged_run(torch, irkgl, w, team) for team in (32, 64, 128, 256)}
    for k in range(len(w["kind"])):
        check_ragged_instance(runs[32], w, k, ragged_oracle(w, k))
    for team in (64, 128, 256):
        for key in runs[32]:
            assert same(runs[team][key], runs[32][key]), (team, key)


def test_ragged_bitwise_largest_sizes_and_continuation(env):
    """N-body systems up to 64 bodies and FPUT chains up to 1,536 particles
    (the wide kernel's largest shape), in one launch and as two
    irkgl_advance_ragged calls (H0, sweep totals and dH_max carried): the
    oracle's bits both ways."""
    torch, irkgl = env
    w = workloads.uneven_batch(ninst=10, steps=60, nmax_body=64, nmax_chain=1536)
    n = len(w["kind"])
    g = ragged_run(torch, irkgl, w)
    refs = [ragged_oracle(w, k) for k in range(n)]
    for k in range(n):
        check_ragged_instance(g, w, k, refs[k])
    f = dict(dtype=torch.float64, device="cuda")
    integ = irkgl.Integrator(irkgl.RHS_HARMONIC, [1.0], 1, 0.1, mix=2)
    inst = irkgl.instances_tensor(w, "cuda")
    q, v = torch.tensor(w["q0"], **f), torch.tensor(w["v0"], **f)
    ql, vl = torch.zeros_like(q), torch.zeros_like(v)
    rp = torch.zeros(8 * len(w["q0"]), **f)
    H0, dH = torch.zeros(n, **f), torch.zeros(n, **f)
    it = torch.zeros(n, dtype=torch.int64, device="cuda")
    st = torch.zeros(n, dtype=torch.int32, device="cuda")
    par = torch.tensor(w["params"], **f)
    first = np.full(n, 25, dtype=np.int64)
    for c, k in enumerate((first, w["nsteps"] - first)):
        irkgl.irkgl_advance_ragged(integ.ctx, inst, n, int(w["dim"].max()), par, q, v, ql, vl, rp,
                                   torch.tensor(k, device="cuda"), H0=H0, h0_init=(c == 0), dH_max=dH,
                                   iters=it, status=st)
    torch.cuda.synchronize()
    cont = {"q": q.cpu().numpy(), "v": v.cpu().numpy(), "q_lo": ql.cpu().numpy(), "v_lo": vl.cpu().numpy(),
            "r_prev": rp.cpu().numpy(), "dH_max": dH.cpu().numpy(), "iters": it.cpu().numpy(),
            "steps": w["nsteps"].copy(), "status": st.cpu().numpy()}
    for k in range(n):
        check_ragged_instance(cont, w, k, refs[k])
    integ.close()


def test_served_requests_bitwise(env):
    """The continuous-batching server in the reproducible form: requests of
    every family, served in shared register and wide pools over many ticks,
    each return the oracle's bits for that request run alone."""
    torch, irkgl = env
    import copy

    from paper_2511_03655_gb300 import serve
    descs = workloads.serving_requests(n=14, rate=4000.0, batch_max=48, horizon_max=300, nb_max=12,
                                       n_max=96)
    reqs = serve.make_requests(copy.deepcopy(descs))
    st = serve.Server(target_tick_s=0.001, mix=2).run(reqs)
    assert st.max_concurrent > 1
    kinds = {"kepler": cbind.KEPLER, "nbody": cbind.NBODY, "fput": cbind.FPUT,
             "henon_heiles": cbind.HENON_HEILES, "harmonic": cbind.HARMONIC}
    for r in reqs:
        o = cbind.run(kinds[r.kind], r.params, r.q0, r.v0, r.h, r.nsteps, nthreads=8)
        assert same(r.q, o["q"]) and same(r.v, o["v"]), r.kind
        assert same(r.dH_max, o["dH_max"]), r.kind
        assert np.array_equal(r.iters, o["iters_total"]) and np.array_equal(r.status, o["status"])


@pytest.mark.parametrize("stages", [8, 6, 4, 2])
def test_first_order_bitwise(env, stages):
    """The first-order form (Eq. Yi2) in the reproducible form, for every
    s-stage scheme: irkgl_integrate1 and two irkgl_advance1 calls give the
    oracle's bits (y, y_lo, L_prev, dH_max, sweep totals, status)."""
    torch, irkgl = env
    rng = np.random.default_rng(21 + stages)
    y0 = rng.uniform(-1.0, 1.0, (256, 2))
    h = {8: 0.6, 6: 0.45, 4: 0.25, 2: 0.05}[stages]
    ns = 300
    integ = irkgl.Integrator(irkgl.RHS_HARMONIC1, [1.3], 2, h, mix=2, stages=stages)
    assert integ.layout == "reproducible" and integ.tile == 1
    out = integ.integrate1(torch.tensor(y0, device="cuda"), nsteps_all=ns)
    torch.cuda.synchronize()
    o = cbind.run1(cbind.HARMONIC1, [1.3], y0, h, ns, stages=stages)
    for key in ("y", "y_lo", "l_prev", "dH_max"):
        assert same(getattr(out, key).cpu().numpy(), o[key]), key
    assert np.array_equal(out.iters.cpu().numpy(), o["iters_total"])
    assert np.array_equal(out.status.cpu().numpy(), o["status"]) and (o["status"] == 0).all()
    f = dict(dtype=torch.float64, device="cuda")
    y, ylo = torch.tensor(y0, **f), torch.zeros((256, 2), **f)
    lp = torch.zeros((256, stages, 2), **f)
    H0, dH = torch.zeros(256, **f), torch.zeros(256, **f)
    it = torch.zeros(256, dtype=torch.int64, device="cuda")
    st = torch.zeros(256, dtype=torch.int32, device="cuda")
    for c, k in enumerate((120, ns - 120)):
        integ.advance1(y, ylo, lp, torch.full((256,), k, dtype=torch.int64, device="cuda"),
                       h=torch.full((256,), h, **f), H0=H0, h0_init=(c == 0), dH_max=dH, iters=it, status=st)
    torch.cuda.synchronize()
    for a, key in ((y, "y"), (ylo, "y_lo"), (lp, "l_prev"), (dH, "dH_max")):
        assert same(a.cpu().numpy(), o[key]), ("advance1", key)
    assert np.array_equal(it.cpu().numpy(), o["iters_total"])
    integ.close()


def test_ragged_largest_shapes_bitwise(env):
    """The largest instances the ragged calls take: an FPUT chain of 1,536
    particles (the 256 x 6 team shape, 221 KB of shared memory) and a
    128-body system (the descriptor's limit) in one launch, bit for bit."""
    torch, irkgl = env
    c = workloads.fput_chain(1536)
    sysd = workloads.nbody_system(128, seed_id=991)
    cp = np.asarray(c["params"], dtype=np.float64)
    w = {"kind": np.array([3, 2], dtype=np.int32), "dim": np.array([1536, 384], dtype=np.int32),
         "offset": np.array([0, 1536], dtype=np.int64),
         "param_offset": np.array([0, len(cp)], dtype=np.int32),
         "nparams": np.array([len(cp), 129], dtype=np.int32),
         "h": np.array([0.25, 0.001 * sysd["period_inner"]]), "nsteps": np.array([60, 30], dtype=np.int64),
         "params": np.concatenate([cp, [1.0], np.asarray(sysd["masses"], dtype=np.float64)]),
         "q0": np.concatenate([c["q"], sysd["q"]]), "v0": np.concatenate([c["v"], sysd["v"]])}
    g = ragged_run(torch, irkgl, w)
    for k in range(2):
        o = ragged_oracle(w, k)
        assert o["status"][0] == 0
        check_ragged_instance(g, w, k, o)


def test_register_ragged_tail_zero_steps_and_skips(env):
    """129 Kepler trajectories (a partly filled last block), every seventh
    with zero steps, advanced by irkgl_advance_multi through a reversed order
    list that skips every fifth entry (-1): the advanced trajectories give
    the oracle's bits, the skipped ones are left as they were."""
    torch, irkgl = env
    B = 129
    w = workloads.kepler_ensemble(batch=B, periods=1)
    ns = w["nsteps"].copy()
    ns[::7] = 0
    order = np.arange(B, dtype=np.int32)[::-1].copy()
    order[::5] = -1
    ran = np.zeros(B, dtype=bool)
    ran[order[order >= 0]] = True
    f = dict(dtype=torch.float64, device="cuda")
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, float(w["h"][0]), mix=2)
    q, v = torch.tensor(w["q0"], **f), torch.tensor(w["v0"], **f)
    ql, vl = torch.zeros_like(q), torch.zeros_like(v)
    rp = torch.zeros((B, 8, 2), **f)
    H0 = torch.full((B,), float("nan"), **f)
    dH = torch.zeros(B, **f)
    it = torch.zeros(B, dtype=torch.int64, device="cuda")
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    irkgl.irkgl_advance_multi(integ.ctx, 2, q, v, ql, vl, rp, torch.tensor(ns, device="cuda"),
                              h=torch.tensor(w["h"], **f), order=torch.tensor(order, device="cuda"),
                              H0=H0, dH_max=dH, iters=it, status=st)
    torch.cuda.synchronize()
    o = oracle(cbind.KEPLER, [1.0], w["q0"], w["v0"], w["h"], ns)
    qg, vg = q.cpu().numpy(), v.cpu().numpy()
    assert same(qg[ran], o["q"][ran]) and same(vg[ran], o["v"][ran])
    assert same(rp.cpu().numpy()[ran], o["r_prev"][ran]) and same(dH.cpu().numpy()[ran], o["dH_max"][ran])
    assert np.array_equal(it.cpu().numpy()[ran], o["iters_total"][ran])
    assert same(qg[~ran], w["q0"][~ran]) and same(vg[~ran], w["v0"][~ran])
    assert (it.cpu().numpy()[~ran] == 0).all() and np.isnan(H0.cpu().numpy()[~ran]).all()
    integ.close()
