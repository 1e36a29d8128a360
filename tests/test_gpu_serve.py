"""The continuous-batching server: every request's result is the same alone and
in the mix (bitwise: a chunked run continues exactly), the requests of a pool
share one launch per tick, admission respects each pool's capacity, a
failure is final, and results agree with the oracle."""
import copy

import numpy as np
import pytest

from oracle import cbind
from paper_2511_03655_gb300 import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def server_mod():
    import torch
    from paper_2511_03655_gb300 import build, irkgl, serve
    build.build()
    irkgl.load()
    torch.cuda.init()
    return serve


def small_requests(n=14, rate=4000.0):
    return workloads.serving_requests(n=n, rate=rate, batch_max=64, horizon_max=400, nb_max=12,
                                      n_max=96)


def same(a, b, dH=True):
    ok = np.array_equal(a.q, b.q) and np.array_equal(a.v, b.v) and np.array_equal(a.iters, b.iters)
    ok = ok and np.array_equal(a.status, b.status)
    return ok and (np.array_equal(a.dH_max, b.dH_max) if dH else True)


def test_result_same_alone_and_in_mix(server_mod):
    serve = server_mod
    descs = small_requests()
    mix = serve.make_requests(copy.deepcopy(descs))
    st = serve.Server(target_tick_s=0.002).run(mix)
    assert st.summary()["requests"] == len(descs)
    assert st.max_concurrent > 1  # requests really overlapped
    for d, r in zip(descs, mix):
        alone = serve.make_requests([copy.deepcopy(d)])
        serve.Server(target_tick_s=0.0003).run(alone)  # different chunking too
        a = alone[0]
        assert (r.status == 0).all() and (a.status == 0).all()
        assert same(r, a), d["kind"]


@pytest.mark.parametrize("stage_mix", [0, 1])
def test_mix_matches_single_launch(server_mod, stage_mix):
    """Served in chunks among other requests, every request gets the bits of
    one uninterrupted launch, with either stage mixing."""
    serve = server_mod
    descs = small_requests(8)
    mix = serve.make_requests(copy.deepcopy(descs))
    serve.Server(target_tick_s=0.001, mix=stage_mix).run(mix)
    plain = serve.make_requests(copy.deepcopy(descs))
    serve.run_plain(plain, mix=stage_mix)
    for r, p in zip(mix, plain):
        assert same(r, p), r.kind


def test_one_launch_per_pool_per_tick(server_mod):
    """Many requests, few pools: every tick launches at most one kernel per
    pool, so the launches do not grow with the number of requests in flight."""
    serve = server_mod
    descs = workloads.serving_requests(n=60, rate=20000.0, batch_max=32, horizon_max=300,
                                       families=("kepler", "fput"), n_max=60)
    reqs = serve.make_requests(copy.deepcopy(descs))
    srv = serve.Server(target_tick_s=0.002)
    st = srv.run(reqs).summary()
    assert st["requests"] == 60
    assert st["launches_per_tick"] <= st["pools"] <= 2
    assert st["max_concurrent_requests"] > 10
    assert st["gpu_launches"] < sum(1 for _ in reqs) * 3  # not one launch per request and chunk
    assert 0.0 < st["gpu_busy"] <= 1.0
    srv.close()


def test_admission_by_pool_capacity(server_mod):
    """With pools that hold only a few requests, the others wait for room,
    every request completes, and the results are those of roomy pools."""
    serve = server_mod
    descs = small_requests(12)
    reqs = serve.make_requests(copy.deepcopy(descs))
    big = max(r.device_bytes() for r in reqs)
    st = serve.Server(pool_bytes=1, target_tick_s=0.001).run(reqs)  # each pool: 2x its largest request
    assert st.summary()["requests"] == 12 and all(r.q is not None for r in reqs)
    roomy = serve.make_requests(copy.deepcopy(descs))
    st2 = serve.Server(pool_bytes=64 * big, target_tick_s=0.001).run(roomy)
    assert st2.max_concurrent >= st.max_concurrent
    for a, b in zip(reqs, roomy):
        assert same(a, b)


@pytest.mark.parametrize("stage_mix", [0, 1])
def test_served_results_match_oracle(server_mod, stage_mix):
    serve = server_mod
    descs = [d for d in small_requests(20) if d["kind"] in ("kepler", "fput")][:4]
    reqs = serve.make_requests(copy.deepcopy(descs))
    serve.Server(target_tick_s=0.001, mix=stage_mix).run(reqs)
    for r in reqs:
        kind = cbind.KEPLER if r.kind == "kepler" else cbind.FPUT
        o = cbind.run(kind, r.params, r.q0, r.v0, r.h, r.nsteps, nthreads=8)
        g = np.concatenate([r.q, r.v], axis=1)
        e = np.concatenate([o["q"], o["v"]], axis=1)
        assert (np.abs(g - e).max(axis=1) / np.abs(e).max(axis=1)).max() <= 1e-11, r.kind


def test_failure_is_final_and_zero_steps(server_mod):
    """A trajectory that fails (a Kepler collision: non-finite stage values)
    keeps its status and sweep total across ticks, as in one launch; a
    request of zero steps returns its initial state."""
    serve = server_mod
    q0 = np.array([[0.0, 0.0], [0.5, 0.0], [0.9, 0.0]])
    v0 = np.array([[0.0, 0.0], [0.0, np.sqrt(3.0)], [0.0, 1.1]])
    d = dict(rid=0, kind="kepler", params=[1.0], dim=2, q0=q0, v0=v0, h=2 * np.pi / 200, nsteps=300)
    z = dict(rid=1, kind="kepler", params=[1.0], dim=2, q0=q0[1:], v0=v0[1:], h=0.01, nsteps=0)
    served = serve.make_requests([copy.deepcopy(d), copy.deepcopy(z)])
    serve.Server(target_tick_s=0.0002).run(served)
    plain = serve.make_requests([copy.deepcopy(d), copy.deepcopy(z)])
    serve.run_plain(plain)
    assert served[0].status[0] == 2 and (served[0].status[1:] == 0).all()
    assert same(served[0], plain[0])
    assert np.array_equal(served[1].q, q0[1:]) and np.array_equal(served[1].v, v0[1:])
    assert (served[1].iters == 0).all() and (served[1].status == 0).all()


def test_sjf_policy_same_results_and_order(server_mod):
    """Shortest-job-first admission changes only the timing: every request's
    result is the bits of the first-in-first-out run; with one slot the
    cheapest waiting request is admitted first."""
    serve = server_mod
    descs = small_requests(16)
    a = serve.make_requests(copy.deepcopy(descs))
    serve.Server(target_tick_s=0.001).run(a)
    b = serve.make_requests(copy.deepcopy(descs))
    serve.Server(target_tick_s=0.001, policy="sjf", max_active=1).run(b)
    for x, y in zip(a, b):
        assert same(x, y)
    # admission order under one slot: after the first, each admitted request
    # was the cheapest among those that had arrived (and routed to any pool)
    admitted = sorted(b, key=lambda r: r.t_admit)
    for k in range(1, len(admitted)):
        waiting_then = [r for r in admitted[k:] if r.arrival <= admitted[k].t_admit
                        and serve.pool_key(r) == serve.pool_key(admitted[k])]
        assert serve.estimated_flops(admitted[k]) <= min(serve.estimated_flops(r) for r in waiting_then)


def test_server_reuse(server_mod):
    """A server serves a second set of requests with the pools of the first
    (no state leaks between runs: the results equal a fresh server's)."""
    serve = server_mod
    descs = small_requests(10)
    srv = serve.Server(target_tick_s=0.001)
    srv.run(serve.make_requests(copy.deepcopy(descs)))
    pools = dict(srv.pools)
    again = serve.make_requests(copy.deepcopy(descs))
    srv.run(again)
    assert all(srv.pools[k] is p for k, p in pools.items())
    fresh = serve.make_requests(copy.deepcopy(descs))
    serve.Server(target_tick_s=0.001).run(fresh)
    for a, b in zip(again, fresh):
        assert same(a, b)
    srv.close()


def test_requests_at_the_top_of_the_config5_ranges(server_mod):
    """An FPUT chain of 1,500 particles (D = 3,000, the wide kernel's
    longest-chain shape), a 64-body system (d = 192) and a Kepler batch,
    served together: each equals the plain per-request form bit for bit and
    the chain agrees with the oracle."""
    serve = server_mod
    c = workloads.fput_chain(1500)
    q = np.repeat(c["q"][None, :], 3, axis=0) * (1.0 + 1e-8 * np.arange(3)[:, None])
    nb = workloads.nbody_ensemble(copies=2, nbodies=64, steps=40, seed_id=77)
    kq, kv = workloads.kepler_ic(np.array([0.1, 0.5, 0.8]))
    descs = [dict(rid=0, kind="fput", params=c["params"], dim=1500, q0=q, v0=np.zeros_like(q), h=0.25,
                  nsteps=60),
             dict(rid=1, kind="nbody", params=nb["params"], dim=192, q0=nb["q0"], v0=nb["v0"],
                  h=float(nb["h"][0]), nsteps=40),
             dict(rid=2, kind="kepler", params=[1.0], dim=2, q0=kq, v0=kv, h=2 * np.pi / 250, nsteps=500)]
    served = serve.make_requests(copy.deepcopy(descs))
    st = serve.Server(target_tick_s=0.002).run(served)
    assert st.pools == 3
    plain = serve.make_requests(copy.deepcopy(descs))
    serve.run_plain(plain)
    for a, b in zip(served, plain):
        assert (a.status == 0).all()
        assert same(a, b), a.kind
    o = cbind.run(cbind.FPUT, c["params"], q, np.zeros_like(q), 0.25, 60, nthreads=8)
    g = np.concatenate([served[0].q, served[0].v], axis=1)
    e = np.concatenate([o["q"], o["v"]], axis=1)
    assert (np.abs(g - e).max(axis=1) / np.abs(e).max(axis=1)).max() <= 1e-12
