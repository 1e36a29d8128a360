"""The continuous-batching server: every request's result is the same alone and
in the mix (bitwise: a chunked run continues exactly), admission respects the
memory budget, and results agree with the oracle."""
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


def small_requests(n=14):
    return workloads.serving_requests(n=n, rate=4000.0, batch_max=64, horizon_max=400, nb_max=12,
                                      n_max=96)


def test_result_same_alone_and_in_mix(server_mod):
    serve = server_mod
    descs = small_requests()
    mix = serve.make_requests(copy.deepcopy(descs))
    st = serve.Server(nstreams=8, chunk_traj_steps=2e3).run(mix)
    assert st.summary()["requests"] == len(descs)
    assert st.max_concurrent > 1  # requests really overlapped
    for d, r in zip(descs, mix):
        alone = serve.make_requests([copy.deepcopy(d)])
        serve.Server(nstreams=1, chunk_traj_steps=7e2).run(alone)  # different chunking too
        a = alone[0]
        assert (r.status == 0).all() and (a.status == 0).all()
        assert np.array_equal(r.q, a.q) and np.array_equal(r.v, a.v), d["kind"]
        assert np.array_equal(r.iters, a.iters) and np.array_equal(r.dH_max, a.dH_max)


@pytest.mark.parametrize("stage_mix", [0, 1])
def test_mix_matches_single_launch(server_mod, stage_mix):
    """Served in chunks among other requests, every request gets the bits of
    one uninterrupted launch, with either stage mixing."""
    serve = server_mod
    descs = small_requests(8)
    mix = serve.make_requests(copy.deepcopy(descs))
    serve.Server(nstreams=4, chunk_traj_steps=1e3, mix=stage_mix).run(mix)
    plain = serve.make_requests(copy.deepcopy(descs))
    serve.run_plain(plain, mix=stage_mix)
    for r, p in zip(mix, plain):
        assert np.array_equal(r.q, p.q) and np.array_equal(r.v, p.v), r.kind
        assert np.array_equal(r.iters, p.iters)


def test_admission_by_memory_budget(server_mod):
    """Admitted requests never hold more device memory than the budget (a
    request larger than the whole budget runs alone), every request
    completes, and a larger budget admits more at once."""
    serve = server_mod
    descs = small_requests(10)
    reqs = serve.make_requests(copy.deepcopy(descs))
    sizes = sorted(r.device_bytes() for r in reqs)
    budget = sizes[0] + sizes[1]
    st = serve.Server(mem_budget_bytes=budget, nstreams=4).run(reqs)
    assert st.summary()["requests"] == 10 and all(r.q is not None for r in reqs)
    assert st.peak_bytes <= max(budget, sizes[-1])
    wide_open = serve.make_requests(copy.deepcopy(descs))
    st2 = serve.Server(mem_budget_bytes=1 << 34, nstreams=4).run(wide_open)
    assert st2.max_concurrent >= st.max_concurrent
    for a, b in zip(reqs, wide_open):
        assert np.array_equal(a.q, b.q)


@pytest.mark.parametrize("stage_mix", [0, 1])
def test_served_results_match_oracle(server_mod, stage_mix):
    serve = server_mod
    descs = [d for d in small_requests(20) if d["kind"] in ("kepler", "fput")][:4]
    reqs = serve.make_requests(copy.deepcopy(descs))
    serve.Server(nstreams=4, chunk_traj_steps=1e3, mix=stage_mix).run(reqs)
    for r in reqs:
        kind = cbind.KEPLER if r.kind == "kepler" else cbind.FPUT
        o = cbind.run(kind, r.params, r.q0, r.v0, r.h, r.nsteps, nthreads=8)
        g = np.concatenate([r.q, r.v], axis=1)
        e = np.concatenate([o["q"], o["v"]], axis=1)
        assert (np.abs(g - e).max(axis=1) / np.abs(e).max(axis=1)).max() <= 1e-11, r.kind


def test_context_pool_reuse(server_mod):
    """Contexts return to the pool when a request finishes and are reused:
    the pool never holds more contexts than requests ran at once, and a
    second run on the same server creates none."""
    serve = server_mod
    descs = small_requests(20)
    srv = serve.Server(nstreams=4, chunk_traj_steps=1e3)
    st = srv.run(serve.make_requests(copy.deepcopy(descs)))
    pooled = sum(len(v) for v in srv._pool.values())
    assert 1 <= pooled <= st.max_concurrent
    before = {k: list(v) for k, v in srv._pool.items()}
    again = serve.make_requests(copy.deepcopy(descs))
    srv2_stats = srv.run(again)
    after = {k: list(v) for k, v in srv._pool.items()}
    assert sum(len(v) for v in after.values()) <= max(pooled, srv2_stats.max_concurrent)
    assert all(set(before[k]) <= set(after.get(k, [])) for k in before)  # the same contexts came back
    first = serve.make_requests(copy.deepcopy(descs))
    serve.Server(nstreams=4, chunk_traj_steps=1e3).run(first)
    for a, b in zip(first, again):
        assert np.array_equal(a.q, b.q) and np.array_equal(a.iters, b.iters)
    srv.close()


def test_sjf_policy_same_results_and_order(server_mod):
    """Shortest-job-first admission changes only the timing: every request's
    result is the bits of the first-in-first-out run; with one slot the
    cheapest waiting request is admitted first."""
    serve = server_mod
    descs = small_requests(16)
    a = serve.make_requests(copy.deepcopy(descs))
    serve.Server(nstreams=4, chunk_traj_steps=1e3).run(a)
    b = serve.make_requests(copy.deepcopy(descs))
    serve.Server(nstreams=4, chunk_traj_steps=1e3, policy="sjf", max_active=1).run(b)
    for x, y in zip(a, b):
        assert np.array_equal(x.q, y.q) and np.array_equal(x.iters, y.iters)
    # admission order under one slot: after the first, each admitted request
    # was the cheapest among those that had arrived
    admitted = sorted(b, key=lambda r: r.t_admit)
    for k in range(1, len(admitted)):
        waiting_then = [r for r in admitted[k:] if r.arrival <= admitted[k].t_admit]
        assert serve.estimated_flops(admitted[k]) <= min(serve.estimated_flops(r) for r in waiting_then)
