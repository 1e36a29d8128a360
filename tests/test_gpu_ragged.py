"""GPU parity for ragged batches (irkgl_integrate_ragged, the wide kernel):
N-body systems and FPUT chains of different sizes in one launch, each
instance checked against the oracle run on its own; team shapes agree
bit for bit; bad descriptors are reported, not faulted on."""
import numpy as np
import pytest

from oracle import cbind
from paper_2511_03655_gb300 import workloads
from tests import sweep_contract

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    return torch


def small_batch(ninst=24, steps=200, nmax_body=20, nmax_chain=200):
    return workloads.uneven_batch(ninst=ninst, steps=steps, nmax_body=nmax_body, nmax_chain=nmax_chain)


def run_gpu(torch, w, team=0, order=None, mix=0):
    from paper_2511_03655_gb300 import irkgl
    n = len(w["kind"])
    integ = irkgl.Integrator(irkgl.RHS_HARMONIC, [1.0], 1, 0.1, mix=mix)  # context for tables/options
    integ.set(irkgl.OPT_WIDE_TEAM, team)
    inst = irkgl.instances_tensor(w, "cuda")
    out = irkgl.RaggedOutputs.allocate(len(w["q0"]), n)
    irkgl.irkgl_integrate_ragged(integ.ctx, inst, n, int(w["dim"].max()),
                                 torch.tensor(w["params"], device="cuda"),
                                 torch.tensor(w["q0"], device="cuda"),
                                 torch.tensor(w["v0"], device="cuda"), out,
                                 order=None if order is None else torch.tensor(order, device="cuda"))
    torch.cuda.synchronize()
    integ.close()
    return out


def oracle_instance(w, k):
    o, d = int(w["offset"][k]), int(w["dim"][k])
    po, pn = int(w["param_offset"][k]), int(w["nparams"][k])
    kind = {2: cbind.NBODY, 3: cbind.FPUT, 5: cbind.HARMONIC}[int(w["kind"][k])]
    return cbind.run(kind, w["params"][po:po + pn], w["q0"][o:o + d], w["v0"][o:o + d],
                     w["h"][k], int(w["nsteps"][k]))


def test_ragged_matches_oracle_per_instance(torch_cuda):
    w = small_batch()
    out = run_gpu(torch_cuda, w)
    q, v = out.q.cpu().numpy(), out.v.cpu().numpy()
    st, steps, it = out.status.cpu().numpy(), out.steps.cpu().numpy(), out.iters.cpu().numpy()
    dH = out.dH_max.cpu().numpy()
    for k in range(len(w["kind"])):
        r = oracle_instance(w, k)
        o, d = int(w["offset"][k]), int(w["dim"][k])
        assert st[k] == r["status"][0] == 0, k
        assert steps[k] == w["nsteps"][k]
        g = np.concatenate([q[o:o + d], v[o:o + d]])
        e = np.concatenate([r["q"][0], r["v"][0]])
        assert np.abs(g - e).max() / np.abs(e).max() <= 1e-11, (k, int(w["kind"][k]), d)
        assert abs(it[k] - r["iters_total"][0]) <= sweep_contract.total_bound("ragged", int(w["nsteps"][k])), k
        assert dH[k] <= max(4 * r["dH_max"][0], 4e-15), (k, dH[k], r["dH_max"][0])


def test_team_shapes_agree_bitwise(torch_cuda):
    w = small_batch(ninst=12, steps=120, nmax_body=20, nmax_chain=60)
    ref = run_gpu(torch_cuda, w, team=32)
    for team in (64, 128, 256):
        out = run_gpu(torch_cuda, w, team=team)
        for f in ("q", "v", "q_lo", "v_lo", "r_prev", "iters", "steps", "status"):
            assert torch_cuda.equal(getattr(ref, f), getattr(out, f)), (team, f)


def test_order_permutation_bitwise(torch_cuda):
    w = small_batch(ninst=16, steps=80)
    a = run_gpu(torch_cuda, w)
    order = np.argsort(-w["dim"].astype(np.int64) ** 2, kind="stable").astype(np.int32)
    b = run_gpu(torch_cuda, w, order=order)
    for f in ("q", "v", "iters", "status"):
        assert torch_cuda.equal(getattr(a, f), getattr(b, f)), f


def test_wide_and_register_kernels_agree(torch_cuda):
    """The same 6-body system through the ragged (wide) and batched (register)
    kernels: different pair summation orders, same result to roundoff."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    e = workloads.nbody_ensemble(copies=3, steps=300)
    d = e["dim"]
    w = {"kind": np.full(3, 2, np.int32), "dim": np.full(3, d, np.int32),
         "offset": np.arange(3, dtype=np.int64) * d, "param_offset": np.zeros(3, np.int32),
         "nparams": np.full(3, len(e["params"]), np.int32), "h": e["h"][:3],
         "nsteps": np.full(3, 300, np.int64), "params": np.array(e["params"]),
         "q0": e["q0"].reshape(-1), "v0": e["v0"].reshape(-1)}
    rg = run_gpu(torch, w)
    integ = irkgl.Integrator(irkgl.RHS_NBODY, e["params"], d, float(e["h"][0]))
    rr = integ.integrate(torch.tensor(e["q0"], device="cuda"), torch.tensor(e["v0"], device="cuda"),
                         nsteps_all=300)
    torch.cuda.synchronize()
    a = np.concatenate([rg.q.cpu().numpy(), rg.v.cpu().numpy()])
    b = np.concatenate([rr.q.cpu().numpy().reshape(-1), rr.v.cpu().numpy().reshape(-1)])
    assert np.abs(a - b).max() / np.abs(b).max() <= 1e-12
    integ.close()


def test_bad_descriptor_reported(torch_cuda):
    """A descriptor whose dimension exceeds dmax is reported through status,
    the other instances are integrated normally."""
    w = small_batch(ninst=6, steps=20, nmax_body=10, nmax_chain=30)
    w["dim"] = w["dim"].copy()
    true_dmax = int(w["dim"].max())
    w["dim"][3] = true_dmax + 100  # lie about one instance's size
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    n = len(w["kind"])
    integ = irkgl.Integrator(irkgl.RHS_HARMONIC, [1.0], 1, 0.1)
    inst = irkgl.instances_tensor(w, "cuda")
    out = irkgl.RaggedOutputs.allocate(len(w["q0"]) + 200, n)
    irkgl.irkgl_integrate_ragged(integ.ctx, inst, n, true_dmax, torch.tensor(w["params"], device="cuda"),
                                 torch.tensor(np.concatenate([w["q0"], np.zeros(200)]), device="cuda"),
                                 torch.tensor(np.concatenate([w["v0"], np.zeros(200)]), device="cuda"), out)
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()
    assert st[3] != 0 and (np.delete(st, 3) == 0).all()
    integ.close()


def test_bucketed_launches_equal_single_launch_bitwise(torch_cuda):
    """ragged.RaggedRunner: one launch per size bucket (own team, own stream)
    gives the state bits, sweep counts and statuses of one launch of the
    whole batch, and of the unbucketed call in the caller's instance order."""
    from paper_2511_03655_gb300 import irkgl, ragged
    torch = torch_cuda
    w = small_batch(ninst=40, steps=60, nmax_body=40, nmax_chain=300)
    tiles = {"nbody:3-8": {"team": 64}, "fput:1-64": {"team": 32}, "fput:257-512": {"team": 256}}
    plan = ragged.RaggedPlan(w, tiles=tiles)
    assert len(plan.buckets) >= 3
    runner = ragged.RaggedRunner(plan, torch.tensor(w["params"], device="cuda"),
                                 torch.tensor(w["q0"], device="cuda"), torch.tensor(w["v0"], device="cuda"))
    a = irkgl.RaggedOutputs.allocate(len(w["q0"]), len(w["kind"]))
    b = irkgl.RaggedOutputs.allocate(len(w["q0"]), len(w["kind"]))
    runner.run(a)
    runner.single(b)
    torch.cuda.synchronize()
    for f in ("q", "v", "q_lo", "v_lo", "r_prev", "iters", "steps", "status"):
        assert torch.equal(getattr(a, f), getattr(b, f)), f
    # the energy monitor sums H over the team (per-warp partials), so its
    # rounding depends on the team size: dH_max agrees to roundoff only
    da, db = a.dH_max.cpu().numpy(), b.dH_max.cpu().numpy()
    assert np.all(np.abs(da - db) <= 1e-15 + 1e-3 * np.abs(db))
    ref = run_gpu(torch, w)
    assert torch.equal(a.q, ref.q) and torch.equal(a.v, ref.v)
    for f in ("iters", "status"):
        assert np.array_equal(plan.unpermute(getattr(a, f).cpu().numpy()), getattr(ref, f).cpu().numpy()), f
    runner.close()


def test_fixed_point_mixing_ragged(torch_cuda):
    """IRKGL_OPT_MIX = 1 on the wide kernel: every instance against the
    oracle (tolerances as above), and team shapes bitwise equal."""
    w = small_batch(ninst=20, steps=150)
    out = run_gpu(torch_cuda, w, mix=1)
    q, v = out.q.cpu().numpy(), out.v.cpu().numpy()
    st, it = out.status.cpu().numpy(), out.iters.cpu().numpy()
    for k in range(len(w["kind"])):
        r = oracle_instance(w, k)
        o, d = int(w["offset"][k]), int(w["dim"][k])
        assert st[k] == r["status"][0] == 0, k
        g = np.concatenate([q[o:o + d], v[o:o + d]])
        e = np.concatenate([r["q"][0], r["v"][0]])
        assert np.abs(g - e).max() / np.abs(e).max() <= 1e-11, (k, int(w["kind"][k]), d)
        assert abs(it[k] - r["iters_total"][0]) <= sweep_contract.total_bound("ragged", int(w["nsteps"][k])), k
    ref = run_gpu(torch_cuda, w, team=64, mix=1)
    for team in (128, 256):
        other = run_gpu(torch_cuda, w, team=team, mix=1)
        for f in ("q", "v", "q_lo", "v_lo", "r_prev", "iters", "steps", "status"):
            assert torch_cuda.equal(getattr(ref, f), getattr(other, f)), (team, f)


def nbody_instances(nbs, steps, frac=0.0025):
    """N-body systems of the given body counts (the ragged batch's generator)
    packed as one ragged batch, h = frac of each system's innermost period."""
    kinds, dims, params, qs, vs, hs = [], [], [], [], [], []
    for k, nb in enumerate(nbs):
        s = workloads.nbody_system(nb, seed_id=30000 + k)
        kinds.append(2)
        dims.append(3 * nb)
        params.append([1.0] + list(s["masses"]))
        qs.append(s["q"])
        vs.append(s["v"])
        hs.append(frac * s["period_inner"])
    off = np.concatenate([[0], np.cumsum(dims)[:-1]]).astype(np.int64)
    pc = np.array([len(p) for p in params])
    return {"kind": np.array(kinds, np.int32), "dim": np.array(dims, np.int32), "offset": off,
            "param_offset": np.concatenate([[0], np.cumsum(pc)[:-1]]).astype(np.int32),
            "nparams": pc.astype(np.int32), "h": np.array(hs), "nsteps": np.full(len(nbs), steps, np.int64),
            "params": np.concatenate([np.asarray(p, np.float64) for p in params]),
            "q0": np.concatenate(qs), "v0": np.concatenate(vs)}


@pytest.mark.parametrize("mix", [0, 1])
def test_large_systems_match_oracle(torch_cuda, mix):
    """Systems of 21 to 128 bodies (the wide kernel's largest, its body
    weights sized for 128): over 10 steps the states agree with the oracle
    within 1e-13."""
    nbs = [21, 24, 30, 33, 40, 47, 48, 64, 100, 128]
    w = nbody_instances(nbs, 10)
    out = run_gpu(torch_cuda, w, mix=mix)
    q, v = out.q.cpu().numpy(), out.v.cpu().numpy()
    st = out.status.cpu().numpy()
    for k, nb in enumerate(nbs):
        r = oracle_instance(w, k)
        o, d = int(w["offset"][k]), int(w["dim"][k])
        assert st[k] == r["status"][0] == 0, nb
        g = np.concatenate([q[o:o + d], v[o:o + d]])
        e = np.concatenate([r["q"][0], r["v"][0]])
        assert np.abs(g - e).max() / np.abs(e).max() <= 1e-13, nb


def test_large_systems_team_shapes_agree_bitwise(torch_cuda):
    """Each body's force is summed over the other bodies in index order
    whatever the team size, so every team shape gives the same bits, up to
    128 bodies."""
    w = nbody_instances([21, 33, 40, 64], 25)
    ref = run_gpu(torch_cuda, w, team=64)
    for team in (128, 256):
        out = run_gpu(torch_cuda, w, team=team)
        for f in ("q", "v", "q_lo", "v_lo", "r_prev", "iters", "steps", "status"):
            assert torch_cuda.equal(getattr(ref, f), getattr(out, f)), (team, f)
    w = nbody_instances([21], 25)  # d = 63 also fits the one-warp team
    a = run_gpu(torch_cuda, w, team=32)
    b = run_gpu(torch_cuda, w, team=256)
    for f in ("q", "v", "iters"):
        assert torch_cuda.equal(getattr(a, f), getattr(b, f)), f
    w = nbody_instances([100, 128], 10)
    a = run_gpu(torch_cuda, w, team=128)
    b = run_gpu(torch_cuda, w, team=256)
    for f in ("q", "v", "iters"):
        assert torch_cuda.equal(getattr(a, f), getattr(b, f)), f


def test_bucketed_run_captured_in_a_cuda_graph(torch_cuda):
    """The bucketed launches (one per size bucket, each on its own stream)
    recorded as one CUDA graph: a replay gives the bits of the direct run,
    and replays repeat them."""
    from paper_2511_03655_gb300 import irkgl, ragged
    torch = torch_cuda
    w = small_batch(ninst=40, steps=60, nmax_body=40, nmax_chain=300)
    plan = ragged.RaggedPlan(w)
    dev = torch.device("cuda")
    runner = ragged.RaggedRunner(plan, torch.tensor(w["params"], device=dev),
                                 torch.tensor(w["q0"], device=dev), torch.tensor(w["v0"], device=dev),
                                 device=dev, mix=1)
    direct = irkgl.RaggedOutputs.allocate(len(w["q0"]), len(w["kind"]), device=dev)
    runner.run(direct)
    torch.cuda.synchronize()
    out = irkgl.RaggedOutputs.allocate(len(w["q0"]), len(w["kind"]), device=dev)
    g = runner.capture(out)
    for _ in range(2):
        for f in ("q", "v"):
            getattr(out, f).zero_()
        g.replay()
        torch.cuda.synchronize()
        for f in ("q", "v", "q_lo", "v_lo", "r_prev", "iters", "steps", "status", "dH_max"):
            assert torch.equal(getattr(direct, f), getattr(out, f)), f
    assert len(plan.buckets) > 1
    runner.close()
