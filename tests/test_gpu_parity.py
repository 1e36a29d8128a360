"""GPU parity: libirkgl.so (through the C-ABI) against the FP64 oracle.

Tolerances:
  * relative state difference ||y_gpu - y_oracle||_inf / ||y_oracle||_inf
    <= 1e-13 per trajectory over steps 1..10, <= 1e-9 at the end of
    non-chaotic runs;
  * fixed-point sweep counts within +-1 per step but for the measured
    roundoff-floor fraction of the sweep-count contract (tests/sweep_contract.py),
    compared from the identical state before every step.
The GPU evaluates the same formulas with fused multiply-adds and its own
reciprocal square root, so bitwise equality is not expected; where two GPU
paths run the same kernel (chunked vs one launch, host vs device buffers,
permuted order) the results must be bitwise equal.
"""
import math

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
    torch.cuda.init()
    return torch


def rel_state_diff(qg, vg, qo, vo):
    g = np.concatenate([np.asarray(qg), np.asarray(vg)], axis=-1)
    o = np.concatenate([np.asarray(qo), np.asarray(vo)], axis=-1)
    return np.abs(g - o).max(axis=-1) / np.abs(o).max(axis=-1)


def dev(torch, a, dtype=None):
    t = torch.tensor(np.ascontiguousarray(a), device="cuda")
    return t if dtype is None else t.to(dtype)


KINDS = {
    "kepler": (cbind.KEPLER, 1),
    "henon_heiles": (cbind.HENON_HEILES, 4),
    "harmonic": (cbind.HARMONIC, 5),
}


def gpu_steps(torch, kind, params, q0, v0, h, nsteps, lpt=0, chunk=None):
    """Step-by-step GPU run recording every step's state and sweep count."""
    from paper_2511_03655_gb300 import irkgl
    B, d = np.asarray(q0).shape
    integ = irkgl.Integrator(kind, params, d, h, lanes_per_traj=lpt)
    q, v = dev(torch, q0), dev(torch, v0)
    qlo, vlo = torch.zeros_like(q), torch.zeros_like(v)
    rp = torch.zeros((B, 8, d), dtype=torch.float64, device="cuda")
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    qs, vs, its = [], [], []
    chunk = chunk or 1
    done = 0
    while done < nsteps:
        k = min(chunk, nsteps - done)
        it = torch.zeros((B, k), dtype=torch.int32, device="cuda")
        integ.step(q, v, qlo, vlo, rp, nsteps=k, iters=it, status=st)
        qs.append(q.cpu().numpy().copy())
        vs.append(v.cpu().numpy().copy())
        its.append(it.cpu().numpy())
        done += k
    integ.close()
    return np.stack(qs, 1), np.stack(vs, 1), np.concatenate(its, 1), st.cpu().numpy(), \
        (q, v, qlo, vlo, rp)


def oracle_steps(kind, params, q0, v0, h, nsteps):
    st = dict(q=q0, v=v0, q_lo=None, v_lo=None, r_prev=None)
    qs, vs, its = [], [], []
    for _ in range(nsteps):
        r = cbind.run(kind, params, st["q"], st["v"], h, 1, q_lo=st["q_lo"], v_lo=st["v_lo"],
                      r_prev=st["r_prev"], iters_len=1)
        st = dict(q=r["q"], v=r["v"], q_lo=r["q_lo"], v_lo=r["v_lo"], r_prev=r["r_prev"])
        qs.append(r["q"].copy())
        vs.append(r["v"].copy())
        its.append(r["iters"][:, 0].copy())
    return np.stack(qs, 1), np.stack(vs, 1), np.stack(its, 1)


@pytest.mark.parametrize("lpt", [1, 2, 4, 8])
def test_kepler_single_first_steps_and_iterations(torch_cuda, lpt):
    """Kepler e = 0.5, h = T/200: states over steps 1..10 within 1e-13 and
    sweep counts within +-1 over the first 1,000 steps, for every tile."""
    from paper_2511_03655_gb300 import irkgl
    w = workloads.kepler_single()
    h = float(w["h"][0])
    qg, vg, _, st, _ = gpu_steps(torch_cuda, irkgl.RHS_KEPLER, [1.0], w["q0"], w["v0"], h, 10,
                                 lpt=lpt, chunk=1)
    qo, vo, _ = oracle_steps(cbind.KEPLER, [1.0], w["q0"], w["v0"], w["h"], 10)
    assert (st == 0).all()
    for s in range(10):
        assert rel_state_diff(qg[:, s], vg[:, s], qo[:, s], vo[:, s]).max() <= 1e-13, s
    # sweep counts over the first 1,000 steps, from the identical state
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, h, lanes_per_traj=lpt)
    diff = sweep_contract.identical_state_diffs(torch_cuda, integ, cbind.KEPLER, [1.0], w["q0"], w["v0"],
                                                h, 1000)
    integ.close()
    sweep_contract.check_steps(diff, "kepler")
    # most steps take exactly the oracle's number of sweeps
    assert (diff == 0).mean() > 0.8, (diff == 0).mean()


@pytest.mark.parametrize("tile", ["default", "lpt2"])
def test_kepler_sweep_counts_ensemble_rate(torch_cuda, tile):
    """Sweep counts over 1,024 orbits x 1,000 steps of the Kepler ensemble
    (a slice of the full measurement behind the contract), from the
    identical state: the contract's rate beyond +-1 and largest difference,
    and most steps equal."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    B, n = 1024, 1000
    w = workloads.kepler_ensemble(batch=B, periods=1)
    kw = dict(mix=1) if tile == "default" else dict(lanes_per_traj=2, layout=1)
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, **kw)
    diff = sweep_contract.identical_state_diffs(torch, integ, cbind.KEPLER, [1.0], w["q0"], w["v0"],
                                                w["h"], n)
    integ.close()
    sweep_contract.check_steps(diff, "kepler")
    assert (diff == 0).mean() >= 0.85, (diff == 0).mean()


def test_kepler_single_full_run(torch_cuda):
    """Config-1 workload: 20,000 steps (100 periods); end state within 1e-9 of
    the oracle, |dH/H| <= 1e-13."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    w = workloads.kepler_single()
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, float(w["h"][0]))
    out = integ.integrate(dev(torch, w["q0"]), dev(torch, w["v0"]), nsteps_all=20000)
    torch.cuda.synchronize()
    r = cbind.run(cbind.KEPLER, [1.0], w["q0"], w["v0"], w["h"], 20000)
    d = rel_state_diff(out.q.cpu(), out.v.cpu(), r["q"], r["v"])
    assert d.max() <= 1e-9, d
    assert out.dH_max.item() <= 1e-13
    assert out.steps.item() == 20000 and out.status.item() == 0
    assert abs(out.iters.item() - r["iters_total"][0]) <= sweep_contract.total_bound("kepler", 20000)
    integ.close()


@pytest.mark.parametrize("mix", [0, 1, 2])
def test_kepler_single_against_the_closed_form(torch_cuda, mix):
    """Config 1 against Kepler's closed form (Kepler's equation solved in
    high precision, tests/closed_forms.py): after 100 periods the exact orbit
    is back at periapsis.  The oracle ends 1.9e-12 (q) and 4.4e-12 (v) from
    it, roundoff accumulated linearly over 20,000 steps; each stage mixing
    must end within 1e-11."""
    import math

    from paper_2511_03655_gb300 import irkgl
    from tests import closed_forms
    torch = torch_cuda
    w = workloads.kepler_single()
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, float(w["h"][0]), mix=mix)
    out = integ.integrate(dev(torch, w["q0"]), dev(torch, w["v0"]), nsteps_all=20000)
    torch.cuda.synchronize()
    qe, ve = closed_forms.kepler_state(0.5, 20000 * float(w["h"][0]))
    assert abs(20000 * float(w["h"][0]) - 100 * 2 * math.pi) < 1e-10
    assert np.abs(out.q.cpu().numpy()[0] - np.array([float(x) for x in qe])).max() <= 1e-11
    assert np.abs(out.v.cpu().numpy()[0] - np.array([float(x) for x in ve])).max() <= 1e-11
    assert out.status.item() == 0 and out.dH_max.item() <= 1e-13
    integ.close()


@pytest.mark.parametrize("lpt", [1, 2, 8])
def test_kepler_ensemble_slice(torch_cuda, lpt):
    """2,048 orbits of the ensemble (e in [0, 0.9)), two periods each, one
    persistent launch: every orbit within 1e-11 of the oracle at the end."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    w = workloads.kepler_ensemble(batch=2048, periods=2)
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, lanes_per_traj=lpt)
    out = integ.integrate(dev(torch, w["q0"]), dev(torch, w["v0"]), nsteps=dev(torch, w["nsteps"]),
                          h=dev(torch, w["h"]))
    torch.cuda.synchronize()
    r = cbind.run(cbind.KEPLER, [1.0], w["q0"], w["v0"], w["h"], w["nsteps"], nthreads=8)
    d = rel_state_diff(out.q.cpu(), out.v.cpu(), r["q"], r["v"])
    assert d.max() <= 1e-11, (d.max(), w["e"][d.argmax()])
    assert (out.steps.cpu().numpy() == w["nsteps"]).all()
    assert (out.status.cpu().numpy() == 0).all()
    # sweep totals: the contract's mean |difference| per step bounds them
    ig = out.iters.cpu().numpy()
    assert (np.abs(ig - r["iters_total"]) <= sweep_contract.total_bound("kepler", w["nsteps"])).all()
    dh_o = r["dH_max"]
    dh_g = out.dH_max.cpu().numpy()
    assert (np.abs(dh_g - dh_o) <= np.maximum(4 * dh_o, 2e-15)).all()
    integ.close()


@pytest.mark.parametrize("mix", [0, 1])
def test_kepler_ensemble_full_size_sampled(torch_cuda, mix):
    """The full 65,536-orbit, 100-period workload in the launch configuration
    the benchmark times (both stage mixings: FP64 FMA chain and fixed-point);
    48 sampled orbits (spread over e) re-run by the oracle must agree within
    1e-9 at the end; every orbit completes."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    w = workloads.kepler_ensemble()
    order = workloads.similarity_order(w["e"])
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, mix=mix)
    out = integ.integrate(dev(torch, w["q0"]), dev(torch, w["v0"]), nsteps=dev(torch, w["nsteps"]),
                          h=dev(torch, w["h"]), order=dev(torch, order))
    torch.cuda.synchronize()
    assert (out.status.cpu().numpy() == 0).all()
    assert (out.steps.cpu().numpy() == w["nsteps"]).all()
    idx = np.linspace(0, len(w["e"]) - 1, 48).astype(int)
    r = cbind.run(cbind.KEPLER, [1.0], w["q0"][idx], w["v0"][idx], w["h"][idx], w["nsteps"][idx],
                  nthreads=8)
    d = rel_state_diff(out.q.cpu().numpy()[idx], out.v.cpu().numpy()[idx], r["q"], r["v"])
    assert d.max() <= 1e-9, d.max()
    # after exactly 100 periods every orbit is back near periapsis
    q = out.q.cpu().numpy()
    assert np.abs(q[:, 0] - (1 - w["e"])).max() < 1e-6
    integ.close()


@pytest.mark.parametrize("name", ["henon_heiles", "harmonic"])
def test_other_rhs_parity(torch_cuda, name):
    from paper_2511_03655_gb300 import irkgl
    if name == "henon_heiles":
        q0, v0 = workloads.henon_heiles_ic()
        kind_o, kind_g, params, h = cbind.HENON_HEILES, irkgl.RHS_HENON_HEILES, [1.0], 0.9
    else:
        q0 = np.array([[1.0, -0.5, 0.25], [0.3, 0.2, 0.1]])
        v0 = np.array([[0.0, 0.3, -0.2], [1.0, 0.0, 0.0]])
        kind_o, kind_g, params, h = cbind.HARMONIC, irkgl.RHS_HARMONIC, [1.3], 0.4
    for lpt in (0, 8):
        qg, vg, _, st, _ = gpu_steps(torch_cuda, kind_g, params, q0, v0, h, 10, lpt=lpt, chunk=1)
        qo, vo, _ = oracle_steps(kind_o, params, q0, v0, h, 10)
        for s in range(10):
            assert rel_state_diff(qg[:, s], vg[:, s], qo[:, s], vo[:, s]).max() <= 1e-13
        # sweep counts compared from the identical state at every step: at
        # h ~ 1 (about eight sweeps per step) the last sweeps sit at the
        # roundoff floor, where the contract allows its measured fraction of
        # steps beyond +-1
        from paper_2511_03655_gb300 import irkgl as _irkgl
        integ = _irkgl.Integrator(kind_g, params, q0.shape[1], h, lanes_per_traj=lpt)
        diff = sweep_contract.identical_state_diffs(torch_cuda, integ, kind_o, params, q0, v0, h, 200)
        integ.close()
        sweep_contract.check_steps(diff, name)
        qg, vg, itg, st, _ = gpu_steps(torch_cuda, kind_g, params, q0, v0, h, 300, lpt=lpt, chunk=300)
        r = cbind.run(kind_o, params, q0, v0, h, 300, iters_len=300)
        assert rel_state_diff(qg[:, -1], vg[:, -1], r["q"], r["v"]).max() <= 1e-11


def test_chunked_equals_single_launch_bitwise(torch_cuda):
    """irkgl_step in chunks with r_prev/lo carried == irkgl_integrate."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    w = workloads.kepler_ensemble(batch=300, periods=1)
    n = 137
    h = float(w["h"][0])
    qg, vg, itg, st, (q, v, qlo, vlo, rp) = gpu_steps(torch, irkgl.RHS_KEPLER, [1.0], w["q0"], w["v0"],
                                                      h, n, chunk=40)
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, h)
    out = integ.integrate(dev(torch, w["q0"]), dev(torch, w["v0"]), nsteps_all=n)
    torch.cuda.synchronize()
    assert torch.equal(out.q, q) and torch.equal(out.v, v)
    assert torch.equal(out.q_lo, qlo) and torch.equal(out.v_lo, vlo)
    assert torch.equal(out.r_prev, rp)
    assert (out.iters.cpu().numpy() == itg.sum(1)).all()
    integ.close()


def test_host_api_and_order_bitwise(torch_cuda):
    """Host-buffer entry point and a permuted processing order give the same
    bits as the device entry point in natural order."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    w = workloads.kepler_ensemble(batch=777, periods=1)
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01)
    a = integ.integrate(dev(torch, w["q0"]), dev(torch, w["v0"]), nsteps=dev(torch, w["nsteps"]),
                        h=dev(torch, w["h"]))
    order = np.random.default_rng(1).permutation(777).astype(np.int32)
    b = integ.integrate(dev(torch, w["q0"]), dev(torch, w["v0"]), nsteps=dev(torch, w["nsteps"]),
                        h=dev(torch, w["h"]), order=dev(torch, order))
    c = integ.integrate_host(torch.tensor(w["q0"]), torch.tensor(w["v0"]),
                             nsteps=torch.tensor(w["nsteps"]), h=torch.tensor(w["h"]))
    torch.cuda.synchronize()
    for x in (b, c):
        for f in ("q", "v", "q_lo", "v_lo", "r_prev", "dH_max", "iters", "steps", "status"):
            assert torch.equal(getattr(a, f).cpu(), getattr(x, f).cpu()), f
    integ.close()


@pytest.mark.parametrize("batch", [1, 3, 31, 33, 129])
def test_ragged_batches(torch_cuda, batch):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    w = workloads.kepler_ensemble(batch=batch, periods=1)
    n = np.minimum(w["nsteps"], 50 + np.arange(batch))
    # the stage-split tiles with the FP64 mixing, and the default tile (the
    # component split with the fixed-point mixing)
    for kw in (dict(lanes_per_traj=1), dict(lanes_per_traj=2), dict(lanes_per_traj=8), dict(mix=1)):
        integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, **kw)
        out = integ.integrate(dev(torch, w["q0"]), dev(torch, w["v0"]), nsteps=dev(torch, n),
                              h=dev(torch, w["h"]))
        torch.cuda.synchronize()
        r = cbind.run(cbind.KEPLER, [1.0], w["q0"], w["v0"], w["h"], n)
        assert rel_state_diff(out.q.cpu(), out.v.cpu(), r["q"], r["v"]).max() <= 1e-12
        assert (out.steps.cpu().numpy() == n).all()
        integ.close()


@pytest.mark.parametrize("mix", [0, 1])
def test_empty_and_zero_steps(torch_cuda, mix):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, mix=mix)
    e = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    out = integ.integrate(e, e, nsteps_all=10)
    assert out.q.shape == (0, 2)
    q0 = dev(torch, [[0.5, 0.0], [0.9, 0.0]])
    v0 = dev(torch, [[0.0, math.sqrt(3.0)], [0.0, 1.1]])
    out = integ.integrate(q0, v0, nsteps=dev(torch, np.array([0, 5], dtype=np.int64)))
    torch.cuda.synchronize()
    assert torch.equal(out.q[0], q0[0]) and torch.equal(out.v[0], v0[0])
    assert out.steps.cpu().tolist() == [0, 5]
    assert out.status.cpu().tolist() == [0, 0]
    # irkgl_step with nsteps = 0 is a no-op
    q, v = q0.clone(), v0.clone()
    integ.step(q, v, nsteps=0)
    assert torch.equal(q, q0)
    integ.close()


@pytest.mark.parametrize("mix", [0, 1])
def test_status_codes(torch_cuda, mix):
    """Iteration cap and non-finite stage values stop a trajectory at the
    start of the failing step, leaving the other trajectories untouched
    (the default FP64 tile and the fixed-point component-split tile)."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    q0 = np.array([[0.5, 0.0], [0.0, 0.0], [0.5, 0.0]])
    v0 = np.array([[0.0, math.sqrt(3.0)], [0.0, 0.0], [0.0, math.sqrt(3.0)]])
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.05, mix=mix)
    out = integ.integrate(dev(torch, q0), dev(torch, v0), nsteps_all=5)
    torch.cuda.synchronize()
    assert out.status.cpu().tolist() == [0, irkgl.STATUS_NONFINITE, 0]
    assert out.steps.cpu().tolist() == [5, 0, 5]
    assert torch.equal(out.q[1].cpu(), torch.tensor([0.0, 0.0], dtype=torch.float64))
    integ.set(irkgl.OPT_KMAX, 2)  # the first step (Rprev = 0) needs more sweeps
    out = integ.integrate(dev(torch, q0[:1]), dev(torch, v0[:1]), nsteps_all=5)
    torch.cuda.synchronize()
    r = cbind.run(cbind.KEPLER, [1.0], q0[:1], v0[:1], 0.05, 5, kmax=2)
    assert out.status.item() == irkgl.STATUS_MAXITER == r["status"][0]
    assert out.steps.item() == 0 and out.iters.item() == 2
    assert torch.equal(out.q.cpu(), torch.tensor(q0[:1]))
    integ.close()


def test_energy_monitor_matches_oracle(torch_cuda):
    """dH_max (Eq. DHglobmax) on the Henon-Heiles reference run (Sec. 5.1):
    roundoff-level, within a factor of 4 of the oracle's."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    q0, v0 = workloads.henon_heiles_ic()
    n = 20000
    integ = irkgl.Integrator(irkgl.RHS_HENON_HEILES, [1.0], 2, 1.0)
    out = integ.integrate(dev(torch, q0), dev(torch, v0), nsteps_all=n)
    torch.cuda.synchronize()
    r = cbind.run(cbind.HENON_HEILES, [1.0], q0, v0, 1.0, n)
    g, o = out.dH_max.item(), r["dH_max"][0]
    assert g <= 1e-13 and o <= 1e-13
    assert g <= 4 * o + 1e-15 and o <= 4 * g + 1e-15
    integ.close()
