"""GPU parity for a right-hand side that depends on t (the non-autonomous
Henon-Heiles system of Sec. 3, lambda + xi sin t), through the C-ABI calls
irkgl_advance_t and irkgl_integrate, against the FP64 oracle.

Tolerances as in test_gpu_parity: relative state difference <= 1e-13 over
steps 1..10; sweep counts within the Henon-Heiles sweep contract; at the end of a
400-step run <= 1e-9 (xi = 0.1 at H = 1/12, where the oracle's own
sensitivity to a 1e-15 change of the initial state stays below 2e-13).
The GPU evaluates sin with CUDA's sin and forms lambda + xi sin with one
fused multiply-add, so it is not bitwise equal to the oracle; where two GPU
paths run the same kernel the results must be bitwise equal.
"""
import numpy as np
import pytest

from oracle import cbind
from paper_2511_03655_gb300 import workloads
from tests import sweep_contract

pytestmark = pytest.mark.gpu

LAM, XI = 1.0, 0.1


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    return torch


def rel(qg, vg, qo, vo):
    g = np.concatenate([qg, vg], axis=-1)
    o = np.concatenate([qo, vo], axis=-1)
    return np.abs(g - o).max(axis=-1) / np.abs(o).max(axis=-1)


class DevState:
    def __init__(self, torch, q0, v0, t0):
        d = lambda a: torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")  # noqa: E731
        B = q0.shape[0]
        self.q, self.v, self.t = d(q0), d(v0), d(t0)
        self.ql, self.vl = torch.zeros_like(self.q), torch.zeros_like(self.v)
        self.tl = torch.zeros_like(self.t)
        self.rp = torch.zeros((B, 8, 2), dtype=torch.float64, device="cuda")
        self.it = torch.zeros(B, dtype=torch.int64, device="cuda")
        self.st = torch.zeros(B, dtype=torch.int32, device="cuda")

    def advance(self, integ, torch, n):
        ns = torch.full((self.q.shape[0],), n, dtype=torch.int64, device="cuda")
        integ.advance_t(self.q, self.v, self.ql, self.vl, self.rp, self.t, ns, t_lo=self.tl,
                        iters=self.it, status=self.st)
        torch.cuda.synchronize()

    def np(self):
        return {k: getattr(self, k).cpu().numpy() for k in ("q", "v", "ql", "vl", "rp", "t", "tl", "it", "st")}


def integrator(lpt=0, xi=XI, h=0.25):
    from paper_2511_03655_gb300 import irkgl
    return irkgl.Integrator(irkgl.RHS_HENON_HEILES_FORCED, [LAM, xi], 2, h, lanes_per_traj=lpt)


@pytest.mark.parametrize("lpt", [1, 2])
def test_steps_1_to_10_and_sweeps(torch_cuda, lpt):
    torch = torch_cuda
    q0, v0, t0 = workloads.henon_heiles_ensemble(256)
    integ = integrator(lpt)
    s = DevState(torch, q0, v0, t0)
    o = {"q": q0, "v": v0, "q_lo": None, "v_lo": None, "r_prev": None, "t": t0, "t_lo": None}
    sweep_diff = []
    for step in range(10):
        before = s.it.clone()
        s.advance(integ, torch, 1)
        g = s.np()
        o = cbind.run(cbind.HH_FORCED, [LAM, XI], o["q"], o["v"], 0.25, 1, q_lo=o["q_lo"],
                      v_lo=o["v_lo"], r_prev=o["r_prev"], t0=o["t"], t_lo=o["t_lo"], iters_len=1)
        assert (g["st"] == 0).all() and (o["status"] == 0).all()
        assert rel(g["q"], g["v"], o["q"], o["v"]).max() <= 1e-13, step
        # the time is the same compensated sum on both sides: bitwise
        assert np.array_equal(g["t"], o["t"]) and np.array_equal(g["tl"], o["t_lo"])
        sweep_diff.append((s.it - before).cpu().numpy() - o["iters"][:, 0])
    # the forced system is the Henon-Heiles right-hand side with a(t) in
    # place of lambda: its contract (here at h = 0.25, far from the floor)
    sweep_contract.check_steps(np.array(sweep_diff), "henon_heiles")
    integ.close()


def test_long_run_matches_oracle(torch_cuda):
    torch = torch_cuda
    q0, v0, t0 = workloads.henon_heiles_ensemble(256)
    integ = integrator()
    s = DevState(torch, q0, v0, t0)
    s.advance(integ, torch, 400)
    g = s.np()
    o = cbind.run(cbind.HH_FORCED, [LAM, XI], q0, v0, 0.25, 400, t0=t0)
    assert (g["st"] == 0).all()
    assert rel(g["q"], g["v"], o["q"], o["v"]).max() <= 1e-9
    assert np.array_equal(g["t"], o["t"]) and np.array_equal(g["tl"], o["t_lo"])
    tot = o["iters_total"].astype(np.float64)
    assert (np.abs(g["it"] - tot) <= sweep_contract.total_bound("henon_heiles", 400)).all()
    integ.close()


def test_chunks_bitwise_equal_one_call(torch_cuda):
    torch = torch_cuda
    q0, v0, t0 = workloads.henon_heiles_ensemble(200, seed_id=11)
    integ = integrator()
    a = DevState(torch, q0, v0, t0)
    a.advance(integ, torch, 90)
    b = DevState(torch, q0, v0, t0)
    for n in (1, 17, 40, 32):
        b.advance(integ, torch, n)
    ga, gb = a.np(), b.np()
    for k in ga:
        assert np.array_equal(ga[k], gb[k]), k
    integ.close()


def test_xi_zero_equals_autonomous_kernel_bitwise(torch_cuda):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    q0, v0, t0 = workloads.henon_heiles_ensemble(128, seed_id=12)
    forced = integrator(lpt=2, xi=0.0)
    s = DevState(torch, q0, v0, t0)
    s.advance(forced, torch, 60)
    auto = irkgl.Integrator(irkgl.RHS_HENON_HEILES, [LAM], 2, 0.25, lanes_per_traj=2)
    out = auto.integrate(torch.tensor(q0, device="cuda"), torch.tensor(v0, device="cuda"), nsteps_all=60)
    torch.cuda.synchronize()
    assert torch.equal(out.q, s.q) and torch.equal(out.v, s.v)
    assert torch.equal(out.q_lo, s.ql) and torch.equal(out.r_prev, s.rp)
    forced.close()
    auto.close()


def test_integrate_starts_at_t0_zero_and_no_monitor(torch_cuda):
    torch = torch_cuda
    q0, v0, _ = workloads.henon_heiles_ensemble(64, seed_id=13)
    integ = integrator()
    out = integ.integrate(torch.tensor(q0, device="cuda"), torch.tensor(v0, device="cuda"), nsteps_all=50)
    s = DevState(torch, q0, v0, np.zeros(64))
    s.advance(integ, torch, 50)
    assert torch.equal(out.q, s.q) and torch.equal(out.v, s.v)
    assert (out.dH_max.cpu().numpy() == 0).all() and (out.status.cpu().numpy() == 0).all()
    integ.close()


def test_advance_t_rejects_autonomous_context(torch_cuda):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01)
    s = DevState(torch, np.array([[1.0, 0.0]]), np.array([[0.0, 1.0]]), np.zeros(1))
    with pytest.raises(irkgl.IrkglError):
        s.advance(integ, torch, 1)
    integ.close()
