"""GPU parity for the first-order form (irkgl_integrate1 / irkgl_advance1,
Eq. Yi2 with Eqs. IRK_init / IRK_FP) against the FP64 oracle, on the
Schwarzschild black-hole system (Eq. Ham_SBH) and the first-order harmonic
oscillator.

Tolerances as for the second-order form: relative state difference
<= 1e-13 over steps 1..10 and <= 1e-9 at the end of a non-chaotic run
(this r0 in [9.5, 16) family: the oracle's own response to a 1e-15 change
of the initial state stays near 1e-13 over t = 4000); sweep counts from
identical states within +-1 on at least 99.5 % of steps and within 3 on all
(the roundoff-floor stops explained in the test).  The GPU forms the
right-hand side with fused multiply-adds, reciprocals and CUDA's sincos,
so it is not bitwise equal to the oracle; two GPU paths that run the same
kernel are.
"""
import numpy as np
import pytest

from oracle import cbind
from paper_2511_03655_gb300 import workloads
from tests import sweep_contract

pytestmark = pytest.mark.gpu
PAR = list(workloads.SBH_PARAMS)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    return torch


def rel(g, o):
    return np.abs(g - o).max(axis=-1) / np.abs(o).max(axis=-1)


def integ(kind=None, lpt=0, h=4.0, params=None):
    from paper_2511_03655_gb300 import irkgl
    kind = irkgl.RHS_SCHWARZSCHILD if kind is None else kind
    D = 4 if kind == irkgl.RHS_SCHWARZSCHILD else 2
    return irkgl.Integrator(kind, params or PAR, D, h, lanes_per_traj=lpt)


class Dev:
    def __init__(self, torch, y0):
        self.torch = torch
        B, D = y0.shape
        self.y = torch.tensor(np.ascontiguousarray(y0), device="cuda")
        self.ylo = torch.zeros_like(self.y)
        self.lp = torch.zeros((B, 8, D), dtype=torch.float64, device="cuda")
        self.H0 = torch.zeros(B, dtype=torch.float64, device="cuda")
        self.dH = torch.zeros(B, dtype=torch.float64, device="cuda")
        self.it = torch.zeros(B, dtype=torch.int64, device="cuda")
        self.st = torch.zeros(B, dtype=torch.int32, device="cuda")
        self.started = False

    def advance(self, ig, n):
        torch = self.torch
        ns = torch.full((self.y.shape[0],), n, dtype=torch.int64, device="cuda")
        ig.advance1(self.y, self.ylo, self.lp, ns, H0=self.H0, h0_init=not self.started, dH_max=self.dH,
                    iters=self.it, status=self.st)
        self.started = True
        torch.cuda.synchronize()


@pytest.mark.parametrize("lpt", [1, 2, 4])
def test_steps_1_to_10_and_sweeps(torch_cuda, lpt):
    torch = torch_cuda
    y0 = workloads.schwarzschild_ensemble(256)
    ig = integ(lpt=lpt)
    s = Dev(torch, y0)
    o = {"y": y0, "y_lo": None, "l_prev": None}
    for step in range(10):
        s.advance(ig, 1)
        o = cbind.run1(cbind.SCHWARZSCHILD, PAR, o["y"], 4.0, 1, y_lo=o["y_lo"], l_prev=o["l_prev"])
        assert (s.st.cpu().numpy() == 0).all() and (o["status"] == 0).all()
        assert rel(s.y.cpu().numpy(), o["y"]).max() <= 1e-13, step
    # sweep counts from identical states (the GPU state handed to the oracle)
    diffs = []
    for _ in range(100):
        before = s.it.clone()
        r = cbind.run1(cbind.SCHWARZSCHILD, PAR, s.y.cpu().numpy(), 4.0, 1, y_lo=s.ylo.cpu().numpy(),
                       l_prev=s.lp.cpu().numpy(), iters_len=1)
        s.advance(ig, 1)
        diffs.append((s.it - before).cpu().numpy() - r["iters"][:, 0])
    # At h = 4 the extrapolated guess is already accurate to roundoff: a step
    # stops at k = 2 when the second sweep changes nothing (Delta = 0), or,
    # when one side's last bit still moves, by the min rule of Eq. stopping
    # at k = 4 or 5; the contract bounds how often that differs
    sweep_contract.check_steps(np.array(diffs), "schwarzschild")
    ig.close()


def test_long_run_matches_oracle_and_conserves_energy(torch_cuda):
    torch = torch_cuda
    y0 = workloads.schwarzschild_ensemble(512, seed_id=9)
    ig = integ()
    out = ig.integrate1(torch.tensor(y0, device="cuda"), nsteps_all=1000)
    torch.cuda.synchronize()
    o = cbind.run1(cbind.SCHWARZSCHILD, PAR, y0, 4.0, 1000)
    assert (out.status.cpu().numpy() == 0).all() and (out.steps.cpu().numpy() == 1000).all()
    assert rel(out.y.cpu().numpy(), o["y"]).max() <= 1e-9
    dH = out.dH_max.cpu().numpy()
    assert dH.max() <= 4 * max(o["dH_max"].max(), 1e-15)
    tot = o["iters_total"].astype(np.float64)
    assert (np.abs(out.iters.cpu().numpy() - tot) <= sweep_contract.total_bound("schwarzschild", 1000)).all()
    ig.close()


def test_harmonic1_matches_oracle(torch_cuda):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    y0 = np.stack([np.linspace(-1, 1, 64), np.linspace(0.5, -0.3, 64)], axis=1)
    for lpt in (1, 2):
        ig = integ(irkgl.RHS_HARMONIC1, lpt=lpt, h=0.4, params=[1.3])
        out = ig.integrate1(torch.tensor(y0, device="cuda"), nsteps_all=500)
        torch.cuda.synchronize()
        o = cbind.run1(cbind.HARMONIC1, [1.3], y0, 0.4, 500)
        assert rel(out.y.cpu().numpy(), o["y"]).max() <= 1e-11
        ig.close()


def test_chunks_bitwise_equal_one_call(torch_cuda):
    torch = torch_cuda
    y0 = workloads.schwarzschild_ensemble(200, seed_id=10)
    ig = integ()
    one = ig.integrate1(torch.tensor(y0, device="cuda"), nsteps_all=120)
    s = Dev(torch, y0)
    for n in (1, 33, 50, 36):
        s.advance(ig, n)
    torch.cuda.synchronize()
    assert torch.equal(one.y, s.y) and torch.equal(one.y_lo, s.ylo) and torch.equal(one.l_prev, s.lp)
    assert torch.equal(one.iters, s.it) and torch.equal(one.dH_max, s.dH)
    ig.close()


def test_wrong_form_calls_are_rejected(torch_cuda):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    ig = integ()
    q = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(irkgl.IrkglError):
        ig.integrate(q, q, nsteps_all=1)
    ig.close()
    kep = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01)
    with pytest.raises(irkgl.IrkglError):
        kep.integrate1(torch.zeros((4, 2), dtype=torch.float64, device="cuda"), nsteps_all=1)
    kep.close()


def test_advance1_nan_h0_joins_like_a_fresh_run(torch_cuda):
    """irkgl_advance1 with h0_init = 0 and H0 entries holding NaN computes
    H0 at each trajectory's first step: two chunks give the bits of one
    fresh integrate1 (state, sweeps, dH_max)."""
    torch = torch_cuda
    y0 = workloads.schwarzschild_ensemble(96, seed_id=41)
    ig = integ()
    one = ig.integrate1(torch.tensor(y0, device="cuda"), nsteps_all=90)
    f = dict(dtype=torch.float64, device="cuda")
    y = torch.tensor(y0, **f)
    ylo = torch.zeros_like(y)
    lp = torch.zeros((96, 8, 4), **f)
    H0 = torch.full((96,), float("nan"), **f)
    dH = torch.zeros(96, **f)
    it = torch.zeros(96, dtype=torch.int64, device="cuda")
    for k in (40, 50):
        ns = torch.full((96,), k, dtype=torch.int64, device="cuda")
        ig.advance1(y, ylo, lp, ns, H0=H0, h0_init=False, dH_max=dH, iters=it)
    torch.cuda.synchronize()
    assert torch.equal(one.y, y) and torch.equal(one.iters, it) and torch.equal(one.dH_max, dH)
    assert torch.isfinite(H0).all()
    ig.close()
