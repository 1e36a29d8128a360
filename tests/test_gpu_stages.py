"""GPU parity for the s-stage IRKGL schemes, s = 2, 4, 6 (the first-order
kernel instantiated with s stages, IRKGL_OPT_STAGES), against the C oracle
run with the same s, on the Schwarzschild black-hole system (Eq. Ham_SBH):
the scheme family of the paper's Sec. 5.2 comparison.  Tolerances as in
test_gpu_first_order; the local energy-error monitor (Eq. DHlocmax) against
the oracle's per-step energies."""
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


@pytest.mark.parametrize("s", [2, 4, 6])
@pytest.mark.parametrize("lpt", [1, 2])
def test_s_stage_parity(torch_cuda, s, lpt):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    h = 0.5 if s == 2 else 2.0
    y0 = workloads.schwarzschild_ensemble(128, seed_id=20 + s)
    ig = irkgl.Integrator(irkgl.RHS_SCHWARZSCHILD, PAR, 4, h, lanes_per_traj=lpt, stages=s)
    assert ig.tile == lpt
    y = torch.tensor(y0, device="cuda")
    ylo = torch.zeros_like(y)
    lp = torch.zeros((128, s, 4), dtype=torch.float64, device="cuda")
    it = torch.zeros(128, dtype=torch.int64, device="cuda")
    st = torch.zeros(128, dtype=torch.int32, device="cuda")
    ones = torch.ones(128, dtype=torch.int64, device="cuda")
    o = {"y": y0, "y_lo": None, "l_prev": None}
    for step in range(10):
        ig.advance1(y, ylo, lp, ones, iters=it, status=st)
        torch.cuda.synchronize()
        o = cbind.run1(cbind.SCHWARZSCHILD, PAR, o["y"], h, 1, y_lo=o["y_lo"], l_prev=o["l_prev"], stages=s)
        assert (st.cpu().numpy() == 0).all()
        assert rel(y.cpu().numpy(), o["y"]).max() <= 1e-13, (s, step)
    out = ig.integrate1(torch.tensor(y0, device="cuda"), nsteps_all=400)
    torch.cuda.synchronize()
    r = cbind.run1(cbind.SCHWARZSCHILD, PAR, y0, h, 400, stages=s)
    assert (out.status.cpu().numpy() == 0).all()
    assert rel(out.y.cpu().numpy(), r["y"]).max() <= 1e-9
    # the Schwarzschild class of the sweep-count contract covers s = 2, 4, 6
    # (measured tighter than for s = 8)
    tot = r["iters_total"].astype(np.float64)
    assert (np.abs(out.iters.cpu().numpy() - tot) <= sweep_contract.total_bound("schwarzschild", 400)).all()
    # dH_max of the global monitor: same size as the oracle's (s = 2 is
    # truncation-dominated, the others roundoff-dominated)
    dg, do = out.dH_max.cpu().numpy(), r["dH_max"]
    assert np.all(dg <= 2 * do + 2e-15) and np.all(do <= 2 * dg + 2e-15)
    ig.close()


def test_local_energy_monitor(torch_cuda):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    s, h, n = 2, 2.0, 200
    y0 = workloads.schwarzschild_ensemble(32, seed_id=30)
    ig = irkgl.Integrator(irkgl.RHS_SCHWARZSCHILD, PAR, 4, h, stages=s)
    ig.set(irkgl.OPT_MONITOR_LOCAL, 1)
    out = ig.integrate1(torch.tensor(y0, device="cuda"), nsteps_all=n)
    torch.cuda.synchronize()
    # the oracle's local error from its per-step states
    o = {"y": y0, "y_lo": None, "l_prev": None}
    Hprev = np.array([cbind.hamiltonian1(cbind.SCHWARZSCHILD, PAR, y) for y in y0])
    loc = np.zeros(32)
    for _ in range(n):
        o = cbind.run1(cbind.SCHWARZSCHILD, PAR, o["y"], h, 1, y_lo=o["y_lo"], l_prev=o["l_prev"], stages=s)
        Hn = np.array([cbind.hamiltonian1(cbind.SCHWARZSCHILD, PAR, y) for y in o["y"]])
        loc = np.maximum(loc, np.abs((Hn - Hprev) / Hprev))
        Hprev = Hn
    g = out.dH_max.cpu().numpy()
    assert np.all(np.abs(g - loc) <= 0.05 * loc + 1e-15), (g[:4], loc[:4])
    ig.close()


def test_second_order_rejects_stage_variants(torch_cuda):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    ig = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, stages=4)
    q = torch.tensor([[1.0, 0.0]], dtype=torch.float64, device="cuda")
    v = torch.tensor([[0.0, 1.0]], dtype=torch.float64, device="cuda")
    with pytest.raises(irkgl.IrkglError):
        ig.integrate(q, v, nsteps_all=1)
    ig.close()
