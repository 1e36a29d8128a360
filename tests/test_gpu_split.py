"""GPU parity for the explicit splitting baselines (irkgl_split_integrate:
Strang and Suzuki's fourth-order composition, Sec. 4) against the C oracle
(oracle/splitting.py, same drift-kick sequence, same compensated sums).
The GPU forms g with fused multiply-adds and its own reciprocal square
root, so states agree to roundoff: <= 1e-13 after 10 steps, <= 1e-10 after
a regular run; the g-evaluation counts are exact (s per step)."""
import numpy as np
import pytest

from oracle import cbind
from paper_2511_03655_gb300 import workloads

pytestmark = pytest.mark.gpu


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


def case(name):
    from paper_2511_03655_gb300 import irkgl
    if name == "henon_heiles":
        q, v, _ = workloads.henon_heiles_ensemble(256, energy=1.0 / 24)
        return irkgl.RHS_HENON_HEILES, cbind.HENON_HEILES, [1.0], q, v, 0.05, 2
    if name == "kepler":
        w = workloads.kepler_ensemble(batch=256, periods=1, emax=0.3)
        return irkgl.RHS_KEPLER, cbind.KEPLER, [1.0], w["q0"], w["v0"], 2 * np.pi / 2000, 2
    e = workloads.nbody_ensemble(copies=64, steps=10)
    return irkgl.RHS_NBODY, cbind.NBODY, e["params"], e["q0"], e["v0"], float(e["h"][0]) / 4, 18


@pytest.mark.parametrize("name", ["henon_heiles", "kepler", "nbody6"])
@pytest.mark.parametrize("scheme", ["strang", "suz90"])
def test_split_matches_oracle(torch_cuda, name, scheme):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    kg, ko, par, q0, v0, h, d = case(name)
    sid = irkgl.SPLIT_STRANG if scheme == "strang" else irkgl.SPLIT_SUZ90
    nk = 1 if scheme == "strang" else 5
    ig = irkgl.Integrator(kg, par, d, h)
    ig.set(irkgl.OPT_MONITOR_LOCAL, 1)
    q, v = torch.tensor(q0, device="cuda"), torch.tensor(v0, device="cuda")
    for n, tol in ((10, 1e-13), (1000, 1e-10)):
        out = ig.split_integrate(sid, q, v, nsteps_all=n)
        torch.cuda.synchronize()
        r = cbind.run_split(scheme, ko, par, q0, v0, h, n, local=True)
        assert (out.status.cpu().numpy() == 0).all() and (out.steps.cpu().numpy() == n).all()
        assert (out.iters.cpu().numpy() == nk * n).all()
        assert rel(out.q.cpu().numpy(), out.v.cpu().numpy(), r["q"], r["v"]).max() <= tol, (n, scheme)
        dg, do = out.dH_max.cpu().numpy(), r["dH_max"]
        assert np.all(np.abs(dg - do) <= 0.05 * do + 2e-15), (np.abs(dg - do).max(), do.max())
    ig.close()


def test_split_rejects_first_order_and_bad_scheme(torch_cuda):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    x = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    ig = irkgl.Integrator(irkgl.RHS_SCHWARZSCHILD, list(workloads.SBH_PARAMS), 4, 1.0)
    with pytest.raises(irkgl.IrkglError):
        ig.split_integrate(irkgl.SPLIT_STRANG, x, x, nsteps_all=1)
    ig.close()
    ig = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01)
    y = torch.ones((2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(irkgl.IrkglError):
        ig.split_integrate(7, y, y, nsteps_all=1)
    ig.close()
