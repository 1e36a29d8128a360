"""The first-order component-split tile (irkgl1_cs.cuh): with FP64 mixing it
agrees with the stage-split first-order kernel to roundoff (the stage sums
are associated differently); with fixed-point mixing (mu exact on the
2^-62 grid, the correctly rounded sum) against the oracle; chunked runs
bitwise equal to one run.  Tolerances as in test_gpu_first_order."""
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


def integ(mix, layout, kind=None, params=None, h=4.0):
    from paper_2511_03655_gb300 import irkgl
    kind = irkgl.RHS_SCHWARZSCHILD if kind is None else kind
    D = 4 if kind == irkgl.RHS_SCHWARZSCHILD else 2
    return irkgl.Integrator(kind, params or PAR, D, h, mix=mix, layout=layout)


@pytest.mark.parametrize("mix", [0, 1])
def test_schwarzschild_cs_against_oracle(torch_cuda, mix):
    torch = torch_cuda
    y0 = workloads.schwarzschild_ensemble(256, seed_id=50)
    ig = integ(mix, 2)
    assert ig.layout == "component split" and ig.tile == 4
    d = torch.tensor(y0, device="cuda")
    for n, tol in ((10, 1e-13), (1000, 1e-9)):
        out = ig.integrate1(d, nsteps_all=n)
        torch.cuda.synchronize()
        r = cbind.run1(cbind.SCHWARZSCHILD, PAR, y0, 4.0, n)
        assert (out.status.cpu().numpy() == 0).all()
        assert rel(out.y.cpu().numpy(), r["y"]).max() <= tol, (n, mix)
        tot = r["iters_total"].astype(np.float64)
        assert (np.abs(out.iters.cpu().numpy() - tot) <= sweep_contract.total_bound("schwarzschild", n)).all()
        dg, do = out.dH_max.cpu().numpy(), r["dH_max"]
        assert np.all(dg <= 2 * do + 2e-15)
    ig.close()


def test_schwarzschild_cs_matches_stage_split(torch_cuda):
    torch = torch_cuda
    y0 = workloads.schwarzschild_ensemble(512, seed_id=51)
    d = torch.tensor(y0, device="cuda")
    a = integ(0, 2).integrate1(d, nsteps_all=300)
    b = integ(0, 1).integrate1(d, nsteps_all=300)
    torch.cuda.synchronize()
    assert rel(a.y.cpu().numpy(), b.y.cpu().numpy()).max() <= 1e-11
    # two GPU tiles: each within the contract of the oracle, so of each other twice over
    assert (np.abs(a.iters.cpu().numpy() - b.iters.cpu().numpy())
            <= 2 * sweep_contract.total_bound("schwarzschild", 300)).all()


def test_default_layout_with_fixed_point_and_chunks(torch_cuda):
    torch = torch_cuda
    y0 = workloads.schwarzschild_ensemble(200, seed_id=52)
    ig = integ(1, 0)
    assert ig.layout == "component split"
    d = torch.tensor(y0, device="cuda")
    one = ig.integrate1(d, nsteps_all=150)
    y = d.clone()
    ylo = torch.zeros_like(y)
    lp = torch.zeros((200, 8, 4), dtype=torch.float64, device="cuda")
    it = torch.zeros(200, dtype=torch.int64, device="cuda")
    H0 = torch.zeros(200, dtype=torch.float64, device="cuda")
    dH = torch.zeros_like(H0)
    first = True
    for n in (1, 49, 50, 50):
        ig.advance1(y, ylo, lp, torch.full((200,), n, dtype=torch.int64, device="cuda"), H0=H0,
                    h0_init=first, dH_max=dH, iters=it)
        first = False
    torch.cuda.synchronize()
    assert torch.equal(one.y, y) and torch.equal(one.y_lo, ylo) and torch.equal(one.l_prev, lp)
    assert torch.equal(one.iters, it) and torch.equal(one.dH_max, dH)
    ig.close()


@pytest.mark.parametrize("mix", [0, 1])
def test_harmonic1_cs(torch_cuda, mix):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    y0 = np.stack([np.linspace(-1, 1, 64), np.linspace(0.5, -0.3, 64)], axis=1)
    ig = integ(mix, 2, kind=irkgl.RHS_HARMONIC1, params=[1.3], h=0.4)
    out = ig.integrate1(torch.tensor(y0, device="cuda"), nsteps_all=500)
    torch.cuda.synchronize()
    r = cbind.run1(cbind.HARMONIC1, [1.3], y0, 0.4, 500)
    assert rel(out.y.cpu().numpy(), r["y"]).max() <= 1e-11
    ig.close()


@pytest.mark.parametrize("batch", [1, 3, 33])
def test_default_tile_ragged_empty_and_status(torch_cuda, batch):
    """The default first-order tile (component split, fixed-point mixing) on
    batch sizes that leave partly filled warps, per-orbit step counts
    (including zero), an empty batch, and an orbit on the polar axis
    (sin theta = 0: the 1/sin^2 terms are infinite, so that orbit stops with
    the non-finite status and leaves the others untouched)."""
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    y0 = workloads.schwarzschild_ensemble(batch, seed_id=53)
    n = (20 + 7 * np.arange(batch)).astype(np.int64)
    n[0] = 0
    ig = integ(1, 0)
    out = ig.integrate1(torch.tensor(y0, device="cuda"), nsteps=torch.tensor(n, device="cuda"))
    torch.cuda.synchronize()
    r = cbind.run1(cbind.SCHWARZSCHILD, PAR, y0, 4.0, n)
    assert (out.steps.cpu().numpy() == n).all() and (out.status.cpu().numpy() == 0).all()
    assert np.array_equal(out.y.cpu().numpy()[0], y0[0])
    if batch > 1:
        assert rel(out.y.cpu().numpy()[1:], r["y"][1:]).max() <= 1e-12
    e = torch.zeros((0, 4), dtype=torch.float64, device="cuda")
    assert ig.integrate1(e, nsteps_all=10).y.shape == (0, 4)
    bad = y0.copy()
    bad[0, 1] = 0.0  # theta = 0
    out = ig.integrate1(torch.tensor(bad, device="cuda"), nsteps_all=5)
    torch.cuda.synchronize()
    st = out.status.cpu().numpy()
    assert st[0] == irkgl.STATUS_NONFINITE and (st[1:] == 0).all()
    assert out.steps.cpu().numpy()[0] == 0
    ig.close()
