"""The component-split tile (IRKGL_OPT_TILE_LAYOUT = 2) performs the
operation sequence of an existing tile, so its results are bit-identical:
with FP64 mixing to the stage-split tile with two lanes per trajectory,
with fixed-point mixing to the one-lane tile (whose parity with the oracle
is tested in test_gpu_parity / test_gpu_fixed_mix)."""
import numpy as np
import pytest

from oracle import cbind
from paper_2511_03655_gb300 import workloads

pytestmark = pytest.mark.gpu
FIELDS = ("q", "v", "q_lo", "v_lo", "r_prev", "dH_max", "iters", "steps", "status")


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    return torch


def run(torch, kind, params, w, **kw):
    from paper_2511_03655_gb300 import irkgl
    ig = irkgl.Integrator(kind, params, 2, 0.01, **kw)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")  # noqa: E731
    out = ig.integrate(d(w["q0"]), d(w["v0"]), nsteps=d(w["nsteps"]), h=d(w["h"]),
                       order=d(workloads.similarity_order(w["e"])))
    torch.cuda.synchronize()
    tile = ig.tile
    ig.close()
    return out, tile


@pytest.mark.parametrize("mix,ref_lanes", [(0, 2), (1, 1)])
def test_kepler_component_split_bitwise(torch_cuda, mix, ref_lanes):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    w = workloads.kepler_ensemble(batch=8192, periods=3)
    a, ta = run(torch, irkgl.RHS_KEPLER, [1.0], w, mix=mix, layout=2)
    b, tb = run(torch, irkgl.RHS_KEPLER, [1.0], w, mix=mix, lanes_per_traj=ref_lanes, layout=1)
    assert ta == 2 and tb == ref_lanes
    for f in FIELDS:
        assert torch.equal(getattr(a, f), getattr(b, f)), f


@pytest.mark.parametrize("mix,ref_lanes", [(0, 2), (1, 1)])
def test_henon_heiles_component_split_bitwise_and_oracle(torch_cuda, mix, ref_lanes):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    q, v, _ = workloads.henon_heiles_ensemble(2048)
    w = {"q0": q, "v0": v, "nsteps": np.full(2048, 400, np.int64), "h": np.full(2048, 0.5),
         "e": np.zeros(2048)}
    a, _ = run(torch, irkgl.RHS_HENON_HEILES, [1.0], w, mix=mix, layout=2)
    b, _ = run(torch, irkgl.RHS_HENON_HEILES, [1.0], w, mix=mix, lanes_per_traj=ref_lanes, layout=1)
    for f in FIELDS:
        assert torch.equal(getattr(a, f), getattr(b, f)), f
    r = cbind.run(cbind.HENON_HEILES, [1.0], q[:64], v[:64], 0.5, 400)
    g = np.concatenate([a.q.cpu().numpy()[:64], a.v.cpu().numpy()[:64]], 1)
    o = np.concatenate([r["q"], r["v"]], 1)
    assert (np.abs(g - o).max(1) / np.abs(o).max(1)).max() <= 1e-10


def test_component_split_continuation_bitwise(torch_cuda):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    w = workloads.kepler_ensemble(batch=1000, periods=1)
    ig = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, mix=1)
    assert ig.layout == "component split"  # the default with the fixed-point mixing
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")  # noqa: E731
    one = ig.integrate(d(w["q0"]), d(w["v0"]), nsteps=d(w["nsteps"]), h=d(w["h"]))
    q, v = d(w["q0"]), d(w["v0"])
    ql, vl = torch.zeros_like(q), torch.zeros_like(v)
    rp = torch.zeros((1000, 8, 2), dtype=torch.float64, device="cuda")
    H0 = torch.zeros(1000, dtype=torch.float64, device="cuda")
    dH = torch.zeros_like(H0)
    it = torch.zeros(1000, dtype=torch.int64, device="cuda")
    left = w["nsteps"].copy()
    first = True
    while left.max() > 0:
        k = np.minimum(left, 97)
        ig.advance(q, v, ql, vl, rp, d(k), h=d(w["h"]), H0=H0, h0_init=first, dH_max=dH, iters=it)
        first = False
        left -= k
    torch.cuda.synchronize()
    assert torch.equal(one.q, q) and torch.equal(one.v, v) and torch.equal(one.r_prev, rp)
    assert torch.equal(one.iters, it) and torch.equal(one.dH_max, dH)
    ig.close()


def test_component_split_unsupported_elsewhere(torch_cuda):
    from paper_2511_03655_gb300 import irkgl
    torch = torch_cuda
    ig = irkgl.Integrator(irkgl.RHS_HARMONIC, [1.0], 3, 0.1, layout=2)
    x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(irkgl.IrkglError):
        ig.integrate(x, x, nsteps_all=1)
    ig.close()
