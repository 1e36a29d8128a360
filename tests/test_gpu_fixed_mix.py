"""The fixed-point stage mixing (IRKGL_OPT_MIX = 1) against exact rational
arithmetic, and the mixed kernel against the oracle.

sum_j eta_ij R_j is formed exactly in 128-bit integers and rounded once, so
for columns whose R_j lie within a factor 2^8 of the largest the result must
equal the correctly rounded value of the exact sum bit for bit."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import cbind, coeffs
from paper_2511_03655_gb300 import workloads
from tests import sweep_contract

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    return torch, irkgl


def test_fixed_mix_is_correctly_rounded(lib):
    torch, irkgl = lib
    eta = coeffs.fp64_tables()["eta"]
    rng = np.random.default_rng(11)
    n = 400
    scale = 10.0 ** rng.uniform(-12, 2, size=(n, 1))
    sign = np.where(rng.uniform(size=(n, 8)) < 0.5, -1.0, 1.0)
    # magnitudes within a factor 2^8 of each other (the exact regime)
    R = sign * scale * (1.0 + rng.uniform(size=(n, 8))) * 2.0 ** rng.integers(0, 7, size=(n, 8))
    R[0] = 0.0                       # all zero
    R[1, :4] = 0.0                   # some zero
    R[2] = -R[3]                     # signs flipped
    out = irkgl.irkgl_diag_fixed_mix(torch.tensor(R, device="cuda")).cpu().numpy()
    for x in range(n):
        for i in range(8):
            exact = sum(Fraction(eta[i][j]) * Fraction(float(R[x, j])) for j in range(8))
            assert out[x, i, 0] == float(exact), (x, i)


def test_fixed_mix_nonfinite_propagates(lib):
    torch, irkgl = lib
    R = np.ones((2, 8))
    R[0, 3] = np.inf
    R[1, 5] = np.nan
    out = irkgl.irkgl_diag_fixed_mix(torch.tensor(R, device="cuda")).cpu().numpy()
    assert np.isnan(out).all()


@pytest.mark.parametrize("block,layout,tile", [(128, 0, 2), (128, 1, 1), (64, 0, 1)])
def test_mixed_kernel_kepler_parity(lib, block, layout, tile):
    """Both tiles of the fixed-point mixing: the component split (the default
    at 128 threads) and the one-lane stage split."""
    torch, irkgl = lib
    w = workloads.kepler_single()
    h = float(w["h"][0])
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, h, mix=1, block_threads=block, layout=layout)
    assert integ.tile == tile
    q, v = torch.tensor(w["q0"], device="cuda"), torch.tensor(w["v0"], device="cuda")
    ql, vl = torch.zeros_like(q), torch.zeros_like(v)
    rp = torch.zeros((1, 8, 2), dtype=torch.float64, device="cuda")
    st = dict(q=w["q0"], v=w["v0"], q_lo=None, v_lo=None, r_prev=None)
    for s in range(10):
        integ.step(q, v, ql, vl, rp, nsteps=1)
        r = cbind.run(cbind.KEPLER, [1.0], st["q"], st["v"], h, 1, q_lo=st["q_lo"],
                      v_lo=st["v_lo"], r_prev=st["r_prev"])
        st = dict(q=r["q"], v=r["v"], q_lo=r["q_lo"], v_lo=r["v_lo"], r_prev=r["r_prev"])
        g = np.concatenate([q.cpu().numpy(), v.cpu().numpy()], axis=1)
        e = np.concatenate([r["q"], r["v"]], axis=1)
        assert (np.abs(g - e).max() / np.abs(e).max()) <= 1e-13, s
    # sweep counts over 1,000 steps from the identical state: the contract;
    # the exact sums round differently from the oracle's separately rounded
    # ones, so fewer steps match exactly than with the FMA chain
    diff = sweep_contract.identical_state_diffs(torch, integ, cbind.KEPLER, [1.0], w["q0"], w["v0"], h, 1000)
    sweep_contract.check_steps(diff, "kepler")
    assert (diff == 0).mean() > 0.7
    out = integ.integrate(torch.tensor(w["q0"], device="cuda"), torch.tensor(w["v0"], device="cuda"),
                          nsteps_all=20000)
    torch.cuda.synchronize()
    r = cbind.run(cbind.KEPLER, [1.0], w["q0"], w["v0"], w["h"], 20000)
    g = np.concatenate([out.q.cpu().numpy(), out.v.cpu().numpy()], axis=1)
    e = np.concatenate([r["q"], r["v"]], axis=1)
    assert np.abs(g - e).max() / np.abs(e).max() <= 1e-9
    assert out.dH_max.item() <= 1e-13
    integ.close()


def test_mixed_kernel_ensemble(lib):
    torch, irkgl = lib
    w = workloads.kepler_ensemble(batch=2048, periods=2)
    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, mix=1)
    out = integ.integrate(torch.tensor(w["q0"], device="cuda"), torch.tensor(w["v0"], device="cuda"),
                          nsteps=torch.tensor(w["nsteps"], device="cuda"),
                          h=torch.tensor(w["h"], device="cuda"))
    torch.cuda.synchronize()
    r = cbind.run(cbind.KEPLER, [1.0], w["q0"], w["v0"], w["h"], w["nsteps"], nthreads=8)
    g = np.concatenate([out.q.cpu().numpy(), out.v.cpu().numpy()], axis=1)
    e = np.concatenate([r["q"], r["v"]], axis=1)
    assert (np.abs(g - e).max(axis=1) / np.abs(e).max(axis=1)).max() <= 1e-11
    assert (out.status.cpu().numpy() == 0).all()
    ig = out.iters.cpu().numpy()
    assert (np.abs(ig - r["iters_total"]) <= sweep_contract.total_bound("kepler", w["nsteps"])).all()
    integ.close()


def test_fixed_mix_rows_form_bitwise(lib):
    """The runtime-row form (one accumulator, signs on the operands, row
    constants) gives the bits of the two-accumulator form for every column,
    inside the exact regime and outside it (spreads beyond 2^8, where both
    truncate the small R_j the same way), for zeros and non-finite values."""
    torch, irkgl = lib
    rng = np.random.default_rng(12)
    n = 4096
    scale = 10.0 ** rng.uniform(-30, 30, size=(n, 1))
    sign = np.where(rng.uniform(size=(n, 8)) < 0.5, -1.0, 1.0)
    R = sign * scale * (1.0 + rng.uniform(size=(n, 8))) * 2.0 ** rng.integers(-40, 40, size=(n, 8))
    R[0] = 0.0
    R[1, :5] = 0.0
    R[2, 3] = np.inf
    R[3, 6] = np.nan
    R[4] = 5e-324 * np.arange(1, 9)          # subnormals
    R[5] = np.array([1.0, -1.0] * 4) * 2.0 ** 60
    Rt = torch.tensor(R, device="cuda")
    a = irkgl.irkgl_diag_fixed_mix(Rt).cpu().numpy()
    b = irkgl.irkgl_diag_fixed_mix_rows(Rt).cpu().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    assert np.array_equal(a.view(np.int64)[~np.isnan(a)], b.view(np.int64)[~np.isnan(b)])


@pytest.mark.parametrize("lanes", [2, 8])
def test_rows_spread_over_lanes_one_step_bitwise(lib, lanes):
    """With the stage rows spread over 2 or 8 lanes, the group agrees on each
    component's exponent, converts its own stages and gathers the rest: the
    sweeps then form the same Q and R as the one-lane tile, so after one step
    R (kept as R_prev) and the sweep counts are bit-identical; q and v differ
    only by the order of the update's stage sums."""
    torch, irkgl = lib
    w = workloads.kepler_ensemble(batch=1024, periods=1)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")  # noqa: E731
    res = {}
    for lpt in (1, lanes):
        integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, 0.01, mix=1, layout=1, lanes_per_traj=lpt)
        assert integ.tile == lpt
        q, v = d(w["q0"]), d(w["v0"])
        ql, vl = torch.zeros_like(q), torch.zeros_like(v)
        rp = torch.zeros((q.shape[0], 8, 2), dtype=torch.float64, device="cuda")
        it = torch.zeros((q.shape[0], 1), dtype=torch.int32, device="cuda")
        integ.step(q, v, ql, vl, rp, h=d(w["h"]), nsteps=1, iters=it)
        torch.cuda.synchronize()
        res[lpt] = (q.cpu().numpy(), v.cpu().numpy(), rp.cpu().numpy(), it.cpu().numpy())
        integ.close()
    a, b = res[1], res[lanes]
    assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])
    for x, y in ((a[0], b[0]), (a[1], b[1])):
        assert (np.abs(x - y).max(axis=1) / np.abs(x).max(axis=1)).max() <= 4e-16
