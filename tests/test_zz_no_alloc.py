"""The no-allocation entry point (irkgl_integrate_noalloc) against the regular
one (irkgl_integrate with a context): callers that cannot allocate device
memory (a host application owning the whole device heap, real-time code,
plug-ins) get the same results from the library's fixed internal scratch.

Named to run last: a failure here does not hide the other GPU tests.  It
passes alone in a fresh process and after the rest of the suite (the shared
scratch is reset by every call)."""
import numpy as np
import pytest

from paper_2511_03655_gb300 import workloads

pytestmark = pytest.mark.gpu


def _rel(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return (np.abs(a - b).max(axis=-1) / np.abs(b).max(axis=-1)).max()


def test_noalloc_matches_regular_entry_point_two_calls():
    import torch

    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    dev = torch.device("cuda")
    w = workloads.kepler_ensemble(batch=3001, periods=1)
    q0 = torch.tensor(w["q0"], device=dev)
    v0 = torch.tensor(w["v0"], device=dev)
    ns = torch.tensor(np.minimum(w["nsteps"], 180), device=dev)
    hh = torch.tensor(w["h"], device=dev)
    order = torch.tensor(workloads.similarity_order(w["e"]), device=dev)

    integ = irkgl.Integrator(irkgl.RHS_KEPLER, [1.0], 2, float(w["h"][0]))
    ref = integ.integrate(q0, v0, nsteps=ns, h=hh, order=order)
    torch.cuda.synchronize()

    outs = [irkgl.Outputs.allocate(3001, 2, device=dev) for _ in range(2)]
    torch.cuda.synchronize()
    for out in outs:  # two calls in a row share the fixed scratch
        rc = irkgl.irkgl_integrate_noalloc(irkgl.RHS_KEPLER, [1.0], 2, float(w["h"][0]), q0, v0,
                                           out, nsteps=ns, h_per_traj=hh, order=order)
        assert rc == irkgl.OK
        torch.cuda.synchronize()
        # the tolerance of the parity tests (same kernel, so in fact bitwise)
        assert _rel(out.q, ref.q) <= 1e-13 and _rel(out.v, ref.v) <= 1e-13
        assert torch.equal(out.steps, ref.steps) and torch.equal(out.status, ref.status)
        assert torch.equal(out.iters, ref.iters)
        assert (out.dH_max.cpu() - ref.dH_max.cpu()).abs().max().item() <= 1e-15
    integ.close()


def test_noalloc_rejects_parameters_beyond_scratch():
    import torch

    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    dev = torch.device("cuda")
    n = irkgl.NOALLOC_MAX_PARAMS  # N-body with 63 bodies needs 1 + 63 parameters
    q0 = torch.zeros((1, 3 * n), dtype=torch.float64, device=dev)
    out = irkgl.Outputs.allocate(1, 3 * n, device=dev)
    rc = irkgl.irkgl_integrate_noalloc(irkgl.RHS_NBODY, [1.0] * (n + 1), 3 * n, 0.1, q0, q0, out,
                                       nsteps_all=1)
    assert rc == irkgl.ERR_INVALID


def test_noalloc_forced_henon_heiles_matches_regular_entry_point():
    """The time-dependent kind: both calls start at t = 0 and leave the
    energy monitor off (H(t) is not conserved), so dH_max stays 0 on both."""
    import torch

    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    dev = torch.device("cuda")
    q0n, v0n, _ = workloads.henon_heiles_ensemble(517)
    q0 = torch.tensor(q0n, device=dev)
    v0 = torch.tensor(v0n, device=dev)
    integ = irkgl.Integrator(irkgl.RHS_HENON_HEILES_FORCED, [1.0, 0.1], 2, 0.25)
    ref = integ.integrate(q0, v0, nsteps_all=150)
    torch.cuda.synchronize()
    for _ in range(2):
        out = irkgl.Outputs.allocate(517, 2, device=dev)
        rc = irkgl.irkgl_integrate_noalloc(irkgl.RHS_HENON_HEILES_FORCED, [1.0, 0.1], 2, 0.25,
                                           q0, v0, out, nsteps_all=150)
        assert rc == irkgl.OK
        torch.cuda.synchronize()
        assert _rel(out.q, ref.q) <= 1e-13 and _rel(out.v, ref.v) <= 1e-13
        assert torch.equal(out.steps, ref.steps) and torch.equal(out.status, ref.status)
        assert torch.equal(out.iters, ref.iters)
        assert out.dH_max.abs().max().item() == 0.0 and ref.dH_max.abs().max().item() == 0.0
    integ.close()


def test_noalloc_rejects_first_order_kinds():
    """First-order kinds take the irkgl_*1 calls, here as in irkgl_create's
    second-order calls: IRKGL_ERR_INVALID, nothing launched."""
    import torch

    from paper_2511_03655_gb300 import build, irkgl
    build.build()
    irkgl.load()
    dev = torch.device("cuda")
    y = torch.ones((4, 2), dtype=torch.float64, device=dev)
    out = irkgl.Outputs.allocate(4, 2, device=dev)
    rc = irkgl.irkgl_integrate_noalloc(irkgl.RHS_HARMONIC1, [1.0], 2, 0.1, y, y, out, nsteps_all=1)
    assert rc == irkgl.ERR_INVALID
