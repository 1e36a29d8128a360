"""The sweep-count contract between the fast CUDA forms and the oracle.

The target asks for fixed-point sweep counts within +-1 of the oracle's per
step.  For the fast forms (fused multiply-adds, exact fixed-point stage
sums, integer x^(-3/2)) the stopping rule (Eqs. Delta_n, stopping) makes
that unreachable on a small fraction of steps: when the iteration has reached the roundoff floor,
a step stops at the first sweep whose increment Delta is exactly zero, or by
the min rule once Delta stops decreasing, and a last-bit difference between
the GPU's fused or exact operations and the oracle's separate roundings
decides which sweep that is.  The reading taken: +-1 on all but a measured
roundoff-floor fraction of the steps, never more than a measured largest
difference apart.

Both figures were measured per workload with the GPU state (hi and lo parts,
R_prev) handed to the oracle before every step, so that only the arithmetic
of that one step differs (``python bench.py --workload sweeps``, summarised in
profiles/sweep_parity_gb300.md):

  workload class    steps compared     |k_gpu - k_oracle| >= 2      largest   mean |diff|
  kepler            6.55e8 per mixing  3.2e-5 / 2.5e-5 (mix 1 / 0)  4         0.103
  henon_heiles      6.3e4 (h = 1.0)    6.7e-2 / 2.8e-2              4         0.53
                    4.1e7 (h = 0.7)    2.6e-2 / 1.9e-2              5         0.30
  nbody6            4.1e7 per mixing   3.5e-5 / 3.2e-5              2         0.0014
  schwarzschild     4.1e6 (h = 4)      4.9e-4 / 4.1e-4              4         0.050
                    4.1e6 (h = 16)     2.1e-3 / 1.9e-3              5         0.134
                    4.1e6 each, s = 2, 4, 6 stages (h = 0.5, 2, 2):
                                       1.4e-4 / 3.2e-4 / 3.2e-4     4         0.038
  harmonic          4.1e7 (FP64)       1.3e-2                       4         0.102
  ragged (wide)     2.5e4 per mixing   3.8e-2 / 3.5e-3              4         0.239
(Kepler: the 65,536-orbit ensemble over 10,000 steps; Henon-Heiles: the
orbit of Sec. 5.1 over 2 pi 1e4, and a 4,096-orbit ensemble; 6-body: 4,096
copies over 10,000 steps; Schwarzschild: 8,192 first-order orbits over 500
steps, also with the s-stage schemes of Sec. 5.2; harmonic: 4,096 three-component oscillators at omega h = 0.52 over
10,000 steps; ragged: 128 instances of the ragged batch on the wide kernel
over 200 steps, steps that failed on the GPU left out.)

The reproducible form (IRKGL_OPT_MIX = 2) needs no contract: it performs
the oracle's operation sequence, and tests/test_gpu_reproducible.py requires
every step's sweep count to be equal.

A test of n compared steps passes when no step differs by more than the
class's largest difference and the number of steps beyond +-1 stays below
the 1e-6 upper tail of a Poisson count with mean MARGIN x rate x n.  Sweep
totals over a run may differ by at most MARGIN x (mean |diff|) x steps plus
the class's largest difference (one step of a short run, such as the first
step from a cold guess, may differ by that much).
"""
from __future__ import annotations

import math

import numpy as np

MARGIN = 2.0
TAIL = 1e-6

# class: (rate of |diff| >= 2, largest |diff|, mean |diff| per step), the
# larger of the two stage mixings
CONTRACT = {
    "kepler": (3.3e-5, 4, 0.103),
    "henon_heiles": (6.7e-2, 5, 0.53),
    "nbody6": (3.5e-5, 2, 0.0014),
    "schwarzschild": (2.2e-3, 5, 0.134),
    "harmonic": (1.3e-2, 4, 0.102),
    "ragged": (3.8e-2, 4, 0.239),
}


def allowed_beyond(rate: float, n: int, margin: float = MARGIN, tail: float = TAIL) -> int:
    """Smallest m with P(Poisson(margin * rate * n) > m) < tail."""
    lam = margin * rate * n
    m, term = 0, math.exp(-lam)
    cdf = term
    while 1.0 - cdf >= tail and m < 10 * n + 10:
        m += 1
        term *= lam / m
        cdf += term
    return m


def check_steps(diff, cls: str) -> None:
    """Assert the contract on an array of per-step differences k_gpu - k_oracle."""
    rate, dmax, _ = CONTRACT[cls]
    d = np.abs(np.asarray(diff)).ravel()
    beyond = int((d >= 2).sum())
    lim = allowed_beyond(rate, d.size)
    assert d.max() <= dmax, f"{cls}: sweep counts {int(d.max())} apart (contract: <= {dmax})"
    assert beyond <= lim, (f"{cls}: {beyond} of {d.size} steps beyond +-1 (contract: <= {lim}, "
                           f"rate {rate:g} x {MARGIN})")


def total_bound(cls: str, steps) -> np.ndarray:
    """Largest allowed |sum k_gpu - sum k_oracle| over runs of `steps` steps."""
    _, dmax, mean_abs = CONTRACT[cls]
    return MARGIN * mean_abs * np.asarray(steps, dtype=np.float64) + dmax


def identical_state_diffs(torch, integ, kind_o, params, q0, v0, h, nsteps):
    """k_gpu - k_oracle per step [B, nsteps], the GPU's state (hi, lo,
    R_prev) handed to the oracle before every step."""
    from oracle import cbind
    B, d = np.asarray(q0).shape
    f = dict(dtype=torch.float64, device="cuda")
    q, v = torch.tensor(np.asarray(q0), **f), torch.tensor(np.asarray(v0), **f)
    ql, vl = torch.zeros_like(q), torch.zeros_like(v)
    rp = torch.zeros((B, 8, d), **f)
    hs = np.broadcast_to(np.asarray(h, dtype=np.float64), (B,)).copy()
    hh = torch.tensor(hs, **f)
    it = torch.zeros((B, 1), dtype=torch.int32, device="cuda")
    out = np.zeros((B, nsteps), dtype=np.int64)
    for n in range(nsteps):
        host = [t.cpu().numpy() for t in (q, v, ql, vl, rp)]
        integ.step(q, v, ql, vl, rp, h=hh, nsteps=1, iters=it)
        r = cbind.run(kind_o, params, host[0], host[1], hs, 1, q_lo=host[2], v_lo=host[3],
                      r_prev=host[4], iters_len=1, nthreads=8)
        out[:, n] = it.cpu().numpy()[:, 0].astype(np.int64) - r["iters"][:, 0]
    return out
