"""Host logic of the bucketed ragged launches (no GPU): the plan is a
permutation, buckets are contiguous and homogeneous, costliest first inside
a bucket, teams come from the tile table, and the flop model matches the
per-unit counts used for the roofline."""
import numpy as np

from paper_2511_03655_gb300 import irkgl, ragged, workloads


def test_plan_is_a_bucketed_permutation():
    w = workloads.uneven_batch(ninst=96, steps=10, nmax_body=64, nmax_chain=512)
    tiles = {"nbody:33-64": {"team": 256}, "fput:129-256": {"team": 64}}
    plan = ragged.RaggedPlan(w, tiles=tiles)
    n = len(w["kind"])
    assert sorted(plan.perm.tolist()) == list(range(n))
    seen = 0
    for b in plan.buckets:
        idx = plan.perm[b.start:b.start + b.count]
        labels = {ragged.bucket_label(int(w["kind"][k]), int(w["dim"][k])) for k in idx}
        assert labels == {b.label}
        assert b.dmax == int(w["dim"][idx].max())
        cost = [ragged.flops_per_sweep(int(w["kind"][k]), int(w["dim"][k])) for k in idx]
        assert cost == sorted(cost, reverse=True)
        assert b.team == tiles.get(b.label, {"team": 0})["team"]
        seen += b.count
    assert seen == n
    starts = sorted((b.start, b.count) for b in plan.buckets)
    assert all(s0 + c0 == s1 for (s0, c0), (s1, _) in zip(starts, starts[1:]))
    a = np.arange(n) * 3.0
    assert np.array_equal(plan.unpermute(a[plan.perm]), a)


def test_flop_model_matches_nbody6_counts():
    # the 6-body counts used by the register-kernel bench line: per step
    # 3882, per sweep 6456 (d = 18, 15 pairs)
    assert ragged.flops_per_step(irkgl.RHS_NBODY, 18) == 3882
    assert ragged.flops_per_sweep(irkgl.RHS_NBODY, 18) == 6456
