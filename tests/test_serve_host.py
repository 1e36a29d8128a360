"""Host logic of the serving loop (no GPU): the range allocator behind the
pools' shared state arrays, request routing to pools, and the union of
launch intervals used for the GPU-busy fraction."""
import random

import numpy as np

from paper_2511_03655_gb300 import ragged, serve, workloads


def test_ranges_first_fit_and_coalescing():
    r = serve._Ranges(100)
    a = r.alloc(30)
    b = r.alloc(30)
    c = r.alloc(30)
    assert (a, b, c) == (0, 30, 60)
    assert r.alloc(11) is None          # only 10 left
    r.release(b)
    assert r.alloc(31) is None          # the hole is 30
    assert r.alloc(20) == 30            # first fit in the hole
    r.release(a)
    r.release(c)
    r.release(30)
    assert r.free == [(0, 100)] and r.used == {} and r.high_water() == 0


def test_ranges_random_against_a_bitmap():
    """Random alloc/release sequences: allocated ranges never overlap, stay in
    bounds, and the free list always covers exactly the unallocated cells."""
    rnd = random.Random(5)
    cap = 500
    r = serve._Ranges(cap)
    owner = np.zeros(cap, dtype=bool)
    held = []
    for _ in range(4000):
        if held and rnd.random() < 0.45:
            s, n = held.pop(rnd.randrange(len(held)))
            assert owner[s:s + n].all()
            owner[s:s + n] = False
            r.release(s)
        else:
            n = rnd.randint(1, 60)
            s = r.alloc(n)
            if s is None:
                # no free run of n cells exists
                runs = np.diff(np.flatnonzero(np.diff(np.concatenate([[1], owner.astype(int), [1]]))))[::2]
                assert (runs < n).all() if len(runs) else True
                continue
            assert 0 <= s and s + n <= cap and not owner[s:s + n].any()
            owner[s:s + n] = True
            held.append((s, n))
        free_cells = np.zeros(cap, dtype=bool)
        for s, n in r.free:
            free_cells[s:s + n] = True
        assert np.array_equal(free_cells, ~owner)
        # coalesced: no two free ranges touch
        for (s0, n0), (s1, _) in zip(r.free, r.free[1:]):
            assert s0 + n0 < s1
        assert r.high_water() == (max(s + n for s, n in held) if held else 0)


def test_union_length():
    assert serve._union_length([]) == 0.0
    assert serve._union_length([(0, 1), (0.5, 2), (3, 4)]) == 3.0
    assert serve._union_length([(2, 3), (0, 1), (0.2, 0.4)]) == 2.0


def test_serving_requests_cover_the_stated_ranges():
    """The config-5 generator draws batch from logU[1, 4096], horizon from
    logU[1e2, 1e5], N-body N in {3..64} and FPUT n up to 1536 (D = 2d up to
    3072), from the four families."""
    descs = workloads.serving_requests(n=400, rate=2000.0)
    B = np.array([d["q0"].shape[0] for d in descs])
    T = np.array([d["nsteps"] for d in descs])
    D = np.array([2 * d["dim"] for d in descs])
    assert B.min() >= 1 and B.max() <= 4096 and B.max() > 1000
    assert T.min() >= 100 and T.max() <= 100000 and T.max() > 30000
    assert D.min() >= 4 and D.max() <= 3072 and D.max() > 2000
    nb = [d["dim"] // 3 for d in descs if d["kind"] == "nbody" and d["dim"] != 18]
    assert min(nb) >= 3 and max(nb) <= 64
    for d in descs:
        ragged.bucket_label(serve.KIND_IDS[d["kind"]], d["dim"])  # every request has a pool


def test_config4_requests_are_the_ragged_batch():
    """The config-4 serving load: one batch-1 request per instance of the
    ragged batch, with that instance's kind, size, parameters, state, step
    and horizon; Poisson arrivals increasing; the same bits on every call."""
    w = workloads.uneven_batch(ninst=12, steps=50)
    reqs = workloads.config4_requests(ninst=12, steps=50)
    again = workloads.config4_requests(ninst=12, steps=50)
    arr = np.array([r["arrival"] for r in reqs])
    assert (np.diff(arr) > 0).all() and arr[0] > 0
    for k, r in enumerate(reqs):
        o, d = int(w["offset"][k]), int(w["dim"][k])
        po, pn = int(w["param_offset"][k]), int(w["nparams"][k])
        assert r["kind"] == {2: "nbody", 3: "fput"}[int(w["kind"][k])] and r["dim"] == d
        assert np.array_equal(r["q0"], w["q0"][o:o + d][None, :]) and r["q0"].shape == (1, d)
        assert np.array_equal(r["v0"], w["v0"][o:o + d][None, :])
        assert r["params"] == list(w["params"][po:po + pn])
        assert r["h"] == w["h"][k] and r["nsteps"] == 50 and r["rid"] == k
        assert r["arrival"] == again[k]["arrival"] and np.array_equal(r["q0"], again[k]["q0"])
