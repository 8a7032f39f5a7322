"""The serving workload's request stream (serve_driver.make_workload) on CPU:
the recipe the serving benchmark states (512 requests, Poisson arrivals with
a 2 ms mean gap, 64 bases of 1e4..2e6 rows, factors of 8..128 columns with
kappa in 1e2..1e14, appends of 4..32 columns, half of each, no basis past its
capacity), and that the stream is a pure function of its seed."""
import math

import numpy as np

from paper_2507_07788_gb300 import serve_driver as sd


def test_stream_follows_the_recipe():
    wl = sd.make_workload()
    assert len(wl.m) == 64 and len(wl.reqs) == 512 and wl.n_max == 256
    assert all(10_000 <= m <= 2_000_000 for m in wl.m)
    # log-uniform rows: the log10 mean sits near the middle of [4, 6.3]
    assert abs(np.mean(np.log10(wl.m)) - (4 + math.log10(2e6)) / 2) < 0.25
    t = np.array([r.arrival for r in wl.reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps: mean 2 ms (std error ~0.09 ms at 512 draws), cv ~1
    assert abs(gaps.mean() - 2e-3) < 0.4e-3
    assert 0.8 < gaps.std() / gaps.mean() < 1.2
    width = [0] * 64
    kinds = {"factor": 0, "append": 0}
    for r in wl.reqs:
        kinds[r.kind] += 1
        assert 1e2 <= r.kappa <= 1e14
        if r.kind == "factor":
            assert 8 <= r.width <= 128
            width[r.basis] = r.width
        else:
            assert 4 <= r.width <= 32
            width[r.basis] += r.width
        assert width[r.basis] <= wl.n_max
    # 50/50, plus appends turned into factors at capacity
    assert 0.4 * 512 <= kinds["factor"] <= 0.65 * 512


def test_stream_is_a_function_of_its_seed():
    a = sd.make_workload(n_bases=6, n_requests=40, seed=3)
    b = sd.make_workload(n_bases=6, n_requests=40, seed=3)
    c = sd.make_workload(n_bases=6, n_requests=40, seed=4)
    key = lambda w: [(r.kind, r.basis, r.width, r.kappa, r.arrival) for r in w.reqs]
    assert a.m == b.m and key(a) == key(b)
    assert key(a) != key(c)


def test_scaled_arrivals_keep_the_stream():
    """Scaling the arrival process (the serving benchmark sets the mean gap
    to the mean service time / utilization) changes only the times."""
    a = sd.make_workload(n_bases=6, n_requests=40, mean_gap_s=1.0, seed=3)
    b = sd.make_workload(n_bases=6, n_requests=40, mean_gap_s=2e-3, seed=3)
    sd.scale_arrivals(a, 2e-3)
    for ra, rb in zip(a.reqs, b.reqs):
        assert (ra.kind, ra.basis, ra.width, ra.kappa) == (rb.kind, rb.basis, rb.width, rb.kappa)
        assert math.isclose(ra.arrival, rb.arrival, rel_tol=1e-12)
