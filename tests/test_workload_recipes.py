"""The synthetic workload recipes, on the host: field edges of the batched
and served workloads are log-uniform multiples of 32 within their ranges,
and the served trace has Poisson arrivals at the requested rate, an even
compress/decompress mix, about 30 % FP64 requests and the two tolerances."""
import math

import numpy as np

from paper_1903_07761_gb300 import workloads as W


def test_edges_are_log_uniform_multiples_of_32():
    rng = np.random.default_rng(0)
    for lo, hi in ((64, 384), (32, 512)):
        e = np.array([W._loguniform_edge(rng, lo, hi) for _ in range(20000)])
        assert e.min() >= lo and e.max() <= hi and np.all(e % 32 == 0)
        # log-uniform: the median sits near the geometric mean of the range
        # (up to the rounding to multiples of 32)
        assert abs(np.median(e) - math.sqrt(lo * hi)) <= 32
        # and the share below the geometric mean is about one half
        assert 0.4 < np.mean(e < math.sqrt(lo * hi)) < 0.6


def test_served_trace_is_poisson_at_the_rate_with_the_recipe_mix():
    from paper_1903_07761_gb300 import cz
    rate, n = 2000.0, 20000
    tr = W._trace(rate, n, seed=4000, max_edge=512)
    t = np.array([r[0] for r in tr])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps: mean 1/rate, coefficient of variation 1
    assert abs(gaps.mean() * rate - 1) < 0.03
    assert abs(gaps.std() / gaps.mean() - 1) < 0.03
    ops = [r[1] for r in tr]
    assert ops.count(cz.OP_COMPRESS) == ops.count(cz.OP_DECOMPRESS) == n // 2
    f64 = np.mean([r[3] for r in tr])
    assert abs(f64 - 0.3) < 0.02
    eps = {r[4] for r in tr}
    assert eps == {1e-3, 1e-4}
    edges = np.array([r[2] for r in tr])
    assert edges.min() >= 32 and edges.max() <= 512 and np.all(edges % 32 == 0)
    # seeded: the same seed gives the same trace
    assert W._trace(rate, n, seed=4000, max_edge=512) == tr
