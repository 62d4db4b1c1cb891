"""Pins for the sampled-source BC estimator and its bound (oracle.approx_bc).

- the draws are the shared seeded generator's (multiply-shift of SplitMix64);
- unbiasedness: over many seeds the estimates average to BC over all sources;
- coverage: the empirical Bernstein interval holds every vertex for every
  one of many seeds (it is allowed to fail with probability alpha);
- the sample variance of a star's centre from the count of draws that hit it.
"""
import math

import numpy as np

import gen
import oracle


def test_draws_are_multiply_shift_of_splitmix():
    s = oracle.sample_sources(1000, 77, 50)
    x = gen.draws(77, 0, 50)
    assert all(int(s[i]) == (int(x[i]) * 1000) >> 64 for i in range(50))
    assert s.min() >= 0 and s.max() < 1000


def test_estimator_is_unbiased():
    g = gen.er(40, 90, 3)
    exact, _ = oracle.bc(g, range(g.n))
    runs = np.stack([oracle.approx_bc(g, seed, 6)[0] for seed in range(400)])
    mean, sd = runs.mean(axis=0), runs.std(axis=0, ddof=1)
    # every vertex within 5 standard errors of the mean of 400 estimates
    assert np.all(np.abs(mean - exact) <= 5.0 * sd / math.sqrt(400) + 1e-9)


def test_bound_covers_every_vertex():
    for g in [gen.er(120, 400, 5), gen.rmat(7, 6, 2), gen.knn2d(150, 4, 1)]:
        n = g.n
        exact = oracle.bc(g, range(n))[0] / ((n - 1.0) * (n - 2.0))
        for seed in range(12):
            est, half, _ = oracle.approx_bc(g, seed, 200, alpha=0.1)
            assert np.all(np.abs(est / ((n - 1.0) * (n - 2.0)) - exact) <= half), (g.name, seed)


def test_star_centre_variance():
    n = 30
    g = gen.star(n)
    k = 64
    _, half, deltas = oracle.approx_bc(g, 11, k)
    srcs = oracle.sample_sources(n, 11, k)
    m = int((srcs == 0).sum())  # draws of the centre: it depends on nothing then
    r = n / (n - 1.0)  # a leaf source gives the centre delta = n - 2, i.e. Y = n / (n - 1)
    mean = (k - m) / k * r
    var = (k - m) * (r - mean) ** 2 / (k - 1) + m * mean ** 2 / (k - 1)
    L = math.log(4.0 * n / 0.1)
    assert abs(half - (math.sqrt(2 * var * L / k) + 7 * r * L / (3 * (k - 1)))) <= 1e-12
    assert np.all(deltas[:, 1:] == 0.0)  # leaves lie on no shortest path
