"""Seeded generators: deterministic, and every graph is a valid undirected CSR."""
import numpy as np
import pytest

import gen


def check_csr(g):
    rp, ci = g.row_ptr.astype(np.int64), g.col_idx.astype(np.int64)
    assert rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 0)
    assert ci.size == 0 or (ci.min() >= 0 and ci.max() < g.n)
    row = np.repeat(np.arange(g.n), np.diff(rp))
    assert not np.any(row == ci), "self-loop"
    key = row * g.n + ci
    assert np.all(np.diff(key) > 0), "rows not strictly sorted (duplicate arc?)"
    rev = np.sort(ci * g.n + row)
    assert np.array_equal(rev, key), "not symmetric"


def test_splitmix64_reference_values():
    # SplitMix64 started at state 0: published first outputs of the generator.
    assert [int(x) for x in gen.draws(0, 0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


@pytest.mark.parametrize("make", [
    lambda: gen.er(2000, 10000, 1),
    lambda: gen.rmat(12, 16, 2),
    lambda: gen.knn2d(3000, 4, 3),
    lambda: gen.grid(7, 9),
    lambda: gen.disjoint_union(gen.star(5), gen.cycle(4), gen.from_edges(2, [])),
])
def test_valid_and_deterministic(make):
    a, b = make(), make()
    check_csr(a)
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)


def test_er_edge_count():
    g = gen.er(2000, 10000, 1)
    assert g.nnz == 20000


def test_knn_degree_at_least_k():
    g, xy = gen.knn2d(4000, 4, 3, return_points=True)
    assert g.degrees().min() >= 4
    # vertex 0's 4 nearest points (by brute force) are among its neighbours
    d2 = ((xy - xy[0]) ** 2).sum(1)
    d2[0] = np.inf
    nearest = np.lexsort((np.arange(g.n), d2))[:4]
    nb = set(g.col_idx[g.row_ptr[0]:g.row_ptr[1]].tolist())
    assert set(nearest.tolist()) <= nb


def test_sources_distinct_and_eligible():
    g = gen.rmat(12, 8, 7)
    s = gen.sources(g, 64, 12)
    assert len(set(s.tolist())) == 64
    assert np.all(g.degrees()[s] >= 1)
    assert np.array_equal(s, gen.sources(g, 64, 12))
    with pytest.raises(ValueError):
        gen.sources(gen.from_edges(3, [(0, 1)]), 3, 1)


def test_poisson_arrivals_rate():
    t = gen.poisson_arrivals(200.0, 60.0, 31)
    assert abs(len(t) / 60.0 - 200.0) < 10.0 and np.all(np.diff(t) > 0)
