"""Pins for the weighted-BC oracle (oracle/weighted.c): checks from outside it.

- exact rationals from the definition (weighted Floyd-Warshall, every
  shortest path listed) on random graphs with small weights (many ties),
  undirected and directed;
- all weights 1: the unweighted oracle, bit for bit;
- scaling every weight by a constant changes nothing;
- paths (one shortest path per pair) and a weighted shortcut by hand;
- distances against the definition (Floyd-Warshall);
- planted mistakes are rejected.
"""
import os

import numpy as np
import pytest

import gen
import oracle
from tests import bruteforce as bf


def weights_for(g, seed, lo=1, hi=3, symmetric=True):
    return gen.edge_weights(g, seed, lo, hi, symmetric)


def close(got, exact, rtol=1e-12):
    exact = np.asarray([float(x) for x in exact])
    return np.all(np.abs(np.asarray(got) - exact) <= rtol * np.maximum(np.abs(exact), 1.0))


def test_random_graphs_against_the_definition():
    for seed in range(40):
        n = 5 + seed % 6
        directed = seed % 2 == 1
        g = gen.random_small_directed(n, 0.3, seed) if directed else gen.random_small(n, 0.45, seed)
        w = weights_for(g, seed, 1, 3, symmetric=not directed)
        got, dist = oracle.bc_weighted(g, w, range(n), directed=directed)
        assert close(got, bf.bc_exact_weighted(g, w, range(n))), seed


def test_unit_weights_are_the_bfs_program():
    for g in [gen.er(600, 2400, 1), gen.rmat(10, 8, 2), gen.grid(20, 23)]:
        srcs = gen.sources(g, 20, 3)
        a, _ = oracle.bc(g, srcs, oracle.PLAIN)
        b, dist = oracle.bc_weighted(g, np.ones(g.nnz, np.int32), srcs)
        assert np.array_equal(a, b)
        assert all(np.array_equal(dist[i], oracle.bfs(g, int(s))) for i, s in enumerate(srcs))
    g = gen.rmat_directed(10, 6, 3)
    srcs = gen.sources(g, 20, 4)
    a, _ = oracle.bc(g, srcs, oracle.PLAIN, directed=True)
    b, _ = oracle.bc_weighted(g, np.ones(g.nnz, np.int32), srcs, directed=True)
    assert np.array_equal(a, b)


def test_scaling_the_weights_changes_nothing():
    g = gen.er(300, 1200, 7)
    w = weights_for(g, 7, 1, 9)
    srcs = gen.sources(g, 30, 8)
    a, da = oracle.bc_weighted(g, w, srcs)
    b, db = oracle.bc_weighted(g, w * 7, srcs)
    assert np.array_equal(a, b) and np.array_equal(da * 7, db)


def test_hand_cases():
    # a path with arbitrary weights keeps one shortest path per pair
    n = 9
    g = gen.path(n)
    w = (np.arange(g.nnz) % 5 + 1).astype(np.int32)
    rows = np.repeat(np.arange(n), np.diff(g.row_ptr))
    w = np.array([1 + (min(u, v) * 3) % 5 for u, v in zip(rows, g.col_idx)], np.int32)
    got, _ = oracle.bc_weighted(g, w, range(n))
    assert close(got, [2 * i * (n - 1 - i) for i in range(n)])
    # a square 0-1-2-3-0 with a heavy edge 0-1 (weight 5): 0 reaches 1 through 3 and 2
    g = gen.from_edges(4, [(0, 1), (1, 2), (2, 3), (3, 0)])
    rows = np.repeat(np.arange(4), np.diff(g.row_ptr))
    w = np.array([5 if {u, v} == {0, 1} else 1 for u, v in zip(rows, g.col_idx)], np.int32)
    got, dist = oracle.bc_weighted(g, w, [0])
    assert list(dist[0]) == [0, 3, 2, 1]
    assert list(got) == [0.0, 0.0, 1.0, 2.0]


def test_distances_match_floyd_warshall():
    g = gen.random_small(12, 0.3, 5)
    w = weights_for(g, 5, 1, 20)
    _, dist = oracle.bc_weighted(g, w, range(12))
    d = [[bf.INF] * 12 for _ in range(12)]
    for v in range(12):
        d[v][v] = 0
        for e in range(g.row_ptr[v], g.row_ptr[v + 1]):
            d[v][g.col_idx[e]] = min(d[v][g.col_idx[e]], int(w[e]))
    for k in range(12):
        for i in range(12):
            for j in range(12):
                d[i][j] = min(d[i][j], d[i][k] + d[k][j])
    assert all(dist[i][j] == (d[i][j] if d[i][j] < bf.INF else -1) for i in range(12) for j in range(12))


MUTATIONS = {
    "parent_test_off_by_one": ("if (dist[u] >= 0 && dist[u] + pw[e] == dist[v])",
                               "if (dist[u] >= 0 && dist[u] + 1 == dist[v])"),
    "child_ignores_weight": ("if (dist[x] == dist[v] + w[e])", "if (dist[x] > dist[v])"),
    "relax_ignores_weight": ("int64_t nd = t.d + w[e];", "int64_t nd = t.d + 1;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    before, after = MUTATIONS[name]
    path = os.path.join(os.path.dirname(oracle.__file__), "weighted.c")
    text = open(path).read()
    assert text.count(before) == 1, name
    src = tmp_path / "w_mutant.c"
    src.write_text(text.replace(before, after))
    lib = oracle.load(oracle.build(force=True, out=str(tmp_path / "m.so"), w_src=str(src)))
    caught = False
    for seed in range(10):
        g = gen.random_small(8, 0.45, seed)
        w = weights_for(g, seed, 1, 3)
        try:
            got, _ = oracle.bc_weighted(g, w, range(8), lib=lib)
        except ValueError:
            caught = True
            break
        if not close(got, bf.bc_exact_weighted(g, w, range(8))):
            caught = True
            break
    assert caught, name
