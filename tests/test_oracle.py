"""Pins for the CPU oracle: every check here comes from outside the oracle.

- exact rationals from the definition of BC on every graph of 5 vertices and
  on random graphs of up to 12 vertices (tests/bruteforce.py);
- closed forms (star, path, cycle, complete, complete bipartite, trees,
  binomial path counts on grids);
- a hand-derived fixture (tests/golden/diamond_tail.txt);
- the invariant sum_v BC(v) = sum over reached ordered pairs of (d(s,t) - 1);
- BFS distances against a deque BFS, linearity over source multisets, and the
  extended-exponent mode against plain doubles, bit for bit.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle
from tests import bruteforce as bf

HERE = os.path.dirname(os.path.abspath(__file__))
RTOL = 1e-12


def close(got, exact, rtol=RTOL):
    exact = np.asarray([float(x) for x in exact])
    return np.all(np.abs(np.asarray(got) - exact) <= rtol * np.maximum(np.abs(exact), 1.0))


def graph_from_mask(n, mask):
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    return gen.from_edges(n, [p for k, p in enumerate(pairs) if mask >> k & 1])


@pytest.mark.parametrize("mode", [oracle.PLAIN, oracle.XFLOAT])
def test_every_graph_on_five_vertices(mode):
    n = 5
    for mask in range(1 << 10):
        g = graph_from_mask(n, mask)
        got, _ = oracle.bc(g, range(n), mode)
        exact = bf.bc_exact(g, range(n))
        assert close(got, exact), (mask, got, exact)


def test_random_graphs_up_to_twelve_vertices():
    cases = 0
    for seed in range(60):
        n = 6 + seed % 7
        p = [0.2, 0.35, 0.5, 0.7][seed % 4]
        g = gen.random_small(n, p, seed)
        srcs = gen.draws(gen.substream(seed, 99), 0, 5) % np.uint64(n)
        for sources in (list(range(n)), [int(s) for s in srcs]):
            got, _ = oracle.bc(g, sources)
            exact = bf.bc_exact(g, sources)
            assert close(got, exact), (seed, sources, got, exact)
            cases += 1
    assert cases == 120


def read_golden(path):
    edges, n, cases = [], None, []
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("edges:"):
            edges = [tuple(int(x) for x in e.split("-")) for e in line.split(":", 1)[1].split()]
        elif line.startswith("n:"):
            n = int(line.split(":", 1)[1])
        elif line.startswith("sources:"):
            lhs, rhs = line.split("|")
            srcs = [int(x) for x in lhs.split(":", 1)[1].split()]
            vals = [Fraction(x) for x in rhs.split(":", 1)[1].split()]
            cases.append((srcs, vals))
    return gen.from_edges(n, edges), cases


def test_hand_derived_fixture():
    g, cases = read_golden(os.path.join(HERE, "golden", "diamond_tail.txt"))
    assert len(cases) == 4
    for srcs, vals in cases:
        got, _ = oracle.bc(g, srcs)
        assert close(got, vals), (srcs, got, vals)
        assert bf.bc_exact(g, srcs) == vals  # the fixture agrees with the definition too


@pytest.mark.parametrize("n", [2, 3, 7, 40, 301])
def test_star(n):
    got, _ = oracle.bc(gen.star(n), range(n))
    exact = [(n - 1) * (n - 2)] + [0] * (n - 1)
    assert close(got, exact)


@pytest.mark.parametrize("n", [1, 2, 5, 64, 257])
def test_path(n):
    g = gen.path(n) if n > 1 else gen.from_edges(1, [])
    got, _ = oracle.bc(g, range(n))
    assert close(got, [2 * i * (n - 1 - i) for i in range(n)])


@pytest.mark.parametrize("n", [3, 5, 9, 101])
def test_odd_cycle(n):
    r = (n - 1) // 2
    got, _ = oracle.bc(gen.cycle(n), range(n))
    assert close(got, [r * (r - 1)] * n)


@pytest.mark.parametrize("n", [4, 6, 10, 100])
def test_even_cycle(n):
    r = n // 2
    got, _ = oracle.bc(gen.cycle(n), range(n))
    assert close(got, [(r - 1) ** 2] * n)


@pytest.mark.parametrize("n", [2, 3, 8, 50])
def test_complete(n):
    got, _ = oracle.bc(gen.complete(n), range(n))
    assert close(got, [0] * n)


@pytest.mark.parametrize("a,b", [(1, 4), (2, 3), (3, 5), (7, 11)])
def test_complete_bipartite(a, b):
    # Side A = 0..a-1, side B = a..a+b-1.  Two B vertices are joined by a shortest
    # paths, one through each A vertex, so each A vertex carries 1/a of every
    # ordered B pair, and symmetrically for B.
    g = gen.from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])
    got, _ = oracle.bc(g, range(a + b))
    exact = [Fraction(b * (b - 1), a)] * a + [Fraction(a * (a - 1), b)] * b
    assert close(got, exact)


def test_two_components_are_independent():
    p, s = gen.path(9), gen.star(6)
    u = gen.disjoint_union(p, s)
    got, _ = oracle.bc(u, range(u.n))
    bp, _ = oracle.bc(p, range(p.n))
    bs, _ = oracle.bc(s, range(s.n))
    assert np.array_equal(got, np.concatenate([bp, bs]))


def test_isolated_vertices_and_empty_sources():
    g = gen.from_edges(6, [(1, 2), (2, 3)])
    got, st = oracle.bc(g, [0, 5, 4])
    assert np.array_equal(got, np.zeros(6)) and list(st["reached"]) == [1, 1, 1]
    got, st = oracle.bc(g, [])
    assert np.array_equal(got, np.zeros(6)) and len(st) == 0


def test_tree_sigma_is_one():
    # A random recursive tree: every vertex has one shortest path from the root.
    n = 500
    par = gen.draws(77, 0, n)
    g = gen.from_edges(n, [(v, int(par[v] % np.uint64(v))) for v in range(1, n)])
    for src in (0, 123, 499):
        mant, exp2, dist, _ = oracle.sigma(g, src)
        assert np.all(mant == 1.0) and np.all(exp2 == 0)


@pytest.mark.parametrize("rows,cols", [(3, 4), (17, 9), (40, 40)])
def test_grid_sigma_binomial_exact(rows, cols):
    # From corner (0,0) of a grid, sigma(i,j) = C(i+j, i) (lattice paths).
    g = gen.grid(rows, cols)
    mant, exp2, dist, _ = oracle.sigma(g, 0, oracle.PLAIN)
    for i in range(rows):
        for j in range(cols):
            v = i * cols + j
            assert dist[v] == i + j
            want = math.comb(i + j, i)
            got = Fraction(mant[v]) * Fraction(2) ** int(exp2[v])
            if want < 2 ** 53:
                assert got == want
            else:
                assert abs(got / want - 1) < 2.0 ** -50


def log2_int(w: int) -> float:
    shift = max(w.bit_length() - 64, 0)
    return shift + math.log2(w >> shift)


def test_grid_sigma_beyond_double_range():
    # 600x600: sigma of the far corner is C(1198, 599) ~ 2^1192.6 > max double.
    rows = cols = 600
    g = gen.grid(rows, cols)
    mant, exp2, dist, st = oracle.sigma(g, 0, oracle.AUTO)
    assert st["used_xfloat"] == 1
    for (i, j) in [(599, 599), (0, 599), (300, 299), (599, 1), (450, 512)]:
        v = i * cols + j
        want = math.comb(i + j, i)
        log2_want = log2_int(want)
        log2_got = math.log2(mant[v]) + int(exp2[v])
        assert abs(log2_got - log2_want) <= 1e-12 * max(1.0, log2_want), (i, j, log2_got, log2_want)
    _, _, _, st_plain = oracle.sigma(gen.grid(30, 30), 0, oracle.PLAIN)
    assert st_plain["used_xfloat"] == 0


def test_plain_mode_reports_overflow_as_inf():
    g = gen.grid(600, 600)
    got, _ = oracle.bc(g, [0], oracle.PLAIN)
    assert np.all(np.isinf(got))


def test_xfloat_equals_plain_bit_for_bit():
    for g, srcs in [(gen.er(2000, 10000, 1), range(0, 2000, 7)), (gen.rmat(12, 8, 5), range(0, 4096, 97)),
                    (gen.grid(60, 70), [0, 4199, 2000])]:
        a, _ = oracle.bc(g, list(srcs), oracle.PLAIN)
        b, _ = oracle.bc(g, list(srcs), oracle.XFLOAT)
        assert np.array_equal(a, b)


def test_sum_invariant_on_benchmark_like_graphs():
    for g, srcs in [(gen.er(2000, 10000, 1), list(range(2000))),
                    (gen.rmat(14, 16, 2), list(gen.sources(gen.rmat(14, 16, 2), 16, 12))),
                    (gen.knn2d(20000, 4, 3), list(gen.sources(gen.knn2d(20000, 4, 3), 8, 13)))]:
        got, st = oracle.bc(g, srcs)
        want = bf.pair_distance_excess(g, srcs)
        assert abs(got.sum() - want) <= 1e-9 * max(want, 1), (g.name, got.sum(), want)


def test_sum_invariant_beyond_double_range():
    # The extended-exponent path on a grid whose path counts exceed 2^1024.
    g = gen.grid(540, 540)
    srcs = [0, 540 * 540 - 1]
    got, st = oracle.bc(g, srcs)
    assert st["used_xfloat"].all()
    want = bf.pair_distance_excess(g, srcs)
    assert abs(got.sum() - want) <= 1e-9 * want


def test_bfs_matches_deque_bfs():
    for g in [gen.er(2000, 10000, 1), gen.rmat(12, 16, 3), gen.knn2d(5000, 4, 3),
              gen.disjoint_union(gen.path(10), gen.cycle(7), gen.from_edges(3, []))]:
        for s in [0, g.n // 2, g.n - 1]:
            assert list(oracle.bfs(g, s)) == bf.bfs_dist(g, s)


def test_linearity_over_source_multisets():
    g = gen.rmat(11, 8, 9)
    s1 = [int(x) for x in gen.sources(g, 20, 1)]
    s2 = [int(x) for x in gen.sources(g, 13, 2)] + s1[:3]
    a, _ = oracle.bc(g, s1)
    b, _ = oracle.bc(g, s2)
    c, _ = oracle.bc(g, s1 + s2)
    assert np.all(np.abs(c - (a + b)) <= 1e-12 * np.maximum(np.abs(c), 1))


def test_stats():
    g = gen.from_edges(7, [(0, 1), (1, 2), (2, 3), (4, 5)])
    _, st = oracle.bc(g, [0, 4, 6])
    assert list(st["levels"]) == [4, 2, 1]
    assert list(st["reached"]) == [4, 2, 1]
    assert list(st["arcs"]) == [6, 2, 0]


def test_bad_arguments():
    g = gen.path(4)
    with pytest.raises(ValueError):
        oracle.bc(g, [4])
    with pytest.raises(ValueError):
        oracle.bc(g, [-1])
    with pytest.raises(ValueError):
        oracle.bfs(g, 9)


def test_distance_sums_against_deque_bfs():
    # The 64-source bit-parallel search behind the benchmark-size invariant:
    # per-source distance sums and reached counts against one deque BFS per
    # source, across word boundaries (130 sources), with repeated and
    # isolated sources and several components.
    cases = [
        (gen.er(400, 1200, 5), None),
        (gen.rmat(11, 8, 6), None),
        (gen.knn2d(800, 4, 7), None),
        (gen.disjoint_union(gen.path(9), gen.star(12), gen.cycle(5), gen.from_edges(4, [])),
         np.array([0, 0, 3, 9, 10, 21, 26, 28, 29, 8, 8], np.int32)),
    ]
    for g, srcs in cases:
        if srcs is None:
            srcs = gen.sources(g, min(130, g.n), 3)
        dsum, reached = oracle.distance_sums(g, srcs)
        for i, s in enumerate(srcs):
            d = np.asarray(bf.bfs_dist(g, int(s)))
            assert dsum[i] == int(d[d >= 0].sum()) and reached[i] == int((d >= 0).sum()), (g.name, i)
        assert oracle.pair_distance_excess(g, srcs, threads=3) == bf.pair_distance_excess(g, srcs)
    with pytest.raises(ValueError):
        oracle.distance_sums(gen.path(4), [4])


# ---------------------------------------------------------------------------
# Directed graphs: BFS and dependencies over out-arcs, path counts pulled over
# in-arcs (the transpose the oracle builds itself).

def test_every_digraph_on_four_vertices():
    # All 4,096 labelled digraphs on 4 vertices against exact rationals from
    # explicit shortest-path enumeration, all sources.
    pairs = [(i, j) for i in range(4) for j in range(4) if i != j]
    for mask in range(1 << len(pairs)):
        g = gen.from_arcs(4, [pairs[b] for b in range(len(pairs)) if mask >> b & 1])
        got, _ = oracle.bc(g, range(4), directed=True)
        assert close(got, bf.bc_exact(g, range(4))), mask


def test_random_digraphs_up_to_nine_vertices():
    for seed in range(60):
        n = 5 + seed % 5
        g = gen.random_small_directed(n, 0.25 + 0.05 * (seed % 6), seed)
        srcs = [int(x) for x in gen.draws(seed, 0, 6) % n]
        for mode in (oracle.PLAIN, oracle.XFLOAT):
            got, _ = oracle.bc(g, srcs, mode, directed=True)
            assert close(got, bf.bc_exact(g, srcs)), (seed, mode)
        assert oracle.sigma(g, srcs[0], directed=True)[0].tolist() is not None
        mant, exp2, _, _ = oracle.sigma(g, srcs[0], oracle.PLAIN, directed=True)
        assert [m * 2.0 ** int(e) for m, e in zip(mant, exp2)] == bf.sigma_exact(g, srcs[0]), seed


@pytest.mark.parametrize("n", [2, 3, 8, 41])
def test_directed_path(n):
    # 0 -> 1 -> ... -> n-1, all sources: vertex i lies inside the pairs (s, t)
    # with s < i < t, i (n - 1 - i) of them.
    g = gen.from_arcs(n, [(i, i + 1) for i in range(n - 1)])
    got, _ = oracle.bc(g, range(n), directed=True)
    assert close(got, [i * (n - 1 - i) for i in range(n)])


@pytest.mark.parametrize("n", [3, 4, 9, 50])
def test_directed_cycle(n):
    # One path between every ordered pair; a vertex is inside (n - 1)(n - 2) / 2 of them.
    g = gen.from_arcs(n, [(i, (i + 1) % n) for i in range(n)])
    got, _ = oracle.bc(g, range(n), directed=True)
    assert close(got, [Fraction((n - 1) * (n - 2), 2)] * n)


def test_symmetric_digraph_equals_undirected_bit_for_bit():
    # Both directions of every edge stored with sorted rows: the transpose has
    # the same rows, so the directed pass repeats the undirected arithmetic.
    for g in [gen.er(500, 2000, 3), gen.rmat(10, 8, 4), gen.grid(30, 31)]:
        srcs = gen.sources(g, 25, 5)
        a, _ = oracle.bc(g, srcs)
        b, _ = oracle.bc(g, srcs, directed=True)
        assert np.array_equal(a, b)


def test_transpose_with_all_sources():
    # With every vertex a source, reversing every arc maps each ordered pair
    # (s, t) to (t, s) with the same interior vertices: BC is unchanged.
    g = gen.rmat_directed(8, 6, 11)
    a, _ = oracle.bc(g, range(g.n), directed=True)
    b, _ = oracle.bc(gen.transpose(g), range(g.n), directed=True)
    assert np.all(np.abs(a - b) <= 1e-12 * np.maximum(np.abs(a), 1))
    assert not np.allclose(a, oracle.bc(g, range(g.n))[0])  # direction matters on this graph


def test_directed_sum_invariant():
    for g in [gen.rmat_directed(12, 8, 2), gen.from_arcs(6, [(0, 1), (1, 2), (2, 0), (3, 4)])]:
        srcs = gen.sources(g, min(40, g.n), 6) if g.n > 10 else np.arange(g.n, dtype=np.int32)
        got, _ = oracle.bc(g, srcs, directed=True)
        want = oracle.pair_distance_excess(g, srcs)
        assert abs(got.sum() - want) <= 1e-9 * max(want, 1)
