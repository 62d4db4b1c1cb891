"""Pins for the PageRank oracle (oracle/pagerank.c): checks from outside it.

- regular graphs (cycles, complete graphs, directed cycles): 1/N at every iteration;
- the fixed point against a direct solve of the linear system
  (I - d M) x = (1 - d)/N 1, M[v][u] = 1/outdeg(u) for each arc u -> v
  (numpy.linalg.solve: a different method from the iteration);
- the star's closed form;
- a directed path with a dangling end: exact after as many iterations as
  vertices (its M is nilpotent);
- sum of ranks = 1 on graphs without dangling vertices;
- planted mistakes are rejected.
"""
import os

import numpy as np
import pytest

import gen
import oracle

D = 0.85


def transition(g):
    """Dense M with M[v][u] = 1/outdeg(u) for every arc u -> v (parallel arcs add up)."""
    m = np.zeros((g.n, g.n))
    deg = np.diff(g.row_ptr.astype(np.int64))
    for u in range(g.n):
        for e in range(g.row_ptr[u], g.row_ptr[u + 1]):
            m[g.col_idx[e], u] += 1.0 / deg[u]
    return m


def solve_fixed_point(g, d=D):
    return np.linalg.solve(np.eye(g.n) - d * transition(g), np.full(g.n, (1.0 - d) / g.n))


@pytest.mark.parametrize("g", [gen.cycle(7), gen.complete(9), gen.from_arcs(5, [(i, (i + 1) % 5) for i in range(5)])],
                         ids=["cycle", "complete", "dcycle"])
def test_regular_graphs_stay_uniform(g):
    for k in (1, 2, 17):
        pr, it, ch = oracle.pagerank(g, D, -1.0, k)  # tol < 0: exactly k iterations
        assert it == k and np.all(np.abs(pr - 1.0 / g.n) <= 1e-16)
        assert ch <= 1e-15
    pr, it, ch = oracle.pagerank(g, D, 0.0, 50)  # stops once an iteration changes nothing (rounding aside)
    assert it <= 2 and ch == 0.0


@pytest.mark.parametrize("g", [gen.er(60, 200, 1), gen.random_small(30, 0.2, 4), gen.rmat_directed(6, 4, 2),
                               gen.random_small_directed(25, 0.15, 5)], ids=["er", "gnp", "drmat", "dgnp"])
def test_fixed_point_matches_a_direct_solve(g):
    pr, it, ch = oracle.pagerank(g, D, 1e-15, 10_000)
    assert ch <= 1e-15 and it < 10_000
    want = solve_fixed_point(g)
    assert np.all(np.abs(pr - want) <= 1e-12 * np.abs(want).max())


@pytest.mark.parametrize("n", [3, 10, 101])
def test_star_closed_form(n):
    g = gen.star(n)
    pr, _, _ = oracle.pagerank(g, D, 1e-16, 100_000)
    centre = (1 + D * (n - 1)) / (n * (1 + D))
    leaf = (1 - D) / n + D * centre / (n - 1)
    assert abs(pr[0] - centre) <= 1e-13 and np.all(np.abs(pr[1:] - leaf) <= 1e-13)


def test_directed_path_with_a_dangling_end():
    n = 6
    g = gen.from_arcs(n, [(i, i + 1) for i in range(n - 1)])
    want = [(1 - D) / n * sum(D ** j for j in range(i + 1)) for i in range(n)]
    pr, it, ch = oracle.pagerank(g, D, 0.0, n)
    assert it == n and np.all(np.abs(pr - want) <= 1e-15)
    pr2, it2, ch2 = oracle.pagerank(g, D, 0.0, n + 3)
    assert ch2 == 0.0 and np.array_equal(pr, pr2)  # nothing changes once the path is settled


def test_mass_is_kept_without_dangling_vertices():
    for g in [gen.er(300, 900, 2), gen.knn2d(400, 4, 3), gen.rmat(9, 8, 1)]:
        g = gen.from_edges(g.n, [(u, v) for u in range(g.n) for v in g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]])
        keep = np.diff(g.row_ptr) > 0
        if not keep.all():  # drop isolated vertices: they keep (1 - d)/N and pass nothing on
            continue
        for k in (1, 5, 40):
            pr, _, _ = oracle.pagerank(g, D, -1.0, k)
            assert abs(pr.sum() - 1.0) <= 1e-12


def test_stopping_rule_and_arguments():
    g = gen.er(200, 800, 3)
    pr1, it1, ch1 = oracle.pagerank(g, D, 1e9, 50)  # the first change is below a huge tol
    assert it1 == 1
    pr, it, ch = oracle.pagerank(g, D, 1e-6, 1000)
    _, _, ch_prev = oracle.pagerank(g, D, 0.0, it - 1)
    assert ch <= 1e-6 < ch_prev
    pr0, it0, _ = oracle.pagerank(g, D, 0.0, 0)
    assert it0 == 0 and np.all(pr0 == 1.0 / g.n)
    with pytest.raises(ValueError):
        oracle.pagerank(g, 1.5, 0.0, 10)


MUTATIONS = {
    "drop_teleport": ("double val = (1.0 - damping) / (double)n + damping * sum;", "double val = damping * sum;"),
    "divide_by_indegree": ("sum = sum + pr[u] / (double)(rp[u + 1] - rp[u]);",
                           "sum = sum + pr[u] / (double)(trp[v + 1] - trp[v]);"),
    "in_place_update": ("            next[v] = val;", "            next[v] = val; pr[v] = val;"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    before, after = MUTATIONS[name]
    path = os.path.join(os.path.dirname(oracle.__file__), "pagerank.c")
    text = open(path).read()
    assert text.count(before) == 1, name
    src = tmp_path / "pr_mutant.c"
    src.write_text(text.replace(before, after))
    lib = oracle.load(oracle.build(force=True, out=str(tmp_path / "m.so"), pr_src=str(src)))
    assert not battery_passes(lib), name


def battery_passes(lib) -> bool:
    """The pins above in compact form: False as soon as one fails."""
    g = gen.random_small_directed(25, 0.15, 5)
    pr, _, _ = oracle.pagerank(g, D, 1e-15, 10_000, lib=lib)
    if not np.all(np.abs(pr - solve_fixed_point(g)) <= 1e-12):
        return False
    g = gen.cycle(11)
    g = gen.from_edges(40, [(i, (i * 7 + 3) % 40) for i in range(40)] + [(i, i + 1) for i in range(39)])
    pr, _, _ = oracle.pagerank(g, D, -1.0, 3, lib=lib)
    if abs(pr.sum() - 1.0) > 1e-12:
        return False
    n = 6
    g = gen.from_arcs(n, [(i, i + 1) for i in range(n - 1)])
    pr, _, _ = oracle.pagerank(g, D, -1.0, n, lib=lib)
    return bool(np.all(np.abs(pr - [(1 - D) / n * sum(D ** j for j in range(i + 1)) for i in range(n)]) <= 1e-15))


def test_unmodified_oracle_passes_the_battery():
    assert battery_passes(oracle.load())
