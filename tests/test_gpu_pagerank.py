"""PageRank on the GPU (sp_pagerank) against the CPU oracle (oracle/pagerank.c).

Both sides run the same number of iterations (tol < 0: exactly max_iter)
and then converge with a tolerance; ranks agree within rtol 1e-10 per vertex,
from the rounding of FP64 sums taken in different orders (warp trees on long
rows) and a per-vertex 1/outdeg, bounded over the iterations by the
damping's contraction; iteration counts agree.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2401_02472_gb300 as sp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
RTOL = 1e-10


def close(got, want, what=""):
    err = np.abs(got - want)
    assert np.all(err <= RTOL * np.abs(want)), f"{what}: max rel err {np.max(err / np.abs(want))}"


def hub_graph():
    base = gen.rmat(13, 8, 5)
    rows = np.repeat(np.arange(base.n), np.diff(base.row_ptr))
    extra = [(0, v) for v in range(1, base.n)] + [(1, v) for v in range(2, base.n, 2)]
    return gen.from_edges(base.n, np.concatenate([np.stack([rows, base.col_idx], 1), np.asarray(extra)], 0), "hub")


CASES = {
    "er2000": (lambda: gen.er(2000, 10000, 1), 0),
    "rmat14": (lambda: gen.rmat(14, 16, 2), 0),
    "hub": (hub_graph, 0),
    "knn": (lambda: gen.knn2d(20000, 4, 3), 0),
    "drmat12": (lambda: gen.rmat_directed(12, 8, 2), sp.SP_GRAPH_DIRECTED),
    "mixed": (lambda: gen.disjoint_union(gen.star(40), gen.cycle(9), gen.from_edges(5, []), gen.path(17)), 0),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_pagerank_fixed_iterations_and_convergence(name):
    make, flags = CASES[name]
    g = make()
    G = sp.Graph(g.row_ptr, g.col_idx, flags=flags)
    for k in (1, 2, 7, 30):
        out = torch.empty(g.n, dtype=torch.float64, device=DEV)
        it, ch = sp.sp_pagerank(G.handle, out, 0.85, -1.0, k)
        want, wit, wch = oracle.pagerank(g, 0.85, -1.0, k)
        assert it == wit == k
        close(out.cpu().numpy(), want, f"{name} after {k} iterations")
        # the change sums |PR' - PR| over nearly equal values: each term carries
        # the ranks' rounding (a few ulps of the largest rank) as absolute error
        assert abs(ch - wch) <= 1e-9 * wch + g.n * 8.0 * np.finfo(float).eps * want.max()
    host = np.empty(g.n, np.float64)
    it, ch = sp.sp_pagerank(G.handle, host, 0.85, 1e-10, 1000)
    want, wit, wch = oracle.pagerank(g, 0.85, 1e-10, 1000)
    assert it == wit and ch <= 1e-10
    close(host, want, f"{name} converged")
    again = np.empty(g.n, np.float64)
    sp.sp_pagerank(G.handle, again, 0.85, 1e-10, 1000)
    assert np.array_equal(host, again)  # bit-identical run to run


def test_pagerank_asynchronous_and_edge_cases():
    g = gen.rmat(12, 8, 3)
    G = sp.Graph(g.row_ptr, g.col_idx)
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    assert sp.sp_pagerank(G.handle, out, 0.85, 1e-12, 500, want_result=False) is None
    sp.sp_graph_sync(G.handle)
    want, _, _ = oracle.pagerank(g, 0.85, 1e-12, 500)
    close(out.cpu().numpy(), want, "asynchronous")
    it, ch = sp.sp_pagerank(G.handle, out, 0.85, 0.0, 0)  # no iteration: the start value
    assert it == 0 and np.all(out.cpu().numpy() == 1.0 / g.n)
    it, _ = sp.sp_pagerank(G.handle, out, 0.0, -1.0, 3)  # damping 0: uniform teleport
    assert np.all(np.abs(out.cpu().numpy() - 1.0 / g.n) <= 1e-18)
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_pagerank(G.handle, out, 1.5, 0.0, 3)
    assert e.value.status == sp.SP_ERR_INVALID_ARG
