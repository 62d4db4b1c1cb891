"""Weighted BC on the GPU (sp_graph_set_weights + sp_bc_ex) against the oracle.

Distances bit-exact (sp_sssp against the oracle's Dijkstra), BC within rtol
1e-9 per vertex, exact zeros where the oracle has them, on graphs with few
distinct weights (many equal-length paths) and weights in [1, 100].
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2401_02472_gb300 as sp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def close(got, want, rtol, what=""):
    assert np.all(np.isfinite(got)), what
    err = np.abs(got - want)
    bad = np.nonzero(err > rtol * np.maximum(np.abs(want), 1.0))[0]
    assert bad.size == 0, f"{what}: {bad.size} off, e.g. {bad[:3]} {got[bad[:3]]} vs {want[bad[:3]]}"
    assert np.all(got[want == 0.0] == 0.0), what


def hub_graph():
    base = gen.rmat(12, 8, 5)
    rows = np.repeat(np.arange(base.n), np.diff(base.row_ptr))
    extra = [(0, v) for v in range(1, base.n, 1)]
    return gen.from_edges(base.n, np.concatenate([np.stack([rows, base.col_idx], 1), np.asarray(extra)], 0), "hub")


CASES = {
    "er_w3": (lambda: gen.er(2000, 8000, 1), 3),
    "rmat_w100": (lambda: gen.rmat(13, 8, 2), 100),
    "knn_w100": (lambda: gen.knn2d(4000, 4, 3), 100),
    "grid_w2": (lambda: gen.grid(40, 45), 2),
    "hub_w5": (hub_graph, 5),
    "mixed_w1": (lambda: gen.disjoint_union(gen.star(30), gen.cycle(9), gen.from_edges(5, []), gen.path(17)), 1),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_weighted_bc_and_distances(name):
    make, hi = CASES[name]
    g = make()
    w = gen.edge_weights(g, 7, 1, hi)
    G = sp.Graph(g.row_ptr, g.col_idx)
    sp.sp_graph_set_weights(G.handle, w)
    srcs = gen.sources(g, min(60, int((g.degrees() > 0).sum())), 9)
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    st = sp.sp_bc_ex(G.handle, torch.as_tensor(srcs, device=DEV), out, sp.make_opts())
    want, wdist = oracle.bc_weighted(g, w, srcs)
    close(out.cpu().numpy(), want, 1e-9, name)
    assert st["form"] == sp.SP_FORM_WEIGHTED
    reached = wdist >= 0
    deg = np.diff(g.row_ptr.astype(np.int64))
    assert st["traversed_arcs"] == int((reached * deg[None, :]).sum())
    assert st["reached"] == int(reached.sum())
    dist = np.empty((len(srcs), g.n), np.int32)
    sp.sp_sssp(G.handle, srcs, dist)
    assert np.array_equal(dist, wdist)
    again = torch.empty(g.n, dtype=torch.float64, device=DEV)
    sp.sp_bc(G.handle, torch.as_tensor(srcs, device=DEV), again)  # runs synchronously for weighted graphs
    assert np.array_equal(out.cpu().numpy(), again.cpu().numpy())


def test_unit_weights_match_the_unweighted_path():
    g = gen.rmat(12, 8, 3)
    srcs = gen.sources(g, 50, 1)
    G = sp.Graph(g.row_ptr, g.col_idx)
    sp.sp_graph_set_weights(G.handle, np.ones(g.nnz, np.int32))
    out = np.empty(g.n, np.float64)
    sp.sp_bc_ex(G.handle, srcs, out, sp.make_opts())
    want, _ = oracle.bc(g, srcs)
    close(out, want, 1e-9, "unit weights")


def test_long_distances_grow_the_cap_and_bad_weights_are_refused():
    # a path of 4,000 vertices with weight 100: distances up to 399,900, past
    # the first distance cap (2^18): the call reruns with a larger one
    g = gen.path(4000)
    G = sp.Graph(g.row_ptr, g.col_idx)
    sp.sp_graph_set_weights(G.handle, np.full(g.nnz, 100, np.int32))
    out = np.empty(g.n, np.float64)
    sp.sp_bc_ex(G.handle, np.array([0, 3999, 1234], np.int32), out, sp.make_opts())
    want, _ = oracle.bc_weighted(g, np.full(g.nnz, 100, np.int32), [0, 3999, 1234])
    close(out, want, 1e-9, "long path")
    bad = np.full(g.nnz, 3, np.int32)
    bad[5] = 4  # unlike its reverse arc
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_graph_set_weights(G.handle, bad)
    assert e.value.status == sp.SP_ERR_BAD_GRAPH
    bad[5] = 0
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_graph_set_weights(G.handle, bad)
    assert e.value.status == sp.SP_ERR_BAD_GRAPH
    d = gen.rmat_directed(8, 4, 1)
    D = sp.Graph(d.row_ptr, d.col_idx, flags=sp.SP_GRAPH_DIRECTED)
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_graph_set_weights(D.handle, np.ones(d.nnz, np.int32))
    assert e.value.status == sp.SP_ERR_INVALID_ARG
