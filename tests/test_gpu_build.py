"""CSR construction on the GPU against the numpy builder of the input generators.

sp_graph_from_edges must give exactly the CSR that gen.from_edges gives
(symmetrised, self-loops dropped, repeats kept once, rows sorted), and
SP_GRAPH_SORT_ROWS must sort the rows of a copied CSR, on rows short enough
for one warp, for one block, and long enough to need merge passes.
"""
import numpy as np
import pytest
import torch

import gen
import paper_2401_02472_gb300 as sp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def edges_of(g):
    """Each arc of a CSR as an edge (so every undirected edge appears twice)."""
    src = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(g.row_ptr))
    return src, g.col_idx.astype(np.int32)


def assert_same_csr(G, g):
    rp, ci = G.csr()
    assert np.array_equal(rp, g.row_ptr) and np.array_equal(ci, g.col_idx)


def random_edges(n, m, seed, extra=()):
    d = gen.draws(seed, 0, 2 * m) % np.uint64(n)
    e = np.stack([d[:m], d[m:]], 1).astype(np.int64)
    e = np.concatenate([e, e[: m // 5][:, ::-1], e[: m // 7], np.asarray(extra, np.int64).reshape(-1, 2)], 0)
    return e[:, 0].astype(np.int32), e[:, 1].astype(np.int32)


@pytest.mark.parametrize("device_input", [False, True])
def test_edge_list_matches_numpy_builder(device_input):
    n = 3000
    hub = [(0, v) for v in range(1, n)] + [(v, 0) for v in range(1, n, 3)] + [(7, 7), (8, 8)]
    src, dst = random_edges(n, 20000, 41, hub)
    want = gen.from_edges(n, np.stack([src, dst], 1))
    if device_input:
        src, dst = torch.as_tensor(src, device=DEV), torch.as_tensor(dst, device=DEV)
    G = sp.Graph.from_edges(src, dst, n)
    assert_same_csr(G, want)
    assert G.info["sorted_rows"] == 1 and G.info["has_duplicates"] == 0 and G.info["has_self_loops"] == 0


def test_edge_list_long_rows_need_merges():
    # rows of 40,000 and 9,000 arcs (4096-arc pieces, 2-4 merge passes) in a random order
    n = 50000
    rng_order = gen.draws(gen.substream(5, 1), 0, 49000)
    nb = (np.argsort(rng_order, kind="stable") + 1).astype(np.int64)
    extra = [(0, int(v)) for v in nb[:40000]] + [(int(v), 1) for v in nb[40000:49000]]
    src, dst = random_edges(n, 30000, 43, extra)
    G = sp.Graph.from_edges(src, dst, n)
    assert_same_csr(G, gen.from_edges(n, np.stack([src, dst], 1)))


def test_edge_list_rmat20_roundtrip():
    g = gen.workload_graph("rmat20")
    src, dst = edges_of(g)
    G = sp.Graph.from_edges(torch.as_tensor(src, device=DEV), torch.as_tensor(dst, device=DEV), g.n)
    assert_same_csr(G, g)


def test_edge_list_edge_cases():
    G = sp.Graph.from_edges(np.zeros(0, np.int32), np.zeros(0, np.int32), 5)
    rp, ci = G.csr()
    assert np.array_equal(rp, np.zeros(6, np.int32)) and ci.size == 0
    G = sp.Graph.from_edges(np.array([3, 3], np.int32), np.array([3, 3], np.int32), 4)  # loops only
    assert G.nnz == 0
    with pytest.raises(sp.StarbcError) as e:
        sp.Graph.from_edges(np.array([0, 1], np.int32), np.array([1, 9], np.int32), 5)
    assert e.value.status == sp.SP_ERR_BAD_GRAPH


def test_sort_rows_flag():
    g = gen.disjoint_union(gen.rmat(13, 8, 5), gen.star(9000), gen.star(40))
    # shuffle every row with a seeded key (deterministic)
    key = gen.draws(gen.substream(9, 2), 0, g.nnz)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    order = np.lexsort((key, rows))
    shuffled = g.col_idx[order].astype(np.int32)
    assert not np.array_equal(shuffled, g.col_idx)
    plain = sp.Graph(g.row_ptr, shuffled)
    assert plain.info["sorted_rows"] == 0
    G = sp.Graph(g.row_ptr, shuffled, flags=sp.SP_GRAPH_SORT_ROWS | sp.SP_GRAPH_CHECK_SYMMETRIC)
    assert G.info["sorted_rows"] == 1 and G.info["symmetric"] == 1
    assert_same_csr(G, g)


def test_bc_on_built_graph_is_identical():
    g = gen.er(4000, 30000, 17)
    src, dst = edges_of(g)
    G1 = sp.Graph(g.row_ptr, g.col_idx)
    G2 = sp.Graph.from_edges(src, dst, g.n)
    srcs = torch.as_tensor(gen.sources(g, 100, 3), device=DEV)
    outs = []
    for G in (G1, G2):
        out = torch.empty(g.n, dtype=torch.float64, device=DEV)
        sp.sp_bc_ex(G.handle, srcs, out, sp.make_opts(form=sp.SP_FORM_BATCHED, batch=64))
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
