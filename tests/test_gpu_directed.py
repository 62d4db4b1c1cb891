"""Directed graphs (SP_GRAPH_DIRECTED) against the CPU oracle's directed mode.

BFS and dependencies follow out-arcs, path counts are pulled over in-arcs;
the library builds the in-arcs on the GPU.  Levels bit-exact, path counts
exact below 2^53, BC within rtol 1e-9 (FP64 dependencies) / 1e-4 (FP32), in
every form and driver, through the C ABI.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2401_02472_gb300 as sp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
RTOL = {sp.SP_FP64: 1e-9, sp.SP_FP32_DELTA: 1e-4}


def close(got, want, rtol, what=""):
    assert np.all(np.isfinite(got)), what
    err = np.abs(got - want)
    bad = np.nonzero(err > rtol * np.maximum(np.abs(want), 1.0))[0]
    assert bad.size == 0, f"{what}: {bad.size} vertices off, e.g. {bad[:3]} {got[bad[:3]]} vs {want[bad[:3]]}"
    assert np.all(got[want == 0.0] == 0.0), what


def hub_digraph():
    """Directed RMAT plus a vertex with 6,000 out-arcs and 5,000 in-arcs, and
    sinks and sources of arcs only (rows split into segments in every form)."""
    base = gen.rmat_directed(13, 6, 9)
    rows = np.repeat(np.arange(base.n), np.diff(base.row_ptr))
    arcs = [np.stack([rows, base.col_idx], 1),
            np.array([(0, v) for v in range(1, 6001)]), np.array([(v, 0) for v in range(3000, 8000)])]
    return gen.from_arcs(base.n, np.concatenate(arcs, 0), "dhub")


GRAPHS = {
    "drmat12": lambda: gen.rmat_directed(12, 8, 2),
    "dsmall": lambda: gen.random_small_directed(40, 0.08, 3),
    "dcycle_path": lambda: gen.from_arcs(60, [(i, (i + 1) % 30) for i in range(30)] +
                                         [(30 + i, 31 + i) for i in range(29)] + [(5, 30), (59, 7)]),
    "dhub": hub_digraph,
}
_cache = {}


def graph(name):
    if name not in _cache:
        g = GRAPHS[name]()
        _cache[name] = (g, sp.Graph(g.row_ptr, g.col_idx, flags=sp.SP_GRAPH_DIRECTED))
    return _cache[name]


def gpu_bc(G, srcs, precision, form, batch=0, **kw):
    out = torch.empty(G.n, dtype=torch.float64, device=DEV)
    st = sp.sp_bc_ex(G.handle, torch.as_tensor(np.asarray(srcs, np.int32), device=DEV), out,
                     sp.make_opts(precision=precision, form=form, batch=batch, **kw))
    torch.cuda.synchronize()
    return out.cpu().numpy(), st


def pick_sources(g, k, seed):
    return gen.sources(g, min(k, int((g.degrees() > 0).sum())), seed)


FORMS = [(sp.SP_FORM_PLAIN, 0, dict(driver=sp.SP_DRIVER_PERSISTENT)),
         (sp.SP_FORM_PLAIN, 0, dict(driver=sp.SP_DRIVER_GRAPH)),
         (sp.SP_FORM_BATCHED, 32, {}), (sp.SP_FORM_BATCHED, 128, {}),
         (sp.SP_FORM_SMALL, 0, {})]


@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
@pytest.mark.parametrize("fi", range(len(FORMS)))
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_directed_bc(name, fi, precision):
    form, batch, kw = FORMS[fi]
    g, G = graph(name)
    if form == sp.SP_FORM_SMALL and g.n > 14000:
        pytest.skip("beyond the small form")
    srcs = pick_sources(g, 150 if form == sp.SP_FORM_BATCHED else 30, 7)
    got, st = gpu_bc(G, srcs, precision, form, batch, **kw)
    want, ost = oracle.bc(g, srcs, directed=True)
    close(got, want, RTOL[precision], f"{name} form {form} B={batch} {kw}")
    assert st["traversed_arcs"] == int(ost["arcs"].sum())
    assert st["reached"] == int(ost["reached"].sum())
    assert st["max_levels"] == int(ost["levels"].max())


@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_directed_levels_and_counts(name):
    g, G = graph(name)
    srcs = np.unique(np.array([0, 1, g.n // 2, g.n - 1], np.int32))
    dist = torch.empty((len(srcs), g.n), dtype=torch.int32, device=DEV)
    sp.sp_bfs(G.handle, torch.as_tensor(srcs, device=DEV), dist)
    got = dist.cpu().numpy()
    for i, s in enumerate(srcs):
        assert np.array_equal(got[i], oracle.bfs(g, int(s))), (name, s)
        mant = np.empty(g.n, np.float64)
        e2 = np.empty(g.n, np.int64)
        sp.sp_sigma(G.handle, int(s), mant, e2)
        om, oe, _, _ = oracle.sigma(g, int(s), directed=True)
        assert np.array_equal(mant, om) and np.array_equal(e2, oe), (name, s)


def test_symmetric_digraph_matches_the_undirected_graph():
    g = gen.rmat(12, 8, 5)
    srcs = pick_sources(g, 100, 4)
    Gu = sp.Graph(g.row_ptr, g.col_idx)
    Gd = sp.Graph(g.row_ptr, g.col_idx, flags=sp.SP_GRAPH_DIRECTED)
    assert Gd.info["directed"] == 1 and Gu.info["directed"] == 0
    want, _ = oracle.bc(g, srcs)
    for form, batch in [(sp.SP_FORM_PLAIN, 0), (sp.SP_FORM_BATCHED, 64), (sp.SP_FORM_SMALL, 0)]:
        a, sa = gpu_bc(Gu, srcs, sp.SP_FP64, form, batch)
        b, sb = gpu_bc(Gd, srcs, sp.SP_FP64, form, batch)
        close(b, want, 1e-9, f"symmetric digraph form {form}")
        close(b, a, 1e-12, f"directed vs undirected form {form}")
        assert sa["traversed_arcs"] == sb["traversed_arcs"]


def test_directed_edge_list_builder_and_async_call():
    g = gen.rmat_directed(11, 8, 12)
    rows = np.repeat(np.arange(g.n, dtype=np.int32), np.diff(g.row_ptr))
    # every arc twice, a self-loop and the arcs in reverse order: the builder
    # keeps each arc once and drops the loop
    src = np.concatenate([rows, rows[::-1], [3]]).astype(np.int32)
    dst = np.concatenate([g.col_idx, g.col_idx[::-1], [3]]).astype(np.int32)
    G = sp.Graph.from_edges(src, dst, g.n, flags=sp.SP_GRAPH_DIRECTED)
    rp, ci = G.csr()
    assert np.array_equal(rp, g.row_ptr) and np.array_equal(ci, g.col_idx)
    srcs = pick_sources(g, 64, 2)
    want, _ = oracle.bc(g, srcs, directed=True)
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    for form, batch in [(sp.SP_FORM_BATCHED, 64), (sp.SP_FORM_PLAIN, 0)]:
        sp.sp_bc_ex(G.handle, torch.as_tensor(srcs, device=DEV), out,
                    sp.make_opts(form=form, batch=batch, driver=sp.SP_DRIVER_PERSISTENT), want_stats=False)
        sp.sp_graph_sync(G.handle)
        close(out.cpu().numpy(), want, 1e-9, f"async directed form {form}")


def test_directed_flags_are_checked():
    g = gen.rmat_directed(8, 4, 1)
    with pytest.raises(sp.StarbcError) as e:
        sp.Graph(g.row_ptr, g.col_idx, flags=sp.SP_GRAPH_DIRECTED | sp.SP_GRAPH_CHECK_SYMMETRIC)
    assert e.value.status == sp.SP_ERR_INVALID_ARG
