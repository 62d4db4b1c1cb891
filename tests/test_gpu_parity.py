"""CUDA path against the CPU oracle, through the C ABI.

Levels must match bit for bit; path counts exactly while below 2^53; BC
within rtol 1e-9 (FP64 dependencies) or 1e-4 (FP32 dependencies) per vertex,
|gpu - oracle| <= rtol * max(|oracle|, 1), and exactly 0 where the oracle has
an exact 0.
"""
import math

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2401_02472_gb300 as sp

pytestmark = pytest.mark.gpu

RTOL = {sp.SP_FP64: 1e-9, sp.SP_FP32_DELTA: 1e-4}
DEV = "cuda:0"


def assert_bc_close(got, want, rtol, what=""):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    assert got.shape == want.shape
    assert np.all(np.isfinite(got)), what
    err = np.abs(got - want)
    bound = rtol * np.maximum(np.abs(want), 1.0)
    bad = np.nonzero(err > bound)[0]
    assert bad.size == 0, f"{what}: {bad.size} vertices off, first {bad[:5]} got {got[bad[:5]]} want {want[bad[:5]]}"
    assert np.all(got[want == 0.0] == 0.0), f"{what}: nonzero where the oracle has exact 0"


def device_graph(g, flags=0):
    return sp.Graph(g.row_ptr, g.col_idx, flags=flags)


def gpu_bc(G, sources, precision=sp.SP_FP64, form=sp.SP_FORM_AUTO, batch=0, device_out=True, **kw):
    src = torch.as_tensor(np.asarray(sources, np.int32), device=DEV)
    out = torch.empty(G.n, dtype=torch.float64, device=DEV) if device_out else np.empty(G.n, np.float64)
    st = sp.sp_bc_ex(G.handle, src, out, sp.make_opts(precision=precision, form=form, batch=batch, **kw))
    torch.cuda.synchronize()
    return (out.cpu().numpy() if device_out else out), st


# ---------------------------------------------------------------------------
GRAPHS = {
    "er2000": lambda: gen.er(2000, 10000, 1),
    "rmat12": lambda: gen.rmat(12, 16, 2),
    "knn5000": lambda: gen.knn2d(5000, 4, 3),
    "grid30x41": lambda: gen.grid(30, 41),
    "path300": lambda: gen.path(300),
    "mixed": lambda: gen.disjoint_union(gen.star(40), gen.cycle(9), gen.from_edges(5, []), gen.path(17),
                                        gen.complete(6)),
}
_cache = {}


def graph(name):
    if name not in _cache:
        g = GRAPHS[name]()
        _cache[name] = (g, device_graph(g))
    return _cache[name]


def hub_graph():
    """A graph with rows far above both hub thresholds (segments in both forms)."""
    if "hub" not in _cache:
        base = gen.rmat(13, 8, 5)
        n = base.n
        extra = [(0, v) for v in range(1, n, 1)] + [(1, v) for v in range(2, n, 2)]
        rp, ci = base.row_ptr, base.col_idx
        rows = np.repeat(np.arange(n), np.diff(rp))
        edges = np.concatenate([np.stack([rows, ci], 1), np.asarray(extra)], 0)
        g = gen.from_edges(n, edges, "hub")
        _cache["hub"] = (g, device_graph(g))
    return _cache["hub"]


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_bfs_levels_bit_exact(name):
    g, G = graph(name)
    srcs = np.unique(np.array([0, g.n // 3, g.n - 1, g.n // 2], np.int32))
    dist = torch.empty((len(srcs), g.n), dtype=torch.int32, device=DEV)
    sp.sp_bfs(G.handle, torch.as_tensor(srcs, device=DEV), dist)
    got = dist.cpu().numpy()
    for i, s in enumerate(srcs):
        assert np.array_equal(got[i], oracle.bfs(g, int(s))), (name, s)


def test_bfs_host_buffers_and_hubs():
    g, G = hub_graph()
    srcs = np.array([0, 1, 77, 4095], np.int32)
    dist = np.empty((4, g.n), np.int32)
    sp.sp_bfs(G.handle, srcs, dist)
    for i, s in enumerate(srcs):
        assert np.array_equal(dist[i], oracle.bfs(g, int(s)))


@pytest.mark.parametrize("name", ["er2000", "rmat12", "grid30x41", "mixed"])
def test_sigma_exact(name):
    g, G = graph(name)
    for s in [0, g.n - 1]:
        mant = np.empty(g.n, np.float64)
        e2 = np.empty(g.n, np.int64)
        sp.sp_sigma(G.handle, s, mant, e2)
        om, oe, od, _ = oracle.sigma(g, s)
        assert np.array_equal(mant, om) and np.array_equal(e2, oe), (name, s)


def test_sigma_beyond_double_range():
    # Path counts up to C(1198, 599) ~ 2^1193: the per-level rescaled FP64 path.
    g = gen.grid(600, 600)
    G = device_graph(g)
    mant = np.empty(g.n, np.float64)
    e2 = np.empty(g.n, np.int64)
    sp.sp_sigma(G.handle, 0, mant, e2)
    for (i, j) in [(599, 599), (0, 599), (300, 299), (599, 1), (450, 512), (10, 10)]:
        v = i * 600 + j
        want = math.comb(i + j, i)
        shift = max(want.bit_length() - 64, 0)
        log2_want = shift + math.log2(want >> shift)
        assert abs(math.log2(mant[v]) + int(e2[v]) - log2_want) <= 1e-12 * max(1.0, log2_want)
    om, oe, _, _ = oracle.sigma(g, 0)
    lg = np.log2(mant) + e2
    lo = np.log2(om) + oe
    assert np.max(np.abs(lg - lo) / np.maximum(lo, 1)) < 1e-12


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_bc_plain(name, precision):
    g, G = graph(name)
    srcs = gen.sources(g, min(12, int((g.degrees() > 0).sum())), 7)
    got, st = gpu_bc(G, srcs, precision, sp.SP_FORM_PLAIN)
    want, ost = oracle.bc(g, srcs)
    assert_bc_close(got, want, RTOL[precision], f"{name} plain")
    assert st["traversed_arcs"] == int(ost["arcs"].sum())
    assert st["max_levels"] == int(ost["levels"].max())


@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
@pytest.mark.parametrize("batch", [32, 64, 128, 256])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_bc_batched(name, batch, precision):
    g, G = graph(name)
    k = min(batch + 37, int((g.degrees() > 0).sum()))  # a ragged last batch
    srcs = gen.sources(g, k, 11)
    got, st = gpu_bc(G, srcs, precision, sp.SP_FORM_BATCHED, batch)
    want, ost = oracle.bc(g, srcs)
    assert_bc_close(got, want, RTOL[precision], f"{name} B={batch}")
    assert st["traversed_arcs"] == int(ost["arcs"].sum())
    assert st["reached"] == int(ost["reached"].sum())
    assert st["max_levels"] == int(ost["levels"].max())


def test_er2000_all_sources_both_forms():
    g, G = graph("er2000")
    srcs = np.arange(g.n, dtype=np.int32)
    want, _ = oracle.bc(g, srcs)
    for form, batch in [(sp.SP_FORM_PLAIN, 0), (sp.SP_FORM_BATCHED, 64), (sp.SP_FORM_SMALL, 0), (sp.SP_FORM_AUTO, 0)]:
        got, st = gpu_bc(G, srcs, sp.SP_FP64, form, batch)
        assert_bc_close(got, want, 1e-9, f"er2000 all sources form={form}")
        if form == sp.SP_FORM_AUTO:
            assert st["form"] == sp.SP_FORM_SMALL  # the benchmark configuration
    # the invariant: sum of BC = sum over reached ordered pairs of (d - 1)
    from tests import bruteforce as bf

    assert abs(got.sum() - bf.pair_distance_excess(g, srcs)) <= 1e-9 * got.sum()


@pytest.mark.parametrize("form", [sp.SP_FORM_PLAIN, sp.SP_FORM_BATCHED, sp.SP_FORM_SMALL])
@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
def test_hubs_split_into_segments(form, precision):
    g, G = hub_graph()
    srcs = np.array([0, 1, 2, 3, 4095, 17, 0, 1000] * 5, np.int32)
    got, _ = gpu_bc(G, srcs, precision, form, 32)
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(got, want, RTOL[precision], "hub graph")


# ---------------------------------------------------------------------------
def test_edge_cases():
    g, G = graph("mixed")
    z, _ = gpu_bc(G, [], sp.SP_FP64)
    assert np.array_equal(z, np.zeros(g.n))
    iso = [int(v) for v in np.nonzero(g.degrees() == 0)[0][:3]]
    z, _ = gpu_bc(G, iso * 20, sp.SP_FP64, sp.SP_FORM_BATCHED, 32)
    assert np.array_equal(z, np.zeros(g.n))
    dup = [0, 0, 0, 41, 41, 50] * 7
    for form in (sp.SP_FORM_PLAIN, sp.SP_FORM_BATCHED, sp.SP_FORM_SMALL):
        got, _ = gpu_bc(G, dup, sp.SP_FP64, form, 32)
        want, _ = oracle.bc(g, dup)
        assert_bc_close(got, want, 1e-9, "duplicates")
    one = gen.from_edges(1, [])
    G1 = device_graph(one)
    for form in (sp.SP_FORM_AUTO, sp.SP_FORM_PLAIN, sp.SP_FORM_SMALL):
        got, _ = gpu_bc(G1, [0, 0], sp.SP_FP64, form)
        assert np.array_equal(got, np.zeros(1))
    two = gen.path(2)
    G2 = device_graph(two)
    got, _ = gpu_bc(G2, [0, 1] * 20, sp.SP_FP64, sp.SP_FORM_BATCHED, 32)
    assert np.array_equal(got, np.zeros(2))


def test_host_output_buffer_matches_device():
    g, G = graph("rmat12")
    srcs = gen.sources(g, 50, 3)
    a, _ = gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_BATCHED, 64, device_out=True)
    b, _ = gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_BATCHED, 64, device_out=False)
    assert np.array_equal(a, b)
    hb = np.empty(g.n, np.float64)
    sp.sp_bc(G.handle, srcs, hb)  # host sources, host output
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(hb, want, 1e-9)


@pytest.mark.parametrize("form,batch", [(sp.SP_FORM_PLAIN, 0), (sp.SP_FORM_BATCHED, 64), (sp.SP_FORM_BATCHED, 128)])
def test_run_to_run_bit_identical(form, batch):
    g, G = hub_graph()
    srcs = gen.sources(g, 150, 9)
    a, _ = gpu_bc(G, srcs, sp.SP_FP32_DELTA, form, batch)
    for _ in range(3):
        b, _ = gpu_bc(G, srcs, sp.SP_FP32_DELTA, form, batch)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_bc_small(name, precision):
    # One block per source with the per-source state in shared memory.
    g, G = graph(name)
    srcs = gen.sources(g, min(40, int((g.degrees() > 0).sum())), 8)
    got, st = gpu_bc(G, srcs, precision, sp.SP_FORM_SMALL)
    want, ost = oracle.bc(g, srcs)
    assert_bc_close(got, want, RTOL[precision], f"{name} small")
    assert st["form"] == sp.SP_FORM_SMALL
    assert st["traversed_arcs"] == int(ost["arcs"].sum())
    assert st["max_levels"] == int(ost["levels"].max())
    again, _ = gpu_bc(G, srcs, precision, sp.SP_FORM_SMALL)
    assert np.array_equal(got, again)


def test_small_form_limits_and_fallback():
    # Path counts past 2^64 on an 80 x 80 grid (C(158, 79) ~ 2^154): the small
    # form stops and the call reruns in the plain form with FP64 counts.
    g = gen.grid(80, 80)
    G = device_graph(g)
    srcs = np.array([0, 79, 6399, 3240], np.int32)
    got, st = gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_SMALL)
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(got, want, 1e-9, "grid80 small -> plain")
    assert st["form"] == sp.SP_FORM_PLAIN and st["sigma_float"] == 1
    # too many vertices for one block's shared memory
    big = gen.rmat(15, 4, 3)
    with pytest.raises(sp.StarbcError) as e:
        gpu_bc(device_graph(big), [1, 2], sp.SP_FP64, sp.SP_FORM_SMALL)
    assert e.value.status == sp.SP_ERR_TOO_LARGE


@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
@pytest.mark.parametrize("name", sorted(GRAPHS))
def test_bc_plain_graph_driver(name, precision):
    # Level loop as a CUDA graph (conditional WHILE node, one kernel per
    # level): same per-source dependencies as the persistent kernel, added
    # into BC in source order, so it equals the running sum of single-source
    # persistent calls bit for bit.
    g, G = graph(name)
    srcs = gen.sources(g, min(12, int((g.degrees() > 0).sum())), 7)
    got, st = gpu_bc(G, srcs, precision, sp.SP_FORM_PLAIN, driver=sp.SP_DRIVER_GRAPH)
    want, ost = oracle.bc(g, srcs)
    assert_bc_close(got, want, RTOL[precision], f"{name} plain, graph driver")
    assert st["driver"] == sp.SP_DRIVER_GRAPH
    assert st["traversed_arcs"] == int(ost["arcs"].sum())
    assert st["max_levels"] == int(ost["levels"].max())
    assert st["launches"] >= len(srcs) + int(ost["levels"].sum())  # a kernel per phase
    acc = np.zeros(g.n)
    for s in srcs:
        one, st1 = gpu_bc(G, [s], precision, sp.SP_FORM_PLAIN, driver=sp.SP_DRIVER_PERSISTENT)
        assert st1["driver"] == sp.SP_DRIVER_PERSISTENT
        acc = acc + one
    assert np.array_equal(got, acc)


def test_graph_driver_rescaled_counts_and_hubs():
    # Path counts past 2^64 (a 600 x 600 grid from its corners: FP64 with
    # per-level exponents over about 1,200 levels) and rows split into
    # segments, both under the graph-driven loop.
    g = gen.grid(600, 600)
    G = device_graph(g)
    srcs = np.array([0, 599, 600 * 600 - 1], np.int32)
    got, st = gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_PLAIN, driver=sp.SP_DRIVER_GRAPH)
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(got, want, 1e-9, "grid600 graph driver")
    assert st["sigma_float"] == 1 and st["max_levels"] == 1199
    gh, GH = hub_graph()
    hs = np.array([0, 1, 77, 4095], np.int32)
    for prec in (sp.SP_FP64, sp.SP_FP32_DELTA):
        got, _ = gpu_bc(GH, hs, prec, sp.SP_FORM_PLAIN, driver=sp.SP_DRIVER_GRAPH)
        want, _ = oracle.bc(gh, hs)
        assert_bc_close(got, want, RTOL[prec], "hub graph, graph driver")


def test_driver_autotuner_picks_and_caches():
    g, G = graph("rmat12")
    srcs = gen.sources(g, 40, 33)
    a, st = gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_PLAIN)
    assert st["driver"] in (sp.SP_DRIVER_PERSISTENT, sp.SP_DRIVER_GRAPH)
    b, st2 = gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_PLAIN)
    assert st2["tuned"] == 0 and st2["driver"] == st["driver"]
    assert np.array_equal(a, b)
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(a, want, 1e-9)


@pytest.mark.parametrize("name", ["rmat12", "er2000", "knn5000", "mixed"])
def test_plain_direction_does_not_change_results(name):
    # Bottom-up discovery on wide levels (any level above n/2, n/20, or never)
    # finds the same levels, so the per-vertex sums and BC are bit-identical.
    g, G = graph(name)
    srcs = gen.sources(g, min(20, int((g.degrees() > 0).sum())), 31)
    runs = [gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_PLAIN, bottom_up=bu)[0] for bu in (-1, 2, 20, 1000)]
    for r in runs[1:]:
        assert np.array_equal(r, runs[0])
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(runs[0], want, 1e-9)


@pytest.mark.parametrize("name", ["er2000", "rmat12", "path300", "mixed"])
def test_dag_counts_and_no_false_overflow(name):
    # Every form counts the shortest-path DAG arcs (v, u), d(u) = d(v) + 1,
    # exactly, and none reports a path-count overflow on graphs whose counts
    # are small (a fresh graph object: no remembered range flags).
    g = GRAPHS[name]()
    G = device_graph(g)
    srcs = gen.sources(g, min(12, int((g.degrees() > 0).sum())), 7)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    want_dag = 0
    for s in srcs:
        dist = oracle.bfs(g, int(s))
        du, dv = dist[rows], dist[g.col_idx]
        want_dag += int(np.sum((du >= 0) & (dv == du + 1)))
    for form in (sp.SP_FORM_PLAIN, sp.SP_FORM_BATCHED, sp.SP_FORM_SMALL):
        _, st = gpu_bc(G, srcs, sp.SP_FP64, form, driver=sp.SP_DRIVER_PERSISTENT)
        assert st["sigma_float"] == 0, (name, form)
        assert st["dag_arcs"] == want_dag, (name, form, st["dag_arcs"], want_dag)
    G.close()


@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
@pytest.mark.parametrize("name", ["rmat12", "knn5000", "grid30x41", "mixed", "hub"])
def test_plain_records_match_arrays(name, precision):
    # The plain form's per-(group, vertex) state as one 32-byte record or as
    # separate arrays: the same arithmetic in the same order, so bit-identical
    # results, with one group and with several.
    g, G = hub_graph() if name == "hub" else graph(name)
    srcs = gen.sources(g, min(24, int((g.degrees() > 0).sum())), 41)
    for blocks in (0, 1):  # max_ctas = 1: a single group
        kw = dict(driver=sp.SP_DRIVER_PERSISTENT, max_ctas=blocks)
        rec, st_r = gpu_bc(G, srcs, precision, sp.SP_FORM_PLAIN, debug_flags=sp.SP_DEBUG_PLAIN_RECORDS, **kw)
        arr, st_a = gpu_bc(G, srcs, precision, sp.SP_FORM_PLAIN, debug_flags=sp.SP_DEBUG_PLAIN_ARRAYS, **kw)
        assert np.array_equal(rec, arr), name
        assert st_r["traversed_arcs"] == st_a["traversed_arcs"]
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(rec, want, RTOL[precision], f"{name} records")


def test_plain_records_rescaled_counts():
    # Records with FP64 path counts and per-level exponents (a 600 x 600 grid
    # from three corners: counts past 2^64), one block group per source.
    g = gen.grid(600, 600)
    G = device_graph(g)
    srcs = np.array([0, 599, 600 * 600 - 1], np.int32)
    got, st = gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_PLAIN, driver=sp.SP_DRIVER_PERSISTENT,
                     debug_flags=sp.SP_DEBUG_PLAIN_RECORDS)
    assert st["sigma_float"] == 1
    arr, _ = gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_PLAIN, driver=sp.SP_DRIVER_PERSISTENT,
                    debug_flags=sp.SP_DEBUG_PLAIN_ARRAYS)
    assert np.array_equal(got, arr)
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(got, want, 1e-9, "grid600 records")


@pytest.mark.parametrize("name", ["rmat12", "er2000", "knn5000", "mixed"])
def test_batched_direction_does_not_change_results(name):
    # Bottom-up discovery on the per-source bitmaps (levels above n/2, n/20,
    # or never) finds the same levels, so BC is bit-identical.
    g, G = graph(name)
    srcs = gen.sources(g, min(100, int((g.degrees() > 0).sum())), 32)
    runs = [gpu_bc(G, srcs, sp.SP_FP64, sp.SP_FORM_BATCHED, 64, bottom_up=bu)[0] for bu in (-1, 2, 20)]
    for r in runs[1:]:
        assert np.array_equal(r, runs[0])
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(runs[0], want, 1e-9)
    gh, GH = hub_graph()
    hs = np.array([0, 1, 2, 3, 4095, 17, 1000] * 5, np.int32)
    a, _ = gpu_bc(GH, hs, sp.SP_FP32_DELTA, sp.SP_FORM_BATCHED, 128, bottom_up=-1)
    b, _ = gpu_bc(GH, hs, sp.SP_FP32_DELTA, sp.SP_FORM_BATCHED, 128, bottom_up=3)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
def test_source_order_only_changes_rounding(precision):
    # The batched form regroups sources by distance from a maximum-degree
    # vertex; with SP_BC_KEEP_ORDER it keeps the caller's order.  Both are BC
    # over the same multiset, so they agree within the tolerance, and the
    # regrouped run is the same for any permutation of the caller's list.
    g, G = graph("rmat12")
    srcs = gen.sources(g, 150, 21)
    a, _ = gpu_bc(G, srcs, precision, sp.SP_FORM_BATCHED, 64)
    b, _ = gpu_bc(G, srcs, precision, sp.SP_FORM_BATCHED, 64, flags=sp.SP_BC_KEEP_ORDER)
    assert_bc_close(a, b, RTOL[precision])
    c, _ = gpu_bc(G, srcs[::-1].copy(), precision, sp.SP_FORM_BATCHED, 64)
    want, _ = oracle.bc(g, srcs)
    assert_bc_close(c, want, RTOL[precision])


def test_linearity_over_calls():
    g, G = graph("knn5000")
    s1, s2 = gen.sources(g, 40, 1), gen.sources(g, 70, 2)
    a, _ = gpu_bc(G, s1, sp.SP_FP64, sp.SP_FORM_BATCHED, 32)
    b, _ = gpu_bc(G, s2, sp.SP_FP64, sp.SP_FORM_BATCHED, 32)
    c, _ = gpu_bc(G, np.concatenate([s1, s2]), sp.SP_FP64, sp.SP_FORM_BATCHED, 32)
    assert_bc_close(c, a + b, 1e-12)


def test_bad_graphs_are_rejected():
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_graph_create(np.array([0, 2, 1, 3], np.int32), np.array([1, 2, 0], np.int32))
    assert e.value.status == sp.SP_ERR_BAD_GRAPH
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_graph_create(np.array([0, 1, 2], np.int32), np.array([1, 5], np.int32))
    assert e.value.status == sp.SP_ERR_BAD_GRAPH
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_graph_create(np.array([0, 1, 1], np.int32), np.array([1], np.int32), flags=sp.SP_GRAPH_CHECK_SYMMETRIC)
    assert e.value.status == sp.SP_ERR_BAD_GRAPH
    g = gen.rmat(10, 8, 1)
    G = device_graph(g, sp.SP_GRAPH_CHECK_SYMMETRIC)
    assert G.info["symmetric"] == 1 and G.info["sorted_rows"] == 1
    assert G.info["max_degree"] == int(g.degrees().max())
    assert G.info["isolated"] == int((g.degrees() == 0).sum())
    _, G = graph("er2000")
    with pytest.raises(sp.StarbcError) as e:
        gpu_bc(G, [0, 2000])
    assert e.value.status == sp.SP_ERR_INVALID_ARG


@pytest.mark.parametrize("form", [sp.SP_FORM_PLAIN, sp.SP_FORM_BATCHED])
def test_barrier_timeout_returns_status(form):
    # One block skips a barrier on purpose; the others give up after 50 ms and
    # the launch ends with SP_ERR_TIMEOUT instead of hanging.
    g, G = graph("er2000")
    with pytest.raises(sp.StarbcError) as e:
        gpu_bc(G, list(range(40)), sp.SP_FP64, form, 32, barrier_timeout_ns=50_000_000,
               debug_flags=sp.SP_DEBUG_SKIP_BARRIER)
    assert e.value.status == sp.SP_ERR_TIMEOUT
    got, _ = gpu_bc(G, list(range(40)), sp.SP_FP64, form, 32)  # the context is still usable
    want, _ = oracle.bc(g, list(range(40)))
    assert_bc_close(got, want, 1e-9)


# ---------------------------------------------------------------------------
# Range handling of path counts (X6 / X9 of the readings)

def diamond_chain(k):
    """k diamonds in a row: a_i - b_i, a_i - c_i, b_i - a_(i+1), c_i - a_(i+1).
    From a_0 the path counts double at every a_i (sigma(a_k) = 2^k) while each
    level holds equal counts, so FP64 counts are needed past 2^64 but a level
    never spreads."""
    edges = []
    for i in range(k):
        a, b, c, a2 = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        edges += [(a, b), (a, c), (b, a2), (c, a2)]
    return gen.from_edges(3 * k + 1, edges, f"diamonds{k}")


@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
@pytest.mark.parametrize("batch", [32, 128])
def test_batched_recentres_rescaled_counts(batch, precision):
    # Path counts up to C(1198, 599) ~ 2^1193 on a 600 x 600 grid from three
    # corners: the batched form reruns with FP64 counts and recentres levels
    # whose exponents leave the bound.  FP32 dependencies cannot hold theta
    # here (a level spans ~2^595), so that call is promoted to FP64.
    g = gen.grid(600, 600)
    G = device_graph(g)
    srcs = np.array([0, 599, 600 * 600 - 1], np.int32)
    got, st = gpu_bc(G, srcs, precision, sp.SP_FORM_BATCHED, batch)
    want, ost = oracle.bc(g, srcs)
    assert ost["used_xfloat"].all()
    assert_bc_close(got, want, RTOL[precision], f"grid600 batched B={batch}")
    assert st["form"] == sp.SP_FORM_BATCHED and st["sigma_float"] == 1
    assert st["recentred"] > 0
    assert st["max_levels"] == 1199
    if precision == sp.SP_FP32_DELTA:
        assert st["promoted"] == 1
    G.close()


def test_plain_fp32_promotion_on_wide_levels():
    # The plain form's FP32 dependencies leave FP32 on the 600 x 600 grid too:
    # the call reruns with FP64 theta and still matches the oracle.
    g = gen.grid(600, 600)
    G = device_graph(g)
    srcs = np.array([0, 600 * 600 - 1], np.int32)
    for driver in (sp.SP_DRIVER_PERSISTENT, sp.SP_DRIVER_GRAPH):
        got, st = gpu_bc(G, srcs, sp.SP_FP32_DELTA, sp.SP_FORM_PLAIN, driver=driver)
        want, _ = oracle.bc(g, srcs)
        assert_bc_close(got, want, 1e-4, f"grid600 plain FP32 driver {driver}")
        assert st["promoted"] == 1 and st["sigma_float"] == 1 and st["recentred"] > 0
    G.close()


@pytest.mark.parametrize("form,kw", [
    (sp.SP_FORM_PLAIN, dict(driver=sp.SP_DRIVER_PERSISTENT, debug_flags=sp.SP_DEBUG_PLAIN_ARRAYS)),
    (sp.SP_FORM_PLAIN, dict(driver=sp.SP_DRIVER_PERSISTENT, debug_flags=sp.SP_DEBUG_PLAIN_RECORDS)),
    (sp.SP_FORM_PLAIN, dict(driver=sp.SP_DRIVER_GRAPH)),
    (sp.SP_FORM_BATCHED, dict(batch=32)),
    (sp.SP_FORM_BATCHED, dict(batch=128)),
    (sp.SP_FORM_SMALL, dict()),
])
def test_fp32_dependencies_stay_fp32_past_2_64(form, kw):
    # Counts reach 2^300 but every level holds equal counts: FP64 counts
    # recentred at +-2^64 keep theta-hat = (1 + delta) / sigma-hat inside FP32,
    # so no form reruns with FP64 dependencies (promoted == 0).  With FP64
    # dependencies the bound is 2^512, which these counts never reach: no
    # level is recentred.  The small form holds exact counts only and hands
    # the call to the plain form.
    g = diamond_chain(300)
    G = device_graph(g)
    srcs = np.array([0, 1, 450, 900], np.int32)
    want, ost = oracle.bc(g, srcs)
    assert not ost["used_xfloat"].any()
    for prec in (sp.SP_FP32_DELTA, sp.SP_FP64):
        got, st = gpu_bc(G, srcs, prec, form, **kw)
        assert_bc_close(got, want, RTOL[prec], f"diamond chain form {form} {kw} precision {prec}")
        assert st["sigma_float"] == 1, st
        assert (st["recentred"] > 0) if prec == sp.SP_FP32_DELTA else (st["recentred"] == 0), st
        assert st["promoted"] == 0, st
        assert st["max_levels"] == int(ost["levels"].max())
    G.close()


@pytest.mark.parametrize("form,batch", [(sp.SP_FORM_PLAIN, 0), (sp.SP_FORM_BATCHED, 32)])
def test_spread_limit_gives_range_error_or_exact_values(form, batch):
    # On a 2,100 x 2,100 grid from a corner the anti-diagonal level holds path
    # counts from 1 to C(2099, 1049) ~ 2^2095: wider than the FP64 exponent
    # range even after centring.  The call must either return values that
    # match the oracle (extended exponents) or SP_ERR_RANGE; never NaN.
    g = gen.grid(2100, 2100)
    G = device_graph(g)
    try:
        got, _ = gpu_bc(G, [0], sp.SP_FP64, form, batch)
    except sp.StarbcError as e:
        assert e.status == sp.SP_ERR_RANGE, e
        got = None
    if got is not None:
        assert np.all(np.isfinite(got))
        want, _ = oracle.bc(g, [0])
        assert_bc_close(got, want, 1e-9, "grid2100")
    G.close()
    # the context is still usable
    g2, G2 = graph("er2000")
    got, _ = gpu_bc(G2, [1, 2, 3], sp.SP_FP64, form, batch)
    want, _ = oracle.bc(g2, [1, 2, 3])
    assert_bc_close(got, want, 1e-9)
