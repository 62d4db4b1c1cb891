"""Serving: continuous batching of BC requests over resident graphs.

Each request's result must equal the oracle within the tolerance and be
bit-identical whether it ran alone or mixed with other requests.
"""
import time

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2401_02472_gb300 as sp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
RTOL = {sp.SP_FP64: 1e-9, sp.SP_FP32_DELTA: 1e-4}


def close(got, want, rtol):
    return bool(np.all(np.abs(got - want) <= rtol * np.maximum(np.abs(want), 1.0)) and
                np.all(got[want == 0.0] == 0.0))


@pytest.fixture(scope="module")
def graphs():
    gs = [gen.rmat(12, 16, 2), gen.knn2d(4000, 4, 3), gen.er(3000, 24000, 5)]
    return gs, [sp.Graph(g.row_ptr, g.col_idx) for g in gs]


def requests(gs, count, seed):
    """(graph index, sources, precision) per request; nsrc log-uniform in [1, 300]."""
    sizes = gen.log_uniform_int(1, 300, seed, count)
    which = gen.draws(gen.substream(seed, 3), 0, count) % np.uint64(len(gs))
    out = []
    for i in range(count):
        gi = int(which[i])
        k = int(min(sizes[i], (gs[gi].degrees() > 0).sum()))
        srcs = gen.sources(gs[gi], k, 1000 + seed * 100 + i)
        out.append((gi, srcs, sp.SP_FP32_DELTA if i % 2 else sp.SP_FP64))
    return out


def serve(Gs, reqs, slots=4, budget=8 << 30, live=True):
    s = sp.sp_server_create(budget, slots)
    sp.sp_server_set_live(s, live)
    ids = [sp.sp_server_add_graph(s, G.handle) for G in Gs]
    outs, handles = [], []
    for gi, srcs, prec in reqs:
        out = torch.full((Gs[gi].n,), -1.0, dtype=torch.float64, device=DEV)
        h = sp.sp_bc_submit(s, ids[gi], srcs, out, sp.make_opts(precision=prec))
        outs.append(out)
        handles.append(h)
    for h in handles:
        assert sp.sp_bc_wait(s, h) == sp.SP_OK
    times = [sp.sp_request_times(s, h) for h in handles]
    stats = [sp.sp_request_stats(s, h) for h in handles]
    sp.sp_server_destroy(s)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs], times, stats


def test_mixed_requests_match_oracle_and_run_alone(graphs):
    gs, Gs = graphs
    reqs = requests(gs, 14, 7)
    mixed, times, stats = serve(Gs, reqs)
    for (gi, srcs, prec), got, (t0, t1, t2), st in zip(reqs, mixed, times, stats):
        want, ost = oracle.bc(gs[gi], srcs)
        assert close(got, want, RTOL[prec]), (gi, len(srcs), prec)
        assert 0 < t0 <= t1 <= t2
        assert st["traversed_arcs"] == int(ost["arcs"].sum())
    # every third request again, alone on a fresh server: bit-identical
    for i in range(0, len(reqs), 3):
        alone, _, _ = serve(Gs, [reqs[i]])
        assert np.array_equal(alone[0], mixed[i]), i


def test_launches_without_live_feeds_give_the_same_results(graphs):
    # With live launches off, each batched launch runs only the requests it
    # started with; results are bit-identical to those of live launches.
    gs, Gs = graphs
    reqs = requests(gs, 8, 13)
    live, _, _ = serve(Gs, reqs, slots=1)
    fixed, _, stats = serve(Gs, reqs, slots=1, live=False)
    for i, (a, b) in enumerate(zip(live, fixed)):
        assert np.array_equal(a, b), i
    assert all(st["joined"] == 0 for st in stats)


def test_requests_join_a_running_launch():
    # A long request on one graph runs as a live launch; requests on the same
    # graph submitted while it runs enter it between its batches (their words
    # run after the words already there).  Each matches the oracle and is
    # bit-identical to the request served alone; traversal counts are the
    # request's own.
    g = gen.rmat(17, 16, 7)
    G = sp.Graph(g.row_ptr, g.col_idx)
    opts = sp.make_opts(precision=sp.SP_FP64)
    big_srcs = gen.sources(g, 1024, 11)
    small = [gen.sources(g, k, 20 + i) for i, k in enumerate([40, 7, 64])]
    joined_any = False
    for attempt in range(3):
        s = sp.sp_server_create(8 << 30, 1)
        gid = sp.sp_server_add_graph(s, G.handle)
        big_out = torch.full((g.n,), -1.0, dtype=torch.float64, device=DEV)
        hb = sp.sp_bc_submit(s, gid, big_srcs, big_out, opts)
        t_end = time.monotonic() + 30.0
        while sp.sp_request_times(s, hb)[1] == 0:  # taken by the slot
            assert time.monotonic() < t_end
        outs, hs = [], []
        for srcs in small:
            out = torch.full((g.n,), -1.0, dtype=torch.float64, device=DEV)
            hs.append(sp.sp_bc_submit(s, gid, srcs, out, opts))
            outs.append(out)
        for h in hs + [hb]:
            assert sp.sp_bc_wait(s, h) == sp.SP_OK
        stats = [sp.sp_request_stats(s, h) for h in hs]
        times = [sp.sp_request_times(s, h) for h in hs + [hb]]
        sp.sp_server_destroy(s)
        torch.cuda.synchronize()
        joined = [st["joined"] == 1 for st in stats]
        if any(joined):
            joined_any = True
            for i in range(len(hs)):
                if joined[i]:  # entered the launch before its first request was done, finished after it
                    assert times[i][1] < times[-1][2] <= times[i][2]
                    assert stats[i]["shared"] > 1
            break
    assert joined_any, "no request joined the running launch in three attempts"
    for srcs, out, st in zip(small, outs, stats):
        got = out.cpu().numpy()
        want, ost = oracle.bc(g, srcs)
        assert close(got, want, RTOL[sp.SP_FP64]), len(srcs)
        assert st["traversed_arcs"] == int(ost["arcs"].sum())
        alone, _, _ = serve([G], [(0, srcs, sp.SP_FP64)], slots=1)
        assert np.array_equal(alone[0], got), len(srcs)
    alone, _, _ = serve([G], [(0, big_srcs, sp.SP_FP64)], slots=1)
    assert np.array_equal(alone[0], big_out.cpu().numpy())


def test_budget_smaller_than_a_request_still_runs(graphs):
    gs, Gs = graphs
    reqs = requests(gs, 5, 11)
    got, _, _ = serve(Gs, reqs, slots=2, budget=1)  # one request at a time
    for (gi, srcs, prec), g in zip(reqs, got):
        want, _ = oracle.bc(gs[gi], srcs)
        assert close(g, want, RTOL[prec])


def test_poll_cancel_and_empty_requests(graphs):
    gs, Gs = graphs
    s = sp.sp_server_create(8 << 30, 1)
    gid = sp.sp_server_add_graph(s, Gs[0].handle)
    big = [sp.sp_bc_submit(s, gid, gen.sources(gs[0], 300, 50 + i),
                           torch.empty(gs[0].n, dtype=torch.float64, device=DEV)) for i in range(3)]
    out = torch.empty(gs[0].n, dtype=torch.float64, device=DEV)
    late = sp.sp_bc_submit(s, gid, gen.sources(gs[0], 200, 99), out)
    rc = sp.sp_bc_cancel(s, late)
    assert rc in (sp.SP_OK, sp.SP_ERR_CANCELLED)
    final = sp.lib.sp_bc_wait(s, late, -1)
    assert final in (sp.SP_ERR_CANCELLED, sp.SP_OK)
    empty_out = torch.full((gs[0].n,), 7.0, dtype=torch.float64, device=DEV)
    e = sp.sp_bc_submit(s, gid, np.zeros(0, np.int32), empty_out)
    assert sp.sp_bc_poll(s, e) == sp.SP_OK
    for h in big:
        assert sp.sp_bc_wait(s, h) == sp.SP_OK
    sp.sp_server_destroy(s)
    assert torch.count_nonzero(empty_out).item() == 0
    with pytest.raises(sp.StarbcError):
        s2 = sp.sp_server_create(1 << 30, 2)
        try:
            sp.sp_bc_submit(s2, 5, np.array([0], np.int32), empty_out)
        finally:
            sp.sp_server_destroy(s2)


def test_requests_on_one_graph_share_launches():
    # Graphs too large for the shared-memory form run in the batched form;
    # requests queued behind a long one on the same graph join one launch,
    # each in source words of its own.  Every result matches the oracle and
    # is bit-identical to the request served alone; traversal counts are the
    # request's own.
    g1, g2 = gen.rmat(15, 8, 6), gen.er(20000, 80000, 9)
    G1, G2 = sp.Graph(g1.row_ptr, g1.col_idx), sp.Graph(g2.row_ptr, g2.col_idx)
    gs, Gs = [g1, g2], [G1, G2]
    sizes = [300, 5, 80, 33, 2, 64, 17, 40]
    reqs = []
    for i, k in enumerate(sizes):
        gi = 0 if i % 3 != 2 else 1
        prec = sp.SP_FP32_DELTA if i % 4 else sp.SP_FP64
        reqs.append((gi, gen.sources(gs[gi], k, 500 + i), prec))
    s = sp.sp_server_create(8 << 30, 1)
    ids = [sp.sp_server_add_graph(s, G.handle) for G in Gs]
    outs, handles = [], []
    for gi, srcs, prec in reqs:
        out = torch.full((Gs[gi].n,), -1.0, dtype=torch.float64, device=DEV)
        handles.append(sp.sp_bc_submit(s, ids[gi], srcs, out, sp.make_opts(precision=prec)))
        outs.append(out)
    for h in handles:
        assert sp.sp_bc_wait(s, h) == sp.SP_OK
    stats = [sp.sp_request_stats(s, h) for h in handles]
    sp.sp_server_destroy(s)
    torch.cuda.synchronize()
    assert max(st["shared"] for st in stats) > 1  # at least one launch was shared
    for (gi, srcs, prec), out, st in zip(reqs, outs, stats):
        got = out.cpu().numpy()
        want, ost = oracle.bc(gs[gi], srcs)
        assert close(got, want, RTOL[prec]), (gi, len(srcs), prec)
        assert st["traversed_arcs"] == int(ost["arcs"].sum())
        assert st["form"] == sp.SP_FORM_BATCHED
        alone, _, _ = serve(Gs, [(gi, srcs, prec)], slots=1)
        assert np.array_equal(alone[0], got), (gi, len(srcs))


def test_pagerank_requests_share_the_server_with_bc(graphs):
    # PageRank requests (the paper's second workload on resident graphs) run
    # through the same queue and slots as BC requests: each result equals the
    # oracle's and, bit for bit, a direct sp_pagerank call on the same graph.
    gs, Gs = graphs
    s = sp.sp_server_create(8 << 30, 2)
    ids = [sp.sp_server_add_graph(s, G.handle) for G in Gs]
    jobs = []
    for i, gi in enumerate([0, 1, 2, 0]):
        srcs = gen.sources(gs[gi], 40, 300 + i)
        bc = torch.full((Gs[gi].n,), -1.0, dtype=torch.float64, device=DEV)
        hb = sp.sp_bc_submit(s, ids[gi], srcs, bc, sp.make_opts(precision=sp.SP_FP64))
        pr = torch.full((Gs[gi].n,), -1.0, dtype=torch.float64, device=DEV)
        iters = 5 + 3 * i
        hp = sp.sp_pagerank_submit(s, ids[gi], pr, 0.85, -1.0, iters)
        jobs.append((gi, srcs, bc, hb, pr, hp, iters))
    for gi, srcs, bc, hb, pr, hp, iters in jobs:
        assert sp.sp_bc_wait(s, hb) == sp.SP_OK
        assert sp.sp_bc_wait(s, hp) == sp.SP_OK
        rc, it, ch = sp.sp_request_pagerank(s, hp)
        assert rc == sp.SP_OK and it == iters
        st = sp.sp_request_stats(s, hp)
        assert st["traversed_arcs"] == gs[gi].nnz * iters and st["kernel_ms"] > 0
        want, wit, wch = oracle.pagerank(gs[gi], 0.85, -1.0, iters)
        got = pr.cpu().numpy()
        assert np.all(np.abs(got - want) <= 1e-10 * np.abs(want))
        direct = torch.empty(Gs[gi].n, dtype=torch.float64, device=DEV)
        dit, dch = sp.sp_pagerank(Gs[gi].handle, direct, 0.85, -1.0, iters)
        assert np.array_equal(direct.cpu().numpy(), got) and dit == it and dch == ch
        assert close(bc.cpu().numpy(), oracle.bc(gs[gi], srcs)[0], RTOL[sp.SP_FP64])
    # a BC handle is not a PageRank request; bad arguments are refused at submission
    with pytest.raises(sp.StarbcError):
        sp.sp_request_pagerank(s, jobs[0][3])
    bad = torch.empty(Gs[0].n, dtype=torch.float64, device=DEV)
    with pytest.raises(sp.StarbcError):
        sp.sp_pagerank_submit(s, ids[0], bad, 1.5, -1.0, 3)
    with pytest.raises(sp.StarbcError):
        sp.sp_pagerank_submit(s, ids[0], np.empty(Gs[0].n), 0.85, -1.0, 3)
    sp.sp_server_destroy(s)


def test_requests_on_a_weighted_graph_run_the_weighted_form():
    # A graph with weights is served in the weighted form, request by
    # request, never in (unweighted) batched launches.
    g = gen.rmat(15, 8, 3)
    w = gen.edge_weights(g, 5, 1, 20)
    G = sp.Graph(g.row_ptr, g.col_idx)
    sp.sp_graph_set_weights(G.handle, w)
    s = sp.sp_server_create(8 << 30, 1)
    gid = sp.sp_server_add_graph(s, G.handle)
    jobs = []
    for i, k in enumerate([30, 2]):
        srcs = gen.sources(g, k, 70 + i)
        out = torch.full((g.n,), -1.0, dtype=torch.float64, device=DEV)
        jobs.append((srcs, out, sp.sp_bc_submit(s, gid, srcs, out)))
    for srcs, out, h in jobs:
        assert sp.sp_bc_wait(s, h) == sp.SP_OK
        assert sp.sp_request_stats(s, h)["form"] == sp.SP_FORM_WEIGHTED
        want, _ = oracle.bc_weighted(g, w, srcs)
        assert close(out.cpu().numpy(), want, RTOL[sp.SP_FP64]), len(srcs)
    sp.sp_server_destroy(s)


def test_live_launch_that_overflows_its_counts_reruns_its_requests():
    # Path counts on a 200 x 200 grid pass 2^32, so a live batched launch in
    # exact u32 counts stops on the overflow; its unfinished requests rerun as
    # one ordinary launch with FP64 counts, and later requests on the graph
    # start in FP64.  Every result matches the oracle.
    g = gen.grid(200, 200)
    G = sp.Graph(g.row_ptr, g.col_idx)
    opts = sp.make_opts(precision=sp.SP_FP64, form=sp.SP_FORM_BATCHED)
    s = sp.sp_server_create(8 << 30, 1)
    gid = sp.sp_server_add_graph(s, G.handle)
    jobs = []
    for srcs in [np.array([0, 199, 200 * 200 - 1], np.int32), np.array([100 * 200 + 100, 5], np.int32)]:
        out = torch.full((g.n,), -1.0, dtype=torch.float64, device=DEV)
        jobs.append((srcs, out, sp.sp_bc_submit(s, gid, srcs, out, opts)))
    for srcs, out, h in jobs:
        assert sp.sp_bc_wait(s, h) == sp.SP_OK
        st = sp.sp_request_stats(s, h)
        assert st["sigma_float"] == 1 and st["form"] == sp.SP_FORM_BATCHED
        want, _ = oracle.bc(g, srcs)
        assert close(out.cpu().numpy(), want, RTOL[sp.SP_FP64]), srcs
    sp.sp_server_destroy(s)
