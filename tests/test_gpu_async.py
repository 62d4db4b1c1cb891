"""Asynchronous calls: sp_bc with a device output enqueues on the stream.

The boundary enqueues BC on the caller's stream and returns; device-side
errors are latched in the graph's error word and returned by the next call on
the graph (or sp_graph_sync); conditions that a wider representation fixes
are handled on the GPU by a fallback launch that runs only when needed.
Every result is compared with the CPU oracle.
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


def close(got, want, rtol, what=""):
    err = np.abs(got - want)
    bad = np.nonzero(err > rtol * np.maximum(np.abs(want), 1.0))[0]
    assert bad.size == 0, f"{what}: {bad.size} vertices off, e.g. {bad[:3]} {got[bad[:3]]} vs {want[bad[:3]]}"
    assert np.all(got[want == 0.0] == 0.0), what


def dev(a, dtype=torch.int32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device=DEV)


def warm(G, srcs, **kw):
    """A blocking call, then an asynchronous one: one-time set-up and tuning
    of the graph shape, and the first launch of every kernel the asynchronous
    path uses (modules load on first use)."""
    out = torch.empty(G.n, dtype=torch.float64, device=DEV)
    sp.sp_bc_ex(G.handle, dev(srcs), out, sp.make_opts(**kw))
    sp.sp_bc_ex(G.handle, dev(srcs), out, sp.make_opts(**kw), want_stats=False)
    sp.sp_graph_sync(G.handle)
    (out * 2.0).sum().item()  # the torch kernels the test launches between calls load here too
    torch.cuda.synchronize()


@pytest.mark.parametrize("form,batch", [(sp.SP_FORM_BATCHED, 64), (sp.SP_FORM_PLAIN, 0), (sp.SP_FORM_SMALL, 0)])
def test_two_calls_and_a_torch_kernel_queue_on_one_stream(form, batch):
    g = gen.rmat(12, 16, 2) if form != sp.SP_FORM_SMALL else gen.er(2000, 10000, 1)
    G = sp.Graph(g.row_ptr, g.col_idx)
    s1, s2 = gen.sources(g, 70, 3), gen.sources(g, 45, 4)
    opts = dict(form=form, batch=batch, driver=sp.SP_DRIVER_PERSISTENT)
    warm(G, s1, **opts)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        d1, d2 = dev(s1), dev(s2)
        out1 = torch.empty(g.n, dtype=torch.float64, device=DEV)
        out2 = torch.empty(g.n, dtype=torch.float64, device=DEV)
        torch.cuda._sleep(200_000_000)  # ~0.1 s of GPU time queued ahead of the calls
        t0 = time.perf_counter()
        sp.sp_bc_ex(G.handle, d1, out1, sp.make_opts(**opts), want_stats=False)
        scaled = out1 * 2.0  # a torch kernel between the two calls, reading the first result
        sp.sp_bc_ex(G.handle, d2, out2, sp.make_opts(**opts), want_stats=False)
        host_s = time.perf_counter() - t0
        queued = not stream.query()
    stream.synchronize()
    assert queued, "the calls waited for the GPU"
    assert host_s < 0.05, host_s
    sp.sp_graph_sync(G.handle)
    w1, _ = oracle.bc(g, s1)
    w2, _ = oracle.bc(g, s2)
    close(out1.cpu().numpy(), w1, 1e-9, "first call")
    close(scaled.cpu().numpy(), 2.0 * w1, 1e-9, "torch kernel on the first result")
    close(out2.cpu().numpy(), w2, 1e-9, "second call")
    G.close()


@pytest.mark.parametrize("form", [sp.SP_FORM_PLAIN, sp.SP_FORM_BATCHED])
def test_timeout_is_latched_and_returned_by_the_next_call(form):
    # One block skips a barrier on purpose; the others give up after 50 ms.
    # The asynchronous call returns SP_OK at once; the next call on the graph
    # returns SP_ERR_TIMEOUT and does nothing else; the one after works.
    g = gen.er(2000, 10000, 1)
    G = sp.Graph(g.row_ptr, g.col_idx)
    srcs = list(range(40))
    opts = dict(form=form, batch=32, driver=sp.SP_DRIVER_PERSISTENT)
    warm(G, srcs, **opts)
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    sp.sp_bc_ex(G.handle, dev(srcs), out,
                sp.make_opts(barrier_timeout_ns=50_000_000, debug_flags=sp.SP_DEBUG_SKIP_BARRIER, **opts),
                want_stats=False)
    torch.cuda.synchronize()
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_bc_ex(G.handle, dev(srcs), out, sp.make_opts(**opts), want_stats=False)
    assert e.value.status == sp.SP_ERR_TIMEOUT
    sp.sp_bc_ex(G.handle, dev(srcs), out, sp.make_opts(**opts), want_stats=False)
    sp.sp_graph_sync(G.handle)
    want, _ = oracle.bc(g, srcs)
    close(out.cpu().numpy(), want, 1e-9, "after the latched timeout")
    G.close()


def test_bad_device_source_is_latched():
    g = gen.rmat(11, 8, 7)
    G = sp.Graph(g.row_ptr, g.col_idx)
    out = torch.zeros(g.n, dtype=torch.float64, device=DEV)
    sp.sp_bc_ex(G.handle, dev([1, 2, g.n]), out, sp.make_opts(form=sp.SP_FORM_BATCHED, batch=32),
                want_stats=False)
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_graph_sync(G.handle)
    assert e.value.status == sp.SP_ERR_INVALID_ARG
    sp.sp_graph_sync(G.handle)  # taken once
    with pytest.raises(sp.StarbcError) as e:  # host sources are checked before return
        sp.sp_bc(G.handle, np.array([0, -1], np.int32), out)
    assert e.value.status == sp.SP_ERR_INVALID_ARG
    G.close()


@pytest.mark.parametrize("precision", [sp.SP_FP64, sp.SP_FP32_DELTA])
def test_device_side_fallback_on_wide_counts(precision):
    # A 300 x 300 grid: counts up to C(598, 299) ~ 2^593 (past u32/u64 and,
    # within a level, past what FP32 dependencies can hold).  Asynchronous
    # calls on a fresh graph shape start with exact integer counts; the
    # device finds the overflow, runs the FP64 fallback in the same stream and
    # records the hint; the next call starts in FP64.  Both match the oracle.
    g = gen.grid(300, 300)
    srcs = np.array([0, 299, 300 * 300 - 1, 150 * 300 + 150], np.int32)
    want, _ = oracle.bc(g, srcs)
    for form, batch in [(sp.SP_FORM_BATCHED, 32), (sp.SP_FORM_PLAIN, 0)]:
        G = sp.Graph(g.row_ptr, g.col_idx)
        for _ in range(2):
            out = torch.full((g.n,), -1.0, dtype=torch.float64, device=DEV)
            sp.sp_bc_ex(G.handle, dev(srcs), out,
                        sp.make_opts(precision=precision, form=form, batch=batch, driver=sp.SP_DRIVER_PERSISTENT),
                        want_stats=False)
            sp.sp_graph_sync(G.handle)
            close(out.cpu().numpy(), want, 1e-9 if precision == sp.SP_FP64 else 1e-4, f"grid300 form {form}")
        G.close()
