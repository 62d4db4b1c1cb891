"""Parity at the benchmark sizes, in the launch configurations bench.py times.

The oracle cannot run every source of the large workloads in test time, so:
  RMAT scale 20, 64 sources:     the whole source set against the oracle;
  4-NN, 10^6 points, 256 sources: 8 sources against the oracle, and the full
                                  call against the invariant sum_v BC(v) =
                                  sum over reached ordered pairs (d - 1) with
                                  distances from the oracle's BFS;
  RMAT scale 22, 1,024 sources:   the first 32 sources, as a call of their
                                  own, against the oracle in FP64 and FP32
                                  (widths 32, 128 and 256), the full autotuned
                                  call against the same invariant (distance
                                  sums from the oracle's 64-source BFS) and
                                  against the sum of two half calls.
"""
from concurrent.futures import ThreadPoolExecutor
import os

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2401_02472_gb300 as sp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def gpu_bc(G, srcs, precision, form=sp.SP_FORM_AUTO, batch=0):
    out = torch.empty(G.n, dtype=torch.float64, device=DEV)
    st = sp.sp_bc_ex(G.handle, torch.as_tensor(np.asarray(srcs, np.int32), device=DEV), out,
                     sp.make_opts(precision=precision, form=form, batch=batch))
    torch.cuda.synchronize()
    return out.cpu().numpy(), st


def assert_close(got, want, rtol, what):
    err = np.abs(got - want)
    bad = np.nonzero(err > rtol * np.maximum(np.abs(want), 1.0))[0]
    assert bad.size == 0, f"{what}: {bad.size} vertices off, e.g. {bad[:3]} {got[bad[:3]]} vs {want[bad[:3]]}"
    assert np.all(got[want == 0.0] == 0.0), what


def test_rmat20_64_sources_all_against_oracle():
    g = gen.workload_graph("rmat20")
    srcs = gen.sources(g, 64, 12)
    G = sp.Graph(g.row_ptr, g.col_idx)
    want, ost = oracle.bc(g, srcs)
    for prec, rtol in [(sp.SP_FP64, 1e-9), (sp.SP_FP32_DELTA, 1e-4)]:
        got, st = gpu_bc(G, srcs, prec, sp.SP_FORM_BATCHED, 64)
        assert_close(got, want, rtol, f"rmat20 precision {prec}")
        assert st["traversed_arcs"] == int(ost["arcs"].sum())


def test_knn_1m_256_sources():
    g = gen.workload_graph("knn4_1m")
    srcs = gen.sources(g, 256, 13)
    G = sp.Graph(g.row_ptr, g.col_idx)
    # eight sources against the oracle (its extended-exponent mode handles the path counts)
    got8, _ = gpu_bc(G, srcs[:8], sp.SP_FP32_DELTA)
    want8, _ = oracle.bc(g, srcs[:8])
    assert_close(got8, want8, 1e-4, "knn 8 sources")
    # the whole call against the pair-distance invariant
    got, st = gpu_bc(G, srcs, sp.SP_FP32_DELTA)
    excess = 0
    for s in srcs:
        d = oracle.bfs(g, int(s))
        r = d[d > 0]
        excess += int((r - 1).sum())
    assert abs(got.sum() - excess) <= 1e-4 * excess
    assert st["max_levels"] > 1000
    assert st["sigma_float"] == 1  # path counts pass 2^64: the FP64 per-level-exponent path ran
    assert st["promoted"] == 0  # recentred at +-2^64, theta-hat stays in FP32


def test_rmat22_sampled_sources_and_split_linearity():
    g = gen.workload_graph("rmat22")
    srcs = gen.sources(g, 1024, 14)
    G = sp.Graph(g.row_ptr, g.col_idx)
    # the oracle over the first 32 sources, one slice per host thread (BC is a
    # sum over sources; the slices differ from one pass by rounding only)
    spot = srcs[:32]
    parts = np.array_split(spot, min(len(spot), os.cpu_count() or 1))
    with ThreadPoolExecutor(len(parts)) as ex:
        want = sum(ex.map(lambda p: oracle.bc(g, p)[0], parts))
    for prec, rtol in [(sp.SP_FP64, 1e-9), (sp.SP_FP32_DELTA, 1e-4)]:
        for width in (32, 128, 256):
            got, _ = gpu_bc(G, spot, prec, sp.SP_FORM_BATCHED, width)
            assert_close(got, want, rtol, f"rmat22 32 sources precision {prec} width {width}")
    full, st = gpu_bc(G, srcs, sp.SP_FP32_DELTA)
    # the whole call: sum of BC = sum over reached ordered pairs of (d - 1)
    excess = oracle.pair_distance_excess(g, srcs, threads=os.cpu_count() or 1)
    assert abs(full.sum() - excess) <= 1e-4 * excess, (full.sum(), excess)
    a, _ = gpu_bc(G, srcs[:512], sp.SP_FP32_DELTA, sp.SP_FORM_BATCHED, st["batch"])
    b, _ = gpu_bc(G, srcs[512:], sp.SP_FP32_DELTA, sp.SP_FORM_BATCHED, st["batch"])
    assert_close(full, a + b, 1e-4, "rmat22 split")
