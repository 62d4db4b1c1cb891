"""sp_bc_noalloc, the entry point for callers that cannot allocate device memory.

It must give the same BC as sp_bc on the same inputs, call after call (the
static scratch it reuses keeps the previous call's contents), and reject
graphs beyond its fixed scratch size.  This file is collected last so that a
run that stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2401_02472_gb300 as sp

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def reference_bc(g, srcs):
    G = sp.Graph(g.row_ptr, g.col_idx)
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    sp.sp_bc_ex(G.handle, torch.as_tensor(srcs, device=DEV), out, sp.make_opts(form=sp.SP_FORM_PLAIN))
    torch.cuda.synchronize()
    G.close()
    return out.cpu().numpy()


def test_matches_sp_bc_on_two_calls_in_a_row():
    for g, k, seed in [(gen.rmat(12, 16, 2), 40, 5), (gen.knn2d(3000, 4, 3), 25, 6)]:
        srcs = gen.sources(g, k, seed)
        want = reference_bc(g, srcs)
        rp = torch.as_tensor(g.row_ptr, device=DEV)
        ci = torch.as_tensor(g.col_idx, device=DEV)
        src = torch.as_tensor(srcs, device=DEV)
        for _ in range(2):
            out = torch.full((g.n,), -1.0, dtype=torch.float64, device=DEV)
            sp.sp_bc_noalloc(rp, ci, src, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.all(np.abs(got - want) <= 1e-9 * np.maximum(np.abs(want), 1.0)), g.name


def test_rejects_graphs_beyond_the_scratch_size():
    rp = torch.zeros(4, dtype=torch.int32, device=DEV)
    ci = torch.zeros(1, dtype=torch.int32, device=DEV)
    src = torch.zeros(1, dtype=torch.int32, device=DEV)
    out = torch.zeros(3, dtype=torch.float64, device=DEV)
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_bc_noalloc(rp, ci, src, out, n=(1 << 18) + 1, nnz=0)
    assert e.value.status == sp.SP_ERR_TOO_LARGE
    with pytest.raises(sp.StarbcError) as e:
        sp.sp_bc_noalloc(rp, ci, src, out, n=3, nnz=(1 << 24) + 1)
    assert e.value.status == sp.SP_ERR_TOO_LARGE
    with pytest.raises(sp.StarbcError) as e:  # host memory is refused
        sp.sp_bc_noalloc(np.zeros(4, np.int32), np.zeros(1, np.int32), np.zeros(1, np.int32),
                         np.zeros(3, np.float64), n=3, nnz=1)
    assert e.value.status == sp.SP_ERR_INVALID_ARG


def test_matches_the_oracle_including_counts_past_64_bits():
    # Against the CPU oracle directly.  The 500 x 500 grid (250,000 vertices,
    # path counts up to C(998, 499) ~ 2^993) overflows the exact 64-bit
    # counts, so the call takes its second attempt with FP64 counts and
    # per-level exponents.
    for g, srcs in [(gen.er(2000, 10000, 1), np.arange(0, 2000, 13, dtype=np.int32)),
                    (gen.grid(500, 500), np.array([0, 499, 500 * 500 - 1], np.int32))]:
        want, _ = oracle.bc(g, srcs)
        rp = torch.as_tensor(g.row_ptr, device=DEV)
        ci = torch.as_tensor(g.col_idx, device=DEV)
        src = torch.as_tensor(srcs, device=DEV)
        for _ in range(2):
            out = torch.full((g.n,), -1.0, dtype=torch.float64, device=DEV)
            sp.sp_bc_noalloc(rp, ci, src, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            err = np.abs(got - want)
            assert np.all(err <= 1e-9 * np.maximum(np.abs(want), 1.0)), (g.name, err.max())
            assert np.all(got[want == 0.0] == 0.0)
