"""Sampled-source BC on the GPU (sp_bc_approx) against the oracle's estimator.

The GPU draws the sources itself (SplitMix64, multiply-shift); the oracle
draws the same ones through the shared seeded generator and computes the
estimate and the empirical Bernstein half-width from exact per-source
dependencies.  Estimates agree within the BC tolerance of the precision,
half-widths within 1e-6 relative (sample variances from sums taken in
another order).
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
    err = np.abs(got - want)
    bad = np.nonzero(err > rtol * np.maximum(np.abs(want), 1.0))[0]
    assert bad.size == 0, f"{what}: {bad.size} off, e.g. {bad[:3]} {got[bad[:3]]} vs {want[bad[:3]]}"


@pytest.mark.parametrize("form,precision", [(sp.SP_FORM_BATCHED, sp.SP_FP64), (sp.SP_FORM_PLAIN, sp.SP_FP64),
                                            (sp.SP_FORM_BATCHED, sp.SP_FP32_DELTA)])
@pytest.mark.parametrize("name", ["er", "rmat", "drmat"])
def test_fixed_sample_matches_the_oracle(name, form, precision):
    g, flags = {"er": (gen.er(1500, 6000, 2), 0), "rmat": (gen.rmat(11, 8, 3), 0),
                "drmat": (gen.rmat_directed(11, 8, 4), sp.SP_GRAPH_DIRECTED)}[name]
    G = sp.Graph(g.row_ptr, g.col_idx, flags=flags)
    k = 300
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    # eps far below reach: exactly k_min = k_max = k sources
    st = sp.sp_bc_approx(G.handle, out, seed=5, eps=1e-12, alpha=0.1, k_min=k, k_max=k,
                         opts=sp.make_opts(precision=precision, form=form))
    assert st["sources"] == k and st["rounds"] == 1 and st["converged"] == 0
    want, half, _ = oracle.approx_bc(g, 5, k, alpha=0.1, directed=bool(flags))
    close(out.cpu().numpy(), want, 1e-9 if precision == sp.SP_FP64 else 1e-4, name)
    assert abs(st["bound"] - half) <= 1e-6 * half


def test_adaptive_rounds_reach_the_bound():
    g = gen.rmat(10, 8, 6)
    G = sp.Graph(g.row_ptr, g.col_idx)
    host = np.empty(g.n, np.float64)
    st = sp.sp_bc_approx(G.handle, host, seed=9, eps=0.05, alpha=0.1, k_min=64, k_max=1 << 16)
    assert st["converged"] == 1 and st["bound"] <= 0.05 and st["rounds"] > 1
    want, half, _ = oracle.approx_bc(g, 9, st["sources"], alpha=0.1)
    close(host, want, 1e-9, "adaptive")
    assert abs(st["bound"] - half) <= 1e-6 * half
    # the estimate is within the bound of BC over all sources (normalised)
    n = g.n
    exact = oracle.bc(g, range(n))[0]
    assert np.all(np.abs(host - exact) / ((n - 1.0) * (n - 2.0)) <= st["bound"])


def test_arguments_are_checked():
    g = gen.er(100, 300, 1)
    G = sp.Graph(g.row_ptr, g.col_idx)
    out = torch.empty(g.n, dtype=torch.float64, device=DEV)
    for kw in [dict(eps=0.0), dict(alpha=1.0), dict(k_min=1), dict(k_min=10, k_max=5)]:
        args = dict(seed=1, eps=0.1, alpha=0.1, k_min=16, k_max=64)
        args.update(kw)
        with pytest.raises(sp.StarbcError) as e:
            sp.sp_bc_approx(G.handle, out, **args)
        assert e.value.status == sp.SP_ERR_INVALID_ARG
