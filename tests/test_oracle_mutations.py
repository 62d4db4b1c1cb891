"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a dropped
term, a transposed operand, a wrong index or sign), builds the copy on the CPU
and checks that at least one pin from test_oracle.py rejects it.  The real
oracle is never modified.
"""
import math
import os

import numpy as np
import pytest

import gen
import oracle
from tests import bruteforce as bf

SRC = os.path.join(os.path.dirname(oracle.__file__), "brandes.c")

MUTATIONS = {
    "drop_one_plus": ("ratio * (1.0 + delta[w])", "ratio * (delta[w])"),
    "transpose_ratio": ("sigma[v] / sigma[w]", "sigma[w] / sigma[v]"),
    "transpose_xratio": ("xf_ratio(xsigma[v], xsigma[w])", "xf_ratio(xsigma[w], xsigma[v])"),
    "pred_wrong_side": ("if (dist[w] != dist[v] - 1) continue;", "if (dist[w] != dist[v] + 1) continue;"),
    "succ_wrong_side": ("if (dist[w] != dist[v] + 1) continue;", "if (dist[w] != dist[v] - 1) continue;"),
    "source_counted": ("for (int64_t i = reached - 1; i >= 1; --i)", "for (int64_t i = reached - 1; i >= 0; --i)"),
    "sigma_src_two": ("else sigma[src] = 1.0;", "else sigma[src] = 2.0;"),
    "xf_align_sign": ("a.m + scale2(b.m, -d)", "a.m + scale2(b.m, d)"),
    "xf_ratio_exp": ("scale2(a.m / b.m, a.e - b.e)", "scale2(a.m / b.m, b.e - a.e)"),
    "forward_skips_last": ("for (int64_t i = 1; i < reached; ++i)", "for (int64_t i = 1; i + 1 < reached; ++i)"),
    "directed_pull_over_out_arcs": ("(*tci)[fill[ci[e]]++] = u;", "(*tci)[fill[ci[e]]++] = ci[e];"),
    "directed_pulls_out_arcs": ("int rc = bc_over(n, rp, ci, trp, tci, sources, nsrc, mode, bc, stats);",
                                "int rc = bc_over(n, rp, ci, rp, ci, sources, nsrc, mode, bc, stats);"),
}


def pins_pass(lib) -> bool:
    """A compact battery of the oracle pins; False as soon as one fails."""
    def close(got, exact, rtol=1e-12):
        exact = np.asarray([float(x) for x in exact])
        return bool(np.all(np.abs(np.asarray(got) - exact) <= rtol * np.maximum(np.abs(exact), 1.0)))

    for seed in range(8):
        g = gen.random_small(7 + seed % 4, 0.4, seed)
        got, _ = oracle.bc(g, range(g.n), lib=lib)
        if not close(got, bf.bc_exact(g, range(g.n))):
            return False
    for seed in range(6):
        g = gen.random_small_directed(6 + seed % 3, 0.3, seed)
        got, _ = oracle.bc(g, range(g.n), lib=lib, directed=True)
        if not close(got, bf.bc_exact(g, range(g.n))):
            return False
    n = 9
    got, _ = oracle.bc(gen.path(n), range(n), lib=lib)
    if not close(got, [2 * i * (n - 1 - i) for i in range(n)]):
        return False
    g = gen.grid(12, 13)
    mant, exp2, dist, _ = oracle.sigma(g, 0, oracle.PLAIN, lib=lib)
    for i in range(12):
        for j in range(13):
            v = i * 13 + j
            if mant[v] * 2.0 ** int(exp2[v]) != math.comb(i + j, i):
                return False
    g = gen.grid(540, 540)
    got, _ = oracle.bc(g, [0], oracle.AUTO, lib=lib)
    want = bf.pair_distance_excess(g, [0])
    if not abs(got.sum() - want) <= 1e-9 * want:
        return False
    mant, exp2, _, _ = oracle.sigma(g, 0, oracle.XFLOAT, lib=lib)
    far = math.comb(1078, 539)
    shift = far.bit_length() - 64
    if abs(math.log2(mant[-1]) + int(exp2[-1]) - (shift + math.log2(far >> shift))) > 1e-9:
        return False
    return True


def test_unmodified_oracle_passes_the_battery():
    assert pins_pass(oracle.load())


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    before, after = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(before) == 1, name
    src = tmp_path / "mutant.c"
    src.write_text(text.replace(before, after))
    lib = oracle.load(oracle.build(force=True, src=str(src), out=str(tmp_path / "mutant.so")))
    assert not pins_pass(lib), name
