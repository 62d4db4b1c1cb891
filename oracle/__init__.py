"""ORACLE — test infrastructure only.

A plain, slow, single-threaded CPU Brandes BC in FP64 (``brandes.c``), written
from the paper's ComputeBC program (Section 2, Fig. 1).  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package; the library under ``paper_2401_02472_gb300`` never does and
shares no code with it.

Functions
---------
bfs(g, src)          -> int32 dist[n] (-1 unreachable), FIFO BFS.
sigma(g, src, mode)  -> (mant, exp2, dist, stats): path counts mant * 2**exp2.
bc(g, sources, mode) -> (bc[n], per-source stats).
bc(..., directed=True), sigma(..., directed=True): the same on a directed
                     graph (CSR of out-arcs): BFS and dependencies over
                     out-arcs, path counts pulled over in-arcs.
bc_weighted(g, weights, sources, directed) -> (bc[n], dist[nsrc][n]): BC under
                     positive integer arc weights (``weighted.c``: Dijkstra
                     distances, then the same sums over the shortest-path DAG).
pagerank(g, damping, tol, max_iter) -> (pr[n], iterations, last L1 change):
                     pull-form PageRank of the paper's reduction listing
                     (``pagerank.c``), over in-arcs, FP64.
distance_sums(g, sources) -> (sum of d(s, t) over reached t, |R_s|) per source,
                     from a 64-source bit-parallel BFS (for the invariant
                     sum_v BC(v) = sum over reached ordered pairs of d - 1).

Modes: PLAIN (doubles; overflow reported as inf), XFLOAT (sigma with a 64-bit
exponent), AUTO (PLAIN per source, rerun in XFLOAT when sigma overflows).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

PLAIN, XFLOAT, AUTO = 0, 1, 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "brandes.c")
_PR_SRC = os.path.join(_HERE, "pagerank.c")
_W_SRC = os.path.join(_HERE, "weighted.c")
_SO = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off: no fused multiply-add, the arithmetic runs exactly as written.
CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


class SrcStats(ctypes.Structure):
    _fields_ = [
        ("levels", ctypes.c_int64),
        ("reached", ctypes.c_int64),
        ("arcs", ctypes.c_int64),
        ("used_xfloat", ctypes.c_int32),
        ("pad", ctypes.c_int32),
        ("max_level_spread_log2", ctypes.c_double),
    ]


STATS_DTYPE = np.dtype(
    [("levels", np.int64), ("reached", np.int64), ("arcs", np.int64), ("used_xfloat", np.int32),
     ("pad", np.int32), ("max_level_spread_log2", np.float64)]
)


def build(force: bool = False, src: str = _SRC, out: str = _SO, pr_src: str = _PR_SRC, w_src: str = _W_SRC) -> str:
    """Compile the oracle into a shared library (also used on tampered copies in tests)."""
    newest = max(os.path.getmtime(src), os.path.getmtime(pr_src), os.path.getmtime(w_src))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, src, pr_src, w_src, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, out)
    return out


def load(path: str | None = None):
    """ctypes handle of the oracle library (the default build unless `path` names another)."""
    global _lib
    if path is None:
        with _lock:
            if _lib is None:
                _lib = _declare(ctypes.CDLL(build()))
        return _lib
    return _declare(ctypes.CDLL(path))


def _declare(lib):
    i32, p = ctypes.c_int32, ctypes.c_void_p
    lib.oracle_bfs.argtypes = [i32, p, p, i32, p]
    lib.oracle_bfs.restype = ctypes.c_int
    lib.oracle_bc.argtypes = [i32, p, p, p, i32, ctypes.c_int, p, p]
    lib.oracle_bc.restype = ctypes.c_int
    lib.oracle_sigma.argtypes = [i32, p, p, i32, ctypes.c_int, p, p, p, p]
    lib.oracle_sigma.restype = ctypes.c_int
    lib.oracle_bc_directed.argtypes = [i32, p, p, p, i32, ctypes.c_int, p, p]
    lib.oracle_bc_directed.restype = ctypes.c_int
    lib.oracle_sigma_directed.argtypes = [i32, p, p, i32, ctypes.c_int, p, p, p, p]
    lib.oracle_sigma_directed.restype = ctypes.c_int
    lib.oracle_bc_weighted.argtypes = [i32, p, p, p, ctypes.c_int, p, i32, p, p]
    lib.oracle_bc_weighted.restype = ctypes.c_int
    lib.oracle_pagerank.argtypes = [i32, p, p, ctypes.c_double, ctypes.c_double, i32, p, p, p]
    lib.oracle_pagerank.restype = ctypes.c_int
    lib.oracle_distance_sums.argtypes = [i32, p, p, p, i32, p, p]
    lib.oracle_distance_sums.restype = ctypes.c_int
    return lib


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, np.int32)
    return rp, ci


def bfs(g, src: int, lib=None) -> np.ndarray:
    lib = lib or load()
    rp, ci = _csr(g)
    dist = np.empty(max(g.n, 1), np.int32)
    rc = lib.oracle_bfs(g.n, rp.ctypes.data, ci.ctypes.data, int(src), dist.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_bfs rc={rc}")
    return dist[: g.n]


def sigma(g, src: int, mode: int = AUTO, lib=None, directed: bool = False):
    lib = lib or load()
    rp, ci = _csr(g)
    mant = np.empty(g.n, np.float64)
    exp2 = np.empty(g.n, np.int64)
    dist = np.empty(g.n, np.int32)
    st = np.zeros(1, STATS_DTYPE)
    fn = lib.oracle_sigma_directed if directed else lib.oracle_sigma
    rc = fn(g.n, rp.ctypes.data, ci.ctypes.data, int(src), mode, mant.ctypes.data,
            exp2.ctypes.data, dist.ctypes.data, st.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_sigma rc={rc}")
    return mant, exp2, dist, st[0]


def bc(g, sources, mode: int = AUTO, lib=None, directed: bool = False):
    lib = lib or load()
    rp, ci = _csr(g)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).reshape(-1))
    out = np.empty(max(g.n, 1), np.float64)
    st = np.zeros(max(src.size, 1), STATS_DTYPE)
    nsrc = int(src.size)
    buf = src if nsrc else np.zeros(1, np.int32)
    fn = lib.oracle_bc_directed if directed else lib.oracle_bc
    rc = fn(g.n, rp.ctypes.data, ci.ctypes.data, buf.ctypes.data, nsrc, mode, out.ctypes.data, st.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_bc rc={rc}")
    return out[: g.n], st[:nsrc]


def distance_sums(g, sources, lib=None):
    """Per source: (sum of hop distances to reached vertices, reached count incl. the source)."""
    lib = lib or load()
    rp, ci = _csr(g)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).reshape(-1))
    nsrc = int(src.size)
    dsum = np.zeros(max(nsrc, 1), np.int64)
    reached = np.zeros(max(nsrc, 1), np.int64)
    buf = src if nsrc else np.zeros(1, np.int32)
    rc = lib.oracle_distance_sums(g.n, rp.ctypes.data, ci.ctypes.data, buf.ctypes.data, nsrc, dsum.ctypes.data,
                                  reached.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_distance_sums rc={rc}")
    return dsum[:nsrc], reached[:nsrc]


def pair_distance_excess(g, sources, threads: int = 1) -> int:
    """sum over sources s and reached t != s of (d(s, t) - 1), the total of all BC values.

    With threads > 1 the sources are cut into slices of 64 searched in parallel
    (the C code keeps no shared state and ctypes releases the GIL)."""
    src = np.asarray(sources, dtype=np.int32).reshape(-1)
    slices = [src[i:i + 64] for i in range(0, src.size, 64)]
    if threads > 1 and len(slices) > 1:
        from concurrent.futures import ThreadPoolExecutor

        with ThreadPoolExecutor(min(threads, len(slices))) as ex:
            parts = list(ex.map(lambda s: distance_sums(g, s), slices))
    else:
        parts = [distance_sums(g, s) for s in slices]
    return int(sum(int(d.sum()) - int((r - 1).sum()) for d, r in parts))


def pagerank(g, damping: float = 0.85, tol: float = 0.0, max_iter: int = 100, lib=None):
    """(pr[n], iterations run, last iteration's L1 change)."""
    lib = lib or load()
    rp, ci = _csr(g)
    pr = np.empty(max(g.n, 1), np.float64)
    it = ctypes.c_int32()
    ch = ctypes.c_double()
    rc = lib.oracle_pagerank(g.n, rp.ctypes.data, ci.ctypes.data, float(damping), float(tol), int(max_iter),
                             pr.ctypes.data, ctypes.byref(it), ctypes.byref(ch))
    if rc != 0:
        raise ValueError(f"oracle_pagerank rc={rc}")
    return pr[: g.n], it.value, ch.value


# ---------------------------------------------------------------------------
# Sampled-source BC (estimator and confidence bound), from the definitions:
# sources drawn uniformly with replacement by multiply-shift of SplitMix64
# outputs (the seeded generator shared with the GPU tests), estimate
# (n / k) sum_i delta_{s_i}(v), and the two-sided empirical Bernstein bound
# (Maurer and Pontil 2009, Theorem 4) with a union over the n vertices.

def sample_sources(n: int, seed: int, count: int, first: int = 0) -> np.ndarray:
    """s_i = floor(x_i * n / 2^64), x_i the SplitMix64 outputs of the seed, i = first ..."""
    import gen

    x = gen.draws(seed, first, count)
    return np.array([(int(v) * n) >> 64 for v in x], dtype=np.int32)


def approx_bc(g, seed: int, k: int, alpha: float = 0.1, directed: bool = False, lib=None):
    """(estimate[n], half-width of the normalised interval, per-source dependencies [k][n])."""
    n = g.n
    srcs = sample_sources(n, seed, k)
    deltas = np.stack([bc(g, [int(s)], lib=lib, directed=directed)[0] for s in srcs])
    estimate = deltas.sum(axis=0) * (n / k)
    c = n / ((n - 1.0) * (n - 2.0))
    y = deltas * c
    var = y.var(axis=0, ddof=1) if k > 1 else np.full(n, np.inf)
    L = np.log(4.0 * n / alpha)
    R = n / (n - 1.0)
    half = np.sqrt(2.0 * var.max() * L / k) + 7.0 * R * L / (3.0 * (k - 1.0))
    return estimate, float(half), deltas


def bc_weighted(g, weights, sources, directed: bool = False, lib=None):
    """(bc[n], dist[nsrc][n] with -1 unreachable) under arc weights parallel to col_idx."""
    lib = lib or load()
    rp, ci = _csr(g)
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.int32).reshape(-1))
    if w.size != g.nnz:
        raise ValueError("one weight per arc")
    wb = w if w.size else np.ones(1, np.int32)
    src = np.ascontiguousarray(np.asarray(sources, dtype=np.int32).reshape(-1))
    nsrc = int(src.size)
    out = np.empty(max(g.n, 1), np.float64)
    dist = np.empty(max(nsrc * g.n, 1), np.int64)
    buf = src if nsrc else np.zeros(1, np.int32)
    rc = lib.oracle_bc_weighted(g.n, rp.ctypes.data, ci.ctypes.data, wb.ctypes.data, int(directed), buf.ctypes.data,
                                nsrc, out.ctypes.data, dist.ctypes.data)
    if rc != 0:
        raise ValueError(f"oracle_bc_weighted rc={rc}")
    return out[: g.n], dist[: nsrc * g.n].reshape(nsrc, g.n)
