"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

Holds no betweenness-centrality arithmetic: random streams, CSR graph
construction and source selection only.  The heavy generators live in
``gen.c`` (built into ``_gen.so`` next to this file on first use); the small
structured graphs (path, star, cycle, grid, ...) are built here with numpy.

Every graph returned is a ``Graph(n, row_ptr, col_idx)`` with int32 arrays,
undirected (both arc directions stored), rows sorted, no self-loops and no
duplicate arcs.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "_gen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into _gen.so (OpenMP if the compiler has it)."""
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O3", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            p = ctypes.c_void_p
            lib.gen_er.argtypes = [i32, i64, u64, p, p, p]
            lib.gen_er.restype = ctypes.c_int
            lib.gen_rmat.argtypes = [i32, i32, f64, f64, f64, u64, p, p, p]
            lib.gen_rmat.restype = ctypes.c_int
            lib.gen_rmat_directed.argtypes = [i32, i32, f64, f64, f64, u64, p, p, p]
            lib.gen_rmat_directed.restype = ctypes.c_int
            lib.gen_knn2d.argtypes = [i32, i32, u64, p, p, p, p]
            lib.gen_knn2d.restype = ctypes.c_int
            lib.gen_sources.argtypes = [i32, p, i32, u64, p]
            lib.gen_sources.restype = i64
            lib.gen_draws.argtypes = [u64, u64, i64, p]
            lib.gen_draws.restype = None
            lib.gen_substream.argtypes = [u64, u64]
            lib.gen_substream.restype = u64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int32[n+1]
    col_idx: np.ndarray  # int32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))


# --------------------------------------------------------------------------
# Large seeded generators (C)

def er(n: int, m: int, seed: int) -> Graph:
    """Erdos-Renyi G(n, m): m distinct undirected edges, uniform endpoints."""
    lib = _load()
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(2 * m, np.int32)
    nnz = np.zeros(1, np.int64)
    rc = lib.gen_er(n, m, seed, _ptr(rp), _ptr(ci), _ptr(nnz))
    if rc != 0:
        raise ValueError(f"gen_er failed ({rc})")
    return Graph(n, rp, ci[: nnz[0]].copy(), f"er_n{n}_m{m}_s{seed}")


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19) -> Graph:
    """RMAT with seeded relabelling, symmetrised, deduped, self-loops dropped."""
    lib = _load()
    n = 1 << scale
    m = edge_factor * n
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(2 * m, np.int32)
    nnz = np.zeros(1, np.int64)
    rc = lib.gen_rmat(scale, edge_factor, a, b, c, seed, _ptr(rp), _ptr(ci), _ptr(nnz))
    if rc != 0:
        raise ValueError(f"gen_rmat failed ({rc})")
    return Graph(n, rp, ci[: nnz[0]].copy(), f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def rmat_directed(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19) -> Graph:
    """Directed RMAT: every draw is one arc u -> v (seeded relabelling, deduped, no self-loops)."""
    lib = _load()
    n = 1 << scale
    m = edge_factor * n
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(m, np.int32)
    nnz = np.zeros(1, np.int64)
    rc = lib.gen_rmat_directed(scale, edge_factor, a, b, c, seed, _ptr(rp), _ptr(ci), _ptr(nnz))
    if rc != 0:
        raise ValueError(f"gen_rmat_directed failed ({rc})")
    return Graph(n, rp, ci[: nnz[0]].copy(), f"drmat_s{scale}_ef{edge_factor}_s{seed}")


def knn2d(n: int, k: int, seed: int, return_points: bool = False):
    """Symmetrised k-nearest-neighbour graph of n uniform points in [0,1)^2."""
    lib = _load()
    xy = np.empty((n, 2), np.float64)
    rp = np.empty(n + 1, np.int32)
    ci = np.empty(2 * k * n, np.int32)
    nnz = np.zeros(1, np.int64)
    rc = lib.gen_knn2d(n, k, seed, _ptr(xy), _ptr(rp), _ptr(ci), _ptr(nnz))
    if rc != 0:
        raise ValueError(f"gen_knn2d failed ({rc})")
    g = Graph(n, rp, ci[: nnz[0]].copy(), f"knn{k}_n{n}_s{seed}")
    return (g, xy) if return_points else g


def sources(g: Graph, k: int, seed: int) -> np.ndarray:
    """k distinct sources, uniform among vertices with degree >= 1, draw order."""
    lib = _load()
    out = np.empty(max(k, 1), np.int32)
    cnt = lib.gen_sources(g.n, _ptr(g.row_ptr), k, seed, _ptr(out))
    if cnt < 0:
        raise ValueError("not enough vertices with degree >= 1")
    return out[:k].copy()


def draws(seed: int, first: int, count: int) -> np.ndarray:
    """Raw 64-bit draws first..first+count-1 of the SplitMix64 stream `seed`."""
    lib = _load()
    out = np.empty(max(count, 1), np.uint64)
    lib.gen_draws(seed, first, count, _ptr(out))
    return out[:count].copy()


def uniforms(seed: int, first: int, count: int) -> np.ndarray:
    """Doubles in [0,1) from the top 53 bits of each draw."""
    return (draws(seed, first, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def substream(seed: int, tag: int) -> int:
    return int(_load().gen_substream(seed, tag))


# --------------------------------------------------------------------------
# Structured graphs (numpy)

def from_edges(n: int, edges, name: str = "") -> Graph:
    """Undirected CSR from an iterable of (u, v) pairs; symmetrised, deduped, loops dropped."""
    e = np.asarray(list(edges) if not isinstance(edges, np.ndarray) else edges, dtype=np.int64).reshape(-1, 2)
    if e.size:
        if e.min() < 0 or e.max() >= n:
            raise ValueError("edge endpoint out of range")
        e = e[e[:, 0] != e[:, 1]]
        both = np.concatenate([e, e[:, ::-1]], axis=0)
        key = np.unique(both[:, 0] * np.int64(max(n, 1)) + both[:, 1])
        src = (key // max(n, 1)).astype(np.int64)
        dst = (key % max(n, 1)).astype(np.int32)
    else:
        src = np.zeros(0, np.int64)
        dst = np.zeros(0, np.int32)
    counts = np.bincount(src, minlength=n) if n > 0 else np.zeros(0, np.int64)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(counts)
    return Graph(n, rp, dst.astype(np.int32), name)


def from_arcs(n: int, arcs, name: str = "") -> Graph:
    """Directed CSR from an iterable of arcs (u, v): rows sorted, repeated arcs once, loops dropped."""
    e = np.asarray(list(arcs) if not isinstance(arcs, np.ndarray) else arcs, dtype=np.int64).reshape(-1, 2)
    if e.size:
        if e.min() < 0 or e.max() >= n:
            raise ValueError("arc endpoint out of range")
        e = e[e[:, 0] != e[:, 1]]
        key = np.unique(e[:, 0] * np.int64(max(n, 1)) + e[:, 1])
        src = (key // max(n, 1)).astype(np.int64)
        dst = (key % max(n, 1)).astype(np.int32)
    else:
        src = np.zeros(0, np.int64)
        dst = np.zeros(0, np.int32)
    counts = np.bincount(src, minlength=n) if n > 0 else np.zeros(0, np.int64)
    rp = np.zeros(n + 1, np.int32)
    rp[1:] = np.cumsum(counts)
    return Graph(n, rp, dst.astype(np.int32), name)


def transpose(g: Graph) -> Graph:
    """The graph with every arc reversed."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr.astype(np.int64)))
    return from_arcs(g.n, np.stack([g.col_idx.astype(np.int64), rows], 1), g.name + "^T")


def random_small_directed(n: int, p: float, seed: int) -> Graph:
    """Random digraph on small n: arc (i, j), i != j, present iff its uniform draw < p."""
    pairs = [(i, j) for i in range(n) for j in range(n) if i != j]
    u = uniforms(substream(seed, 8), 0, len(pairs))
    return from_arcs(n, [pq for pq, x in zip(pairs, u) if x < p], f"dgnp{n}_{p}_s{seed}")


def _mix64_np(z: np.ndarray) -> np.ndarray:
    """SplitMix64's finaliser (Steele, Lea, Flood 2014), vectorised over uint64."""
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def edge_weights(g: Graph, seed: int, lo: int = 1, hi: int = 100, symmetric: bool = True) -> np.ndarray:
    """Integer weights in [lo, hi], uniform, one per arc (parallel to col_idx), seeded per edge:
    key = (u, v), or (min, max) when symmetric so both arcs of an undirected edge agree."""
    rows = np.repeat(np.arange(g.n, dtype=np.uint64), np.diff(g.row_ptr.astype(np.int64)))
    cols = g.col_idx.astype(np.uint64)
    if symmetric:
        rows, cols = np.minimum(rows, cols), np.maximum(rows, cols)
    key = rows * np.uint64(max(g.n, 1)) + cols
    with np.errstate(over="ignore"):
        x = _mix64_np(np.uint64(seed) + (key + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15))
    span = np.uint64(hi - lo + 1)
    return (lo + (x % span).astype(np.int64)).astype(np.int32)


def path(n: int) -> Graph:
    return from_edges(n, [(i, i + 1) for i in range(n - 1)], f"path{n}")


def star(n: int) -> Graph:
    return from_edges(n, [(0, i) for i in range(1, n)], f"star{n}")


def cycle(n: int) -> Graph:
    return from_edges(n, [(i, (i + 1) % n) for i in range(n)], f"cycle{n}")


def complete(n: int) -> Graph:
    return from_edges(n, [(i, j) for i in range(n) for j in range(i + 1, n)], f"K{n}")


def grid(rows: int, cols: int) -> Graph:
    """rows x cols 4-connected grid; vertex id = i * cols + j."""
    ids = np.arange(rows * cols, dtype=np.int64).reshape(rows, cols)
    h = np.stack([ids[:, :-1].ravel(), ids[:, 1:].ravel()], axis=1)
    v = np.stack([ids[:-1, :].ravel(), ids[1:, :].ravel()], axis=1)
    return from_edges(rows * cols, np.concatenate([h, v], axis=0), f"grid{rows}x{cols}")


def disjoint_union(*graphs: Graph) -> Graph:
    rps, cis, off, eoff = [np.zeros(1, np.int64)], [], 0, 0
    for g in graphs:
        rps.append(g.row_ptr[1:].astype(np.int64) + eoff)
        cis.append(g.col_idx.astype(np.int64) + off)
        off += g.n
        eoff += g.nnz
    rp = np.concatenate(rps).astype(np.int32)
    ci = np.concatenate(cis).astype(np.int32) if cis else np.zeros(0, np.int32)
    return Graph(off, rp, ci, "+".join(g.name for g in graphs))


def random_small(n: int, p: float, seed: int) -> Graph:
    """G(n, p) on small n: edge {i<j} present iff its uniform draw < p."""
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    u = uniforms(substream(seed, 7), 0, len(pairs))
    return from_edges(n, [pq for pq, x in zip(pairs, u) if x < p], f"gnp{n}_{p}_s{seed}")


# --------------------------------------------------------------------------
# Named workloads (synthetic stand-ins for the paper's input table)

def workload_graph(name: str) -> Graph:
    """The five benchmark graphs, by name."""
    if name == "er2000":
        return er(2000, 10000, 1)
    if name == "rmat20":
        return rmat(20, 16, 2)
    if name == "knn4_1m":
        return knn2d(1_000_000, 4, 3)
    if name == "rmat22":
        return rmat(22, 16, 4)
    if name == "rmat21":
        return rmat(21, 16, 4)
    if name == "drmat22":
        return rmat_directed(22, 16, 4)
    raise KeyError(name)


def poisson_arrivals(rate_per_s: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process: exponential gaps by inversion."""
    expect = int(rate_per_s * duration_s * 1.5 + 64)
    u = uniforms(substream(seed, 11), 0, expect)
    gaps = -np.log1p(-u) / rate_per_s
    t = np.cumsum(gaps)
    return t[t < duration_s]


def log_uniform_int(lo: int, hi: int, seed: int, count: int) -> np.ndarray:
    """Integers in [lo, hi] whose logarithm is uniform."""
    u = uniforms(substream(seed, 12), 0, count)
    x = np.exp(math.log(lo) + u * (math.log(hi + 1) - math.log(lo)))
    return np.clip(np.floor(x).astype(np.int64), lo, hi)
