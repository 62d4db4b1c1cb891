"""Python binding of libstarbc (Brandes betweenness centrality on GB300).

Argument marshalling only: every function here calls the C entry point of the
same name in ``include/starbc.h``; all graph work runs in the library's CUDA
kernels.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; their
data pointers are passed through unchanged, so device tensors stay on the
device.  ``stream`` defaults to torch's current CUDA stream.

The shared library is built in-tree (``_build.py``) and there is no fallback:
importing this package on a machine where the library can neither be loaded
nor built raises ImportError.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build

SP_OK, SP_NOT_READY = 0, 1
SP_ERR_INVALID_ARG, SP_ERR_OOM, SP_ERR_CUDA, SP_ERR_TOO_LARGE = -1, -2, -3, -4
SP_ERR_RANGE, SP_ERR_TIMEOUT, SP_ERR_CANCELLED, SP_ERR_BAD_GRAPH, SP_ERR_NO_DEVICE = -5, -6, -7, -8, -9
SP_FP64, SP_FP32_DELTA = 0, 1
SP_FORM_AUTO, SP_FORM_PLAIN, SP_FORM_BATCHED, SP_FORM_SMALL, SP_FORM_WEIGHTED = 0, 1, 2, 3, 4
SP_DRIVER_AUTO, SP_DRIVER_PERSISTENT, SP_DRIVER_GRAPH = 0, 1, 2
SP_GRAPH_CHECK_SYMMETRIC, SP_GRAPH_SORT_ROWS, SP_GRAPH_DIRECTED = 0x1, 0x2, 0x4
SP_DEBUG_SKIP_BARRIER = 0x1
SP_DEBUG_PLAIN_RECORDS = 0x2
SP_DEBUG_PLAIN_ARRAYS = 0x4
SP_BC_KEEP_ORDER = 0x1


class sp_bc_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("form", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("max_ctas", ctypes.c_int32), ("barrier_timeout_ns", ctypes.c_int64),
                ("debug_flags", ctypes.c_int32), ("flags", ctypes.c_int32), ("bottom_up", ctypes.c_int32),
                ("driver", ctypes.c_int32)]


class sp_bc_stats(ctypes.Structure):
    _fields_ = [("traversed_arcs", ctypes.c_int64), ("reached", ctypes.c_int64), ("entries", ctypes.c_int64),
                ("scanned_arcs", ctypes.c_int64), ("dag_arcs", ctypes.c_int64), ("kernel_ms", ctypes.c_double),
                ("max_levels", ctypes.c_int32), ("batches", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("form", ctypes.c_int32), ("promoted", ctypes.c_int32), ("sigma_float", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("tuned", ctypes.c_int32), ("driver", ctypes.c_int32),
                ("bottom_up", ctypes.c_int32), ("shared", ctypes.c_int32), ("recentred", ctypes.c_int32),
                ("joined", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sp_approx_stats(ctypes.Structure):
    _fields_ = [("sources", ctypes.c_int64), ("rounds", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("bound", ctypes.c_double), ("kernel_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sp_graph_info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("max_degree", ctypes.c_int32), ("nnz", ctypes.c_int64),
                ("isolated", ctypes.c_int64), ("sorted_rows", ctypes.c_int32), ("has_self_loops", ctypes.c_int32),
                ("has_duplicates", ctypes.c_int32), ("symmetric", ctypes.c_int32), ("directed", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class StarbcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(message)
        self.status = status


# Every exported C symbol with its argument and result types.
_P, _I32, _I64, _U32, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t
SIGNATURES = {
    "sp_graph_create": ([_P, _P, _I32, _I64, _U32, _P, _P], ctypes.c_int),
    "sp_graph_destroy": ([_P], ctypes.c_int),
    "sp_graph_sync": ([_P, _P], ctypes.c_int),
    "sp_graph_set_weights": ([_P, _P, _P], ctypes.c_int),
    "sp_sssp": ([_P, _P, _I32, _P, _P], ctypes.c_int),
    "sp_graph_get_info": ([_P, _P], ctypes.c_int),
    "sp_graph_from_edges": ([_P, _P, _I64, _I32, _U32, _P, _P], ctypes.c_int),
    "sp_graph_get_csr": ([_P, _P, _P, _P], ctypes.c_int),
    "sp_bc_opts_default": ([_P], None),
    "sp_bc": ([_P, _P, _I32, _P, _P], ctypes.c_int),
    "sp_bc_ex": ([_P, _P, _I32, _P, _P, _P, _P], ctypes.c_int),
    "sp_bfs": ([_P, _P, _I32, _P, _P], ctypes.c_int),
    "sp_sigma": ([_P, _I32, _P, _P, _P], ctypes.c_int),
    "sp_pagerank": ([_P, ctypes.c_double, ctypes.c_double, _I32, _P, _P, _P, _P], ctypes.c_int),
    "sp_bc_approx": ([_P, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, _I64, _I64, _P, _P, _P, _P],
                     ctypes.c_int),
    "sp_bc_noalloc": ([_P, _P, _I32, _I64, _P, _I32, _P, _P], ctypes.c_int),
    "sp_server_create": ([_SZ, _I32, _P], ctypes.c_int),
    "sp_server_add_graph": ([_P, _P, _P], ctypes.c_int),
    "sp_server_set_live": ([_P, _I32], ctypes.c_int),
    "sp_bc_submit": ([_P, _I32, _P, _I32, _P, _P, _P], ctypes.c_int),
    "sp_pagerank_submit": ([_P, _I32, ctypes.c_double, ctypes.c_double, _I32, _P, _P], ctypes.c_int),
    "sp_request_pagerank": ([_P, _I64, _P, _P], ctypes.c_int),
    "sp_bc_poll": ([_P, _I64], ctypes.c_int),
    "sp_bc_wait": ([_P, _I64, _I64], ctypes.c_int),
    "sp_bc_cancel": ([_P, _I64], ctypes.c_int),
    "sp_request_times": ([_P, _I64, _P, _P, _P], ctypes.c_int),
    "sp_request_stats": ([_P, _I64, _P], ctypes.c_int),
    "sp_server_destroy": ([_P], ctypes.c_int),
    "sp_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "sp_last_error": ([], ctypes.c_char_p),
}


def _load():
    path = _build.LIB
    if _build.stale():
        try:
            path = _build.build()
        except Exception as e:  # no nvcc, or a compile error: no fallback exists
            raise ImportError(f"libstarbc could not be built: {e}") from e
    lib = ctypes.CDLL(path)
    for name, (args, res) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    return lib


lib = _load()
LIB_PATH = _build.LIB


def _check(rc: int, what: str):
    if rc not in (SP_OK,):
        msg = (lib.sp_last_error() or b"").decode()
        name = (lib.sp_status_string(rc) or b"").decode()
        raise StarbcError(rc, f"{what}: {name}: {msg}")


def _ptr(x) -> int:
    """Data pointer of a torch tensor or numpy array (must be contiguous)."""
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _check_dtype(x, kind: str, what: str):
    name = str(getattr(x, "dtype", ""))
    if not name.endswith(kind):
        raise TypeError(f"{what} must be {kind}, got {name}")


def _stream(stream) -> int:
    if stream is not None:
        return int(stream)
    try:
        import torch

        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return 0


def _count(x) -> int:
    return int(x.numel()) if hasattr(x, "numel") else int(np.asarray(x).size)


# ---------------------------------------------------------------------------
# C entry points, same names

def sp_graph_create(row_ptr, col_idx, n: int | None = None, nnz: int | None = None, flags: int = 0,
                    stream=None) -> int:
    _check_dtype(row_ptr, "int32", "row_ptr")
    _check_dtype(col_idx, "int32", "col_idx")
    n = _count(row_ptr) - 1 if n is None else n
    nnz = _count(col_idx) if nnz is None else nnz
    h = ctypes.c_void_p()
    _check(lib.sp_graph_create(_ptr(row_ptr), _ptr(col_idx) if nnz else None, n, nnz, flags, _stream(stream),
                               ctypes.byref(h)), "sp_graph_create")
    return h.value


def sp_graph_destroy(g: int):
    _check(lib.sp_graph_destroy(g), "sp_graph_destroy")


def sp_graph_sync(g: int, stream=None):
    """Wait for the stream; raise the error an earlier asynchronous call on g latched."""
    _check(lib.sp_graph_sync(g, _stream(stream)), "sp_graph_sync")


def sp_graph_set_weights(g: int, weights, stream=None):
    _check_dtype(weights, "int32", "weights")
    _check(lib.sp_graph_set_weights(g, _ptr(weights), _stream(stream)), "sp_graph_set_weights")


def sp_sssp(g: int, sources, dist_out, stream=None):
    _check_dtype(sources, "int32", "sources")
    _check_dtype(dist_out, "int32", "dist_out")
    _check(lib.sp_sssp(g, _ptr(sources), _count(sources), _ptr(dist_out), _stream(stream)), "sp_sssp")


def sp_graph_from_edges(src, dst, n: int, flags: int = 0, stream=None) -> int:
    _check_dtype(src, "int32", "src")
    _check_dtype(dst, "int32", "dst")
    m = _count(src)
    if _count(dst) != m:
        raise ValueError("src and dst differ in length")
    h = ctypes.c_void_p()
    _check(lib.sp_graph_from_edges(_ptr(src) if m else None, _ptr(dst) if m else None, m, n, flags,
                                   _stream(stream), ctypes.byref(h)), "sp_graph_from_edges")
    return h.value


def sp_graph_get_csr(g: int, row_ptr_out, col_idx_out, stream=None):
    _check_dtype(row_ptr_out, "int32", "row_ptr_out")
    _check_dtype(col_idx_out, "int32", "col_idx_out")
    _check(lib.sp_graph_get_csr(g, _ptr(row_ptr_out), _ptr(col_idx_out), _stream(stream)), "sp_graph_get_csr")


def sp_graph_get_info(g: int) -> dict:
    info = sp_graph_info()
    _check(lib.sp_graph_get_info(g, ctypes.byref(info)), "sp_graph_get_info")
    return info.as_dict()


def make_opts(precision=SP_FP64, form=SP_FORM_AUTO, batch=0, max_ctas=0, barrier_timeout_ns=0,
              debug_flags=0, flags=0, bottom_up=0, driver=SP_DRIVER_AUTO) -> sp_bc_opts:
    o = sp_bc_opts()
    lib.sp_bc_opts_default(ctypes.byref(o))
    o.precision, o.form, o.batch, o.max_ctas = precision, form, batch, max_ctas
    o.barrier_timeout_ns, o.debug_flags, o.flags, o.bottom_up = barrier_timeout_ns, debug_flags, flags, bottom_up
    o.driver = driver
    return o


def sp_bc(g: int, sources, bc_out, stream=None):
    _check_dtype(sources, "int32", "sources")
    _check_dtype(bc_out, "float64", "bc_out")
    _check(lib.sp_bc(g, _ptr(sources), _count(sources), _ptr(bc_out), _stream(stream)), "sp_bc")


def sp_bc_ex(g: int, sources, bc_out, opts: sp_bc_opts | None = None, stream=None, want_stats: bool = True):
    _check_dtype(sources, "int32", "sources")
    _check_dtype(bc_out, "float64", "bc_out")
    st = sp_bc_stats()
    _check(lib.sp_bc_ex(g, _ptr(sources), _count(sources), ctypes.byref(opts) if opts is not None else None,
                        _ptr(bc_out), ctypes.byref(st) if want_stats else None, _stream(stream)), "sp_bc_ex")
    return st.as_dict() if want_stats else None


def sp_bfs(g: int, sources, dist_out, stream=None):
    _check_dtype(sources, "int32", "sources")
    _check_dtype(dist_out, "int32", "dist_out")
    _check(lib.sp_bfs(g, _ptr(sources), _count(sources), _ptr(dist_out), _stream(stream)), "sp_bfs")


def sp_sigma(g: int, src: int, mant_out, exp2_out, stream=None):
    _check_dtype(mant_out, "float64", "mant_out")
    _check_dtype(exp2_out, "int64", "exp2_out")
    _check(lib.sp_sigma(g, int(src), _ptr(mant_out), _ptr(exp2_out), _stream(stream)), "sp_sigma")


def sp_bc_approx(g: int, bc_out, seed: int, eps: float, alpha: float = 0.1, k_min: int = 256,
                 k_max: int = 1 << 20, opts: sp_bc_opts | None = None, stream=None) -> dict:
    """Sampled-source BC estimate into bc_out; returns the sampling statistics."""
    _check_dtype(bc_out, "float64", "bc_out")
    st = sp_approx_stats()
    _check(lib.sp_bc_approx(g, int(seed) & (2**64 - 1), float(eps), float(alpha), int(k_min), int(k_max),
                            ctypes.byref(opts) if opts is not None else None, _ptr(bc_out), ctypes.byref(st),
                            _stream(stream)), "sp_bc_approx")
    return st.as_dict()


def sp_pagerank(g: int, pr_out, damping: float = 0.85, tol: float = 0.0, max_iter: int = 100, stream=None,
                want_result: bool = True):
    """PageRank into pr_out; returns (iterations, last L1 change), or None when want_result is False
    (then a device pr_out makes the call asynchronous)."""
    _check_dtype(pr_out, "float64", "pr_out")
    it = ctypes.c_int32()
    ch = ctypes.c_double()
    _check(lib.sp_pagerank(g, float(damping), float(tol), int(max_iter), _ptr(pr_out),
                           ctypes.byref(it) if want_result else None, ctypes.byref(ch) if want_result else None,
                           _stream(stream)), "sp_pagerank")
    return (it.value, ch.value) if want_result else None


def sp_bc_noalloc(row_ptr, col_idx, sources, bc_out, n: int | None = None, nnz: int | None = None, stream=None):
    """BC with no device allocation; every array must be device memory (see include/starbc.h)."""
    _check_dtype(row_ptr, "int32", "row_ptr")
    _check_dtype(col_idx, "int32", "col_idx")
    _check_dtype(sources, "int32", "sources")
    _check_dtype(bc_out, "float64", "bc_out")
    n = _count(row_ptr) - 1 if n is None else n
    nnz = _count(col_idx) if nnz is None else nnz
    _check(lib.sp_bc_noalloc(_ptr(row_ptr), _ptr(col_idx), n, nnz, _ptr(sources), _count(sources), _ptr(bc_out),
                             _stream(stream)), "sp_bc_noalloc")


def sp_server_create(hbm_budget_bytes: int, max_slots: int) -> int:
    h = ctypes.c_void_p()
    _check(lib.sp_server_create(hbm_budget_bytes, max_slots, ctypes.byref(h)), "sp_server_create")
    return h.value


def sp_server_set_live(s: int, on: bool) -> None:
    _check(lib.sp_server_set_live(s, 1 if on else 0), "sp_server_set_live")


def sp_server_add_graph(s: int, g: int) -> int:
    gid = ctypes.c_int32()
    _check(lib.sp_server_add_graph(s, g, ctypes.byref(gid)), "sp_server_add_graph")
    return gid.value


def sp_bc_submit(s: int, graph_id: int, sources, bc_out, opts: sp_bc_opts | None = None) -> int:
    _check_dtype(sources, "int32", "sources")
    _check_dtype(bc_out, "float64", "bc_out")
    req = ctypes.c_int64()
    _check(lib.sp_bc_submit(s, graph_id, _ptr(sources), _count(sources),
                            ctypes.byref(opts) if opts is not None else None, _ptr(bc_out), ctypes.byref(req)),
           "sp_bc_submit")
    return req.value


def sp_pagerank_submit(s: int, graph_id: int, pr_out, damping: float = 0.85, tol: float = 1e-10,
                       max_iter: int = 100) -> int:
    _check_dtype(pr_out, "float64", "pr_out")
    req = ctypes.c_int64()
    _check(lib.sp_pagerank_submit(s, graph_id, float(damping), float(tol), int(max_iter), _ptr(pr_out),
                                  ctypes.byref(req)), "sp_pagerank_submit")
    return req.value


def sp_request_pagerank(s: int, req: int):
    """(status, iterations, last change) of a PageRank request; status SP_NOT_READY while it runs."""
    it, ch = ctypes.c_int32(), ctypes.c_double()
    rc = lib.sp_request_pagerank(s, req, ctypes.byref(it), ctypes.byref(ch))
    if rc not in (SP_OK, SP_NOT_READY):
        _check(rc, "sp_request_pagerank")
    return rc, it.value, ch.value


def sp_bc_poll(s: int, req: int) -> int:
    rc = lib.sp_bc_poll(s, req)
    if rc not in (SP_OK, SP_NOT_READY):
        _check(rc, "sp_bc_poll")
    return rc


def sp_bc_wait(s: int, req: int, timeout_ns: int = -1) -> int:
    rc = lib.sp_bc_wait(s, req, timeout_ns)
    if rc not in (SP_OK, SP_NOT_READY):
        _check(rc, "sp_bc_wait")
    return rc


def sp_bc_cancel(s: int, req: int) -> int:
    return lib.sp_bc_cancel(s, req)


def sp_request_times(s: int, req: int):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib.sp_request_times(s, req, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "sp_request_times")
    return a.value, b.value, c.value


def sp_request_stats(s: int, req: int) -> dict:
    st = sp_bc_stats()
    _check(lib.sp_request_stats(s, req, ctypes.byref(st)), "sp_request_stats")
    return st.as_dict()


def sp_server_destroy(s: int):
    _check(lib.sp_server_destroy(s), "sp_server_destroy")


def sp_status_string(st: int) -> str:
    return lib.sp_status_string(st).decode()


def sp_last_error() -> str:
    return lib.sp_last_error().decode()


# ---------------------------------------------------------------------------
# Convenience wrapper owning a graph handle

class Graph:
    """A resident graph (owns the handle; destroyed with the object)."""

    def __init__(self, row_ptr, col_idx, flags: int = 0, stream=None):
        self.handle = sp_graph_create(row_ptr, col_idx, flags=flags, stream=stream)
        self.info = sp_graph_get_info(self.handle)
        self.n = self.info["n"]
        self.nnz = self.info["nnz"]

    @classmethod
    def from_edges(cls, src, dst, n: int, flags: int = 0, stream=None) -> "Graph":
        """Symmetric, deduplicated graph built on the GPU from an edge list."""
        self = cls.__new__(cls)
        self.handle = sp_graph_from_edges(src, dst, n, flags, stream)
        self.info = sp_graph_get_info(self.handle)
        self.n = self.info["n"]
        self.nnz = self.info["nnz"]
        return self

    def csr(self):
        """The resident CSR as numpy arrays (row_ptr, col_idx)."""
        rp = np.empty(self.n + 1, np.int32)
        ci = np.empty(max(self.nnz, 1), np.int32)
        sp_graph_get_csr(self.handle, rp, ci)
        return rp, ci[: self.nnz]

    def close(self):
        if getattr(self, "handle", None):
            sp_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
