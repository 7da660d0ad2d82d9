"""Thin Python binding of the C ABI in ``include/dawn.h`` (libdawn.so).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  Functions keep the C names.  Arrays may be numpy arrays (host) or
torch tensors (host or CUDA); the library tells host from device pointers
itself.  ``stream`` defaults to torch's current CUDA stream.  A non-zero
status raises :class:`DawnError`.  There is no CPU fallback: if the library
cannot be built or loaded, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import re
from pathlib import Path

import numpy as np

from . import _build

DAWN_OK = 0
DAWN_E_INVALID = 1
DAWN_E_NOMEM = 2
DAWN_E_OVERFLOW = 3
DAWN_E_TIMEOUT = 4
DAWN_E_CUDA = 5
DAWN_E_STATE = 6

DAWN_DIRECTED = 0
DAWN_SYMMETRIC = 1

DAWN_MODE_AUTO = 0
DAWN_MODE_PUSH = 1
DAWN_MODE_PULL = 2

DAWN_SOURCE_MAJOR = 0
DAWN_VERTEX_MAJOR = 1

DAWN_MSBFS_SLICED = 1
DAWN_MSBFS_PER_LEVEL = 2

DAWN_REQ_PENDING = 0
DAWN_REQ_RUNNING = 1
DAWN_REQ_DONE = 2
DAWN_REQ_FAILED = 3

DAWN_ENGINE_AUTO = 0
DAWN_ENGINE_GRID = 1
DAWN_ENGINE_CLUSTER = 2

DAWN_SERVE_AUTO = 0
DAWN_SERVE_DENSE = 1
DAWN_SERVE_FRONTIER = 2

_NAMES = {1: "DAWN_E_INVALID", 2: "DAWN_E_NOMEM", 3: "DAWN_E_OVERFLOW", 4: "DAWN_E_TIMEOUT",
          5: "DAWN_E_CUDA", 6: "DAWN_E_STATE"}


class DawnError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{_NAMES.get(code, code)}: {message}")
        self.code = code


class dawn_sssp_opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("alpha", ctypes.c_int32), ("beta", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("spin_limit", ctypes.c_int64),
                ("trace", ctypes.c_void_p), ("trace_cap", ctypes.c_int32), ("pull_serial", ctypes.c_int32),
                ("engine", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class dawn_sssp_stats(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("push_steps", ctypes.c_int32), ("pull_steps", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("reached", ctypes.c_int64), ("edges", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class dawn_tuning(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_int32), ("beta", ctypes.c_int32), ("pull_serial", ctypes.c_int32),
                ("lanes", ctypes.c_int32), ("sssp_us", ctypes.c_double), ("msbfs_sources_per_s", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class dawn_msbfs_opts(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("trace_cap", ctypes.c_int32), ("spin_limit", ctypes.c_int64),
                ("trace", ctypes.c_void_p), ("kernel", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class dawn_wsssp_stats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("reserved", ctypes.c_int32), ("reached", ctypes.c_int64),
                ("relaxations", ctypes.c_int64), ("improvements", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class dawn_apsp_summary(ctypes.Structure):
    _fields_ = [("diameter", ctypes.c_int32), ("radius", ctypes.c_int32), ("pairs", ctypes.c_int64),
                ("dist_total", ctypes.c_int64)]


_lib = None
_vp, _i32, _i64, _u32, _u64, _sz = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                    ctypes.c_uint64, ctypes.c_size_t)

_SIGNATURES = {
    "dawn_graph_upload": [_vp, _vp, _i32, _i64, _u32, _vp, ctypes.POINTER(_vp)],
    "dawn_graph_free": [_vp],
    "dawn_graph_info": [_vp, _vp, _vp, _vp],
    "dawn_graph_sync": [_vp, _vp],
    "dawn_sssp": [_vp, _i32, _vp, _vp],
    "dawn_sssp_ex": [_vp, _i32, _vp, _vp, _vp, _vp],
    "dawn_sssp_async": [_vp, _i32, _vp, _vp, _vp, _vp],
    "dawn_sssp_noalloc": [_vp, _vp, _i32, _i64, _i32, _vp, _vp],
    "dawn_sssp_many": [_vp, _vp, _i32, _vp, _vp, _vp, _vp],
    "dawn_sssp_tree": [_vp, _i32, _vp, _vp, _vp],
    "dawn_sssp_tree_async": [_vp, _i32, _vp, _vp, _vp],
    "dawn_msbfs": [_vp, _vp, _i32, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp],
    "dawn_msbfs_ex": [_vp, _vp, _i32, _vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp],
    "dawn_centrality": [_vp, _vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "dawn_autotune": [_vp, _vp, _i32, _vp, _vp],
    "dawn_set_tuning": [_vp, _vp],
    "dawn_serve_create": [_vp, ctypes.c_int, _sz, ctypes.c_int, ctypes.POINTER(_vp)],
    "dawn_serve_create_ex": [_vp, ctypes.c_int, _sz, ctypes.c_int, _vp, ctypes.POINTER(_vp)],
    "dawn_serve_submit": [_vp, ctypes.c_int, _vp, _i32, ctypes.c_int, _vp, ctypes.POINTER(_u64)],
    "dawn_serve_poll": [_vp, _u64, ctypes.POINTER(ctypes.c_int)],
    "dawn_serve_times": [_vp, _u64, _vp, _vp],
    "dawn_serve_drain": [_vp, _i64],
    "dawn_serve_destroy": [_vp],
    "dawn_l2_read_gbs": [_i64, _i32, _vp, _vp],
    "dawn_graph_set_weights": [_vp, _vp, _vp],
    "dawn_wsssp": [_vp, _i32, _vp, _vp, _vp],
    "dawn_wsssp_async": [_vp, _i32, _vp, _vp, _vp],
    "dawn_last_error": [],
    "dawn_version": [],
}


def load(path: str | Path | None = None) -> ctypes.CDLL:
    """Load libdawn.so (building it in-tree with nvcc when missing or stale)."""
    global _lib
    if _lib is None:
        so = Path(path) if path else _build.build_dawn()
        lib = ctypes.CDLL(str(so))
        for name, args in _SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name == "dawn_last_error" else ctypes.c_int
        _lib = lib
    return _lib


def header_entry_points() -> list[str]:
    """Names of every entry point declared in include/dawn.h."""
    text = (_build.INCLUDE / "dawn.h").read_text()
    return re.findall(r"DAWN_API\s+[\w\s\*]+?\b(dawn_\w+)\s*\(", text)


def _check(rc: int) -> None:
    if rc != DAWN_OK:
        raise DawnError(rc, load().dawn_last_error().decode())


def _ptr(a) -> int | None:
    """Address of a numpy array or torch tensor (contiguous), None for None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _opts(opts: dict | None, cls):
    if opts is None:
        return None
    o = cls()
    for k, v in opts.items():
        setattr(o, k, v)
    return o


# --------------------------------------------------------------- graphs --

def dawn_graph_upload(row_ptr, col_idx, n: int | None = None, m: int | None = None,
                      flags: int = DAWN_DIRECTED, stream=None) -> int:
    """Upload a CSR (numpy or torch int32) and return the graph handle."""
    n = int(row_ptr.shape[0] - 1) if n is None else n
    m = int(col_idx.shape[0]) if m is None else m
    h = _vp()
    _check(load().dawn_graph_upload(_ptr(row_ptr), _ptr(col_idx) if m > 0 else None, n, m, flags,
                                    _stream(stream), ctypes.byref(h)))
    return h.value


def dawn_graph_free(g: int) -> None:
    _check(load().dawn_graph_free(g))


def dawn_graph_info(g: int) -> tuple[int, int, int]:
    n, m, f = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_uint32()
    _check(load().dawn_graph_info(g, ctypes.byref(n), ctypes.byref(m), ctypes.byref(f)))
    return n.value, m.value, f.value


def dawn_graph_sync(g: int, stream=None) -> None:
    _check(load().dawn_graph_sync(g, _stream(stream)))


# --------------------------------------------------------- single source --

def dawn_sssp(g: int, src: int, dist, stream=None) -> None:
    """Fill dist (int32[n], host or device) with distances from src."""
    _check(load().dawn_sssp(g, int(src), _ptr(dist), _stream(stream)))


def dawn_sssp_ex(g: int, src: int, dist, opts: dict | None = None, stream=None) -> dict:
    """dawn_sssp with options; returns the call's statistics."""
    st = dawn_sssp_stats()
    o = _opts(opts, dawn_sssp_opts)
    _check(load().dawn_sssp_ex(g, int(src), _ptr(dist), ctypes.byref(o) if o else None,
                               ctypes.byref(st), _stream(stream)))
    return st.as_dict()


def dawn_sssp_many(g: int, sources, k: int | None = None, dist=None, stats=None, opts: dict | None = None,
                   stream=None) -> None:
    """k sources, one distance row each (dist: host or device, k x n int32)."""
    k = int(sources.shape[0]) if k is None else k
    o = _opts(opts, dawn_sssp_opts)
    _check(load().dawn_sssp_many(g, _ptr(sources), k, _ptr(dist), _ptr(stats), ctypes.byref(o) if o else None,
                                 _stream(stream)))


def dawn_graph_set_weights(g: int, weights, stream=None) -> None:
    """Attach non-negative int32 arc weights (aligned with the uploaded col_idx)."""
    _check(load().dawn_graph_set_weights(g, _ptr(weights), _stream(stream)))


def dawn_wsssp(g: int, src: int, dist, stream=None) -> dict:
    """Weighted SSSP ((min, +) rounds) into int64 dist; returns the call's statistics."""
    st = dawn_wsssp_stats()
    _check(load().dawn_wsssp(g, int(src), _ptr(dist), ctypes.byref(st), _stream(stream)))
    return st.as_dict()


def dawn_wsssp_async(g: int, src: int, dist_dev, stats_dev=None, stream=None) -> None:
    """Stream-ordered dawn_wsssp (device int64 dist, device stats or None)."""
    _check(load().dawn_wsssp_async(g, int(src), _ptr(dist_dev), _ptr(stats_dev), _stream(stream)))


def dawn_sssp_tree(g: int, src: int, dist, parent, stream=None) -> None:
    """Distances and the min-id shortest-path tree (host or device int32[n] each)."""
    _check(load().dawn_sssp_tree(g, int(src), _ptr(dist), _ptr(parent), _stream(stream)))


def dawn_sssp_tree_async(g: int, src: int, dist_dev, parent_dev, stream=None) -> None:
    """Enqueue dawn_sssp_tree on the stream (device outputs, no synchronization)."""
    _check(load().dawn_sssp_tree_async(g, int(src), _ptr(dist_dev), _ptr(parent_dev), _stream(stream)))


def dawn_sssp_async(g: int, src: int, dist_dev, opts: dict | None = None, stats_dev=None, stream=None) -> None:
    """Enqueue one source without synchronizing (dist_dev, stats_dev on the device)."""
    o = _opts(opts, dawn_sssp_opts)
    _check(load().dawn_sssp_async(g, int(src), _ptr(dist_dev), ctypes.byref(o) if o else None,
                                  _ptr(stats_dev), _stream(stream)))


def dawn_sssp_noalloc(row_ptr_dev, col_idx_dev, src: int, dist_dev, n: int | None = None,
                      m: int | None = None, stream=None) -> None:
    """Allocation-free single source on a device-resident CSR (see include/dawn.h)."""
    n = int(row_ptr_dev.shape[0] - 1) if n is None else n
    m = int(col_idx_dev.shape[0]) if m is None else m
    _check(load().dawn_sssp_noalloc(_ptr(row_ptr_dev), _ptr(col_idx_dev), n, m, int(src),
                                    _ptr(dist_dev), _stream(stream)))


STATS_WORDS = ctypes.sizeof(dawn_sssp_stats) // 8  # int64 words per stats record
WSTATS_WORDS = ctypes.sizeof(dawn_wsssp_stats) // 8  # int64 words per weighted stats record


def wstats_from_words(words) -> dict:
    """dawn_wsssp_stats from WSTATS_WORDS int64 words (a device stats row copied back)."""
    raw = np.ascontiguousarray(words, dtype=np.int64).tobytes()
    return dawn_wsssp_stats.from_buffer_copy(raw).as_dict()


def stats_from_words(words) -> dict:
    """Decode one dawn_sssp_stats record read back as int64 words."""
    raw = np.ascontiguousarray(np.asarray(words, dtype=np.int64)).tobytes()
    return dawn_sssp_stats.from_buffer_copy(raw).as_dict()


# ---------------------------------------------------------- multi source --

def dawn_msbfs(g: int, sources, k: int | None = None, dist_block=None, dist_bytes: int = 2,
               layout: int = DAWN_SOURCE_MAJOR, ecc=None, dsum=None, stream=None) -> None:
    k = int(sources.shape[0]) if k is None else k
    _check(load().dawn_msbfs(g, _ptr(sources), k, _ptr(dist_block), dist_bytes, layout,
                             _ptr(ecc), _ptr(dsum), _stream(stream)))


def dawn_msbfs_ex(g: int, sources, k: int | None = None, dist_block=None, dist_bytes: int = 2,
                  layout: int = DAWN_SOURCE_MAJOR, ecc=None, dsum=None, reached=None,
                  opts: dict | None = None, stream=None) -> None:
    k = int(sources.shape[0]) if k is None else k
    o = _opts(opts, dawn_msbfs_opts)
    _check(load().dawn_msbfs_ex(g, _ptr(sources), k, _ptr(dist_block), dist_bytes, layout,
                                _ptr(ecc), _ptr(dsum), _ptr(reached), ctypes.byref(o) if o else None,
                                _stream(stream)))


def dawn_centrality(g: int, sources, k: int | None = None, ecc=None, dsum=None, reached=None, closeness=None,
                    harmonic=None, opts: dict | None = None, stream=None) -> dict:
    """Batched level loop without distance rows; fills the given per-source
    arrays (host or device) and returns the whole-run summary."""
    k = int(sources.shape[0]) if k is None else k
    o = _opts(opts, dawn_msbfs_opts)
    summ = dawn_apsp_summary()
    _check(load().dawn_centrality(g, _ptr(sources), k, _ptr(ecc), _ptr(dsum), _ptr(reached), _ptr(closeness),
                                  _ptr(harmonic), ctypes.byref(summ), ctypes.byref(o) if o else None,
                                  _stream(stream)))
    return {f: getattr(summ, f) for f, _ in summ._fields_}


def dawn_l2_read_gbs(nbytes: int = 64 << 20, passes: int = 50, stream=None) -> float:
    """This GPU's L2 read bandwidth (GB/s) from an L2-resident buffer."""
    out = ctypes.c_double(0.0)
    _check(load().dawn_l2_read_gbs(nbytes, passes, ctypes.byref(out), _stream(stream)))
    return out.value


# -------------------------------------------------------------- autotune --

def dawn_autotune(g: int, sample, k: int | None = None, stream=None) -> dict:
    """Time short trials on g and keep the fastest settings in g; returns them."""
    k = int(sample.shape[0]) if k is None else k
    t = dawn_tuning()
    _check(load().dawn_autotune(g, _ptr(sample), k, ctypes.byref(t), _stream(stream)))
    return t.as_dict()


def dawn_set_tuning(g: int, tuning: dict) -> None:
    t = dawn_tuning()
    for f, _ in dawn_tuning._fields_:
        setattr(t, f, tuning.get(f, 0))
    _check(load().dawn_set_tuning(g, ctypes.byref(t)))


# --------------------------------------------------------------- serving --

def dawn_serve_create(graphs: list[int], mem_budget_bytes: int = 0, max_lanes: int = 256) -> int:
    arr = (_vp * len(graphs))(*graphs)
    h = _vp()
    _check(load().dawn_serve_create(arr, len(graphs), mem_budget_bytes, max_lanes, ctypes.byref(h)))
    return h.value


def dawn_serve_create_ex(graphs: list[int], mem_budget_bytes: int = 0, max_lanes: int = 256,
                         modes: list[int] | None = None) -> int:
    """modes: one DAWN_SERVE_* per graph, or None for all DAWN_SERVE_AUTO."""
    arr = (_vp * len(graphs))(*graphs)
    marr = (_i32 * len(graphs))(*modes) if modes is not None else None
    h = _vp()
    _check(load().dawn_serve_create_ex(arr, len(graphs), mem_budget_bytes, max_lanes,
                                       ctypes.cast(marr, _vp) if marr is not None else None, ctypes.byref(h)))
    return h.value


def dawn_serve_submit(s: int, graph_idx: int, sources, k: int | None = None, dist_bytes: int = 2,
                      dist_out=None) -> int:
    k = int(sources.shape[0]) if k is None else k
    rid = _u64()
    _check(load().dawn_serve_submit(s, graph_idx, _ptr(sources), k, dist_bytes, _ptr(dist_out),
                                    ctypes.byref(rid)))
    return rid.value


def dawn_serve_poll(s: int, req_id: int) -> int:
    st = ctypes.c_int()
    _check(load().dawn_serve_poll(s, req_id, ctypes.byref(st)))
    return st.value


def dawn_serve_times(s: int, req_id: int) -> tuple[float, float]:
    """(submit, done) host steady-clock seconds of a request (done = 0 while open)."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().dawn_serve_times(s, req_id, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def dawn_serve_drain(s: int, timeout_ms: int = -1) -> None:
    _check(load().dawn_serve_drain(s, timeout_ms))


def dawn_serve_destroy(s: int) -> None:
    _check(load().dawn_serve_destroy(s))


def dawn_last_error() -> str:
    return load().dawn_last_error().decode()


def dawn_version() -> int:
    return load().dawn_version()
