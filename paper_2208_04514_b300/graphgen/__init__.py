"""Seeded synthetic graphs shaped like the paper's workloads (Sec. 4.1).

Input side only: this module draws graphs and sources and holds none of the
shortest-path arithmetic.  Both the CPU oracle and the CUDA path are fed from
it.  Every graph is a CSR pair ``(row_ptr int32[n+1], col_idx int32[m])`` with
sorted rows, no duplicate arcs and no self-loops.

Workloads (seeds fixed so that every run sees the same graphs):

====================  ===========================================================
``er_1024``           directed Erdos-Renyi, n = 1024, Poisson(8) out-degrees, seed 1
``rmat(20)``          RMAT scale 20, edge factor 16, (.57,.19,.19,.05), permuted,
                      symmetrised, seed 2
``lattice(4096)``     4096 x 4096 4-neighbour lattice, bonds deleted with p = 0.1, seed 3
``rmat(16, seed=4)``  RMAT scale 16 for the batched all-sources workload
``arc_weights``       integer arc weights for the weighted extension, uniform on
                      [lo, hi] (default [1, 255], seed 7), symmetric per edge
====================  ===========================================================
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from .. import _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build_graphgen()
        lib = ctypes.CDLL(str(path))
        vp, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        lib.gg_er.restype = vp
        lib.gg_er.argtypes = [i32, f64, u64]
        lib.gg_rmat.restype = vp
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int, f64, f64, f64, u64, ctypes.c_int]
        lib.gg_lattice.restype = vp
        lib.gg_lattice.argtypes = [i32, i32, f64, u64]
        lib.gg_n.restype = i32
        lib.gg_n.argtypes = [vp]
        lib.gg_m.restype = i64
        lib.gg_m.argtypes = [vp]
        lib.gg_copy.restype = None
        lib.gg_copy.argtypes = [vp, vp, vp]
        lib.gg_free.restype = None
        lib.gg_free.argtypes = [vp]
        lib.gg_sample_sources.restype = i32
        lib.gg_sample_sources.argtypes = [vp, i32, i32, u64, vp]
        lib.gg_uniform_vertices.restype = None
        lib.gg_uniform_vertices.argtypes = [i32, i32, u64, vp]
        lib.gg_splitmix64_first.restype = u64
        lib.gg_splitmix64_first.argtypes = [u64]
        lib.gg_xoshiro_stream.restype = None
        lib.gg_xoshiro_stream.argtypes = [u64, i64, vp]
        lib.gg_arc_weights.restype = None
        lib.gg_arc_weights.argtypes = [vp, vp, i32, i32, i32, u64, ctypes.c_int, vp]
        _lib = lib
    return _lib


@dataclass
class Graph:
    """A CSR graph on the host.  ``symmetric`` is True when every arc has its reverse."""

    name: str
    row_ptr: np.ndarray
    col_idx: np.ndarray
    symmetric: bool

    @property
    def n(self) -> int:
        return int(self.row_ptr.shape[0] - 1)

    @property
    def m(self) -> int:
        return int(self.col_idx.shape[0])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr)


def _take(handle, name: str, symmetric: bool) -> Graph:
    lib = _load()
    if not handle:
        raise MemoryError(f"graph generator failed for {name}")
    try:
        n = lib.gg_n(handle)
        m = lib.gg_m(handle)
        rp = np.empty(n + 1, dtype=np.int32)
        ci = np.empty(max(m, 0), dtype=np.int32)
        lib.gg_copy(handle, rp.ctypes.data, ci.ctypes.data if m > 0 else None)
    finally:
        lib.gg_free(handle)
    return Graph(name, rp, ci, symmetric)


def erdos_renyi(n: int = 1024, lam: float = 8.0, seed: int = 1) -> Graph:
    """Directed ER: Poisson(lam) out-degree per vertex, uniform targets."""
    return _take(_load().gg_er(n, lam, seed), f"er_n{n}_l{lam:g}_s{seed}", False)


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 2, symmetrise: bool = True) -> Graph:
    """Graph500-style RMAT, vertex ids permuted; symmetrised by default."""
    h = _load().gg_rmat(scale, edge_factor, a, b, c, seed, 1 if symmetrise else 0)
    return _take(h, f"rmat{scale}_ef{edge_factor}_s{seed}", symmetrise)


def lattice(rows: int, cols: int | None = None, p_delete: float = 0.1, seed: int = 3) -> Graph:
    """rows x cols 4-neighbour lattice with independent bond deletion (both arcs per bond)."""
    cols = rows if cols is None else cols
    h = _load().gg_lattice(rows, cols, p_delete, seed)
    return _take(h, f"lattice{rows}x{cols}_p{p_delete:g}_s{seed}", True)


def sample_sources(g: Graph, k: int, seed: int) -> np.ndarray:
    """k distinct sources drawn uniformly from vertices with out-degree >= 1."""
    out = np.empty(k, dtype=np.int32)
    got = _load().gg_sample_sources(g.row_ptr.ctypes.data, g.n, k, seed, out.ctypes.data)
    if got < 0:
        raise MemoryError("sample_sources")
    return out[:got].copy()


def uniform_vertices(n: int, k: int, seed: int) -> np.ndarray:
    """k vertices uniform on [0, n), repeats allowed (isolated vertices included)."""
    out = np.empty(k, dtype=np.int32)
    _load().gg_uniform_vertices(n, k, seed, out.ctypes.data)
    return out


def splitmix64_first(seed: int) -> int:
    return int(_load().gg_splitmix64_first(seed))


def xoshiro_stream(seed: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _load().gg_xoshiro_stream(seed, count, out.ctypes.data)
    return out


def arc_weights(g: Graph, lo: int = 1, hi: int = 255, seed: int = 7) -> np.ndarray:
    """int32 weight per arc (aligned with ``col_idx``), uniform on [lo, hi] from a
    hash of the arc's endpoints and ``seed``; both arcs of an undirected edge get
    the same weight when ``g.symmetric``."""
    if not (0 <= lo <= hi <= 2**31 - 1):
        raise ValueError("need 0 <= lo <= hi <= 2^31 - 1")
    out = np.empty(max(g.m, 1), dtype=np.int32)
    _load().gg_arc_weights(g.row_ptr.ctypes.data, np.ascontiguousarray(g.col_idx, dtype=np.int32).ctypes.data
                           if g.m else None, g.n, lo, hi, seed, 1 if g.symmetric else 0, out.ctypes.data)
    return out[:g.m].copy()


def from_arcs(n: int, src, dst, name: str = "arcs", symmetric: bool = False) -> Graph:
    """CSR from an explicit arc list (small hand-built test graphs).

    Self-loops and duplicate arcs are kept exactly as given, so that tests can
    check that both are tolerated; rows are sorted.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    order = np.lexsort((dst, src))
    src, dst = src[order], dst[order]
    rp = np.zeros(n + 1, dtype=np.int32)
    np.add.at(rp, src + 1, 1)
    rp = np.cumsum(rp).astype(np.int32)
    return Graph(name, rp, dst.astype(np.int32), symmetric)


def transpose(g: Graph) -> Graph:
    """In-adjacency (CSC of the same matrix) as a CSR of the reversed graph."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.out_degree())
    return from_arcs(g.n, g.col_idx.astype(np.int64), src, g.name + "_T", g.symmetric)


def stats(g: Graph) -> dict:
    deg = g.out_degree()
    indeg = np.bincount(g.col_idx, minlength=g.n) if g.m else np.zeros(g.n, dtype=np.int64)
    return {
        "n": g.n,
        "m": g.m,
        "isolated": int(np.count_nonzero((deg == 0) & (indeg == 0))),
        "max_out_degree": int(deg.max()) if g.n else 0,
        "avg_out_degree": float(g.m / g.n) if g.n else 0.0,
    }
