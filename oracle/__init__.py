"""CPU oracle for DAWN (ICS '24) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA path
(``paper_2208_04514_b300``): the C source ``dawn_oracle.c`` is compiled on its
own with gcc, and this module only marshals numpy arrays into it.

What each function follows (the C file carries the same notes):

* ``sssp_sovm``     -- Alg. 3 (SOVM, Eq. 5-7), dense alpha/beta, push over CSR.
* ``sssp_bovm``     -- Alg. 1 (BOVM, Eq. 2-4), pull over CSC, first-hit exit,
                       alpha/beta merged after the vertex loop.
* ``bfs_queue``     -- Alg. 2 (General BFS), FIFO queue.
* ``apsp_floyd``    -- Floyd-Warshall brute force (pin, small n).
* ``apsp_powers``   -- Thm 1 / Lemma 1 with Boolean matrix powers (pin, small n).
* ``certificate``   -- O(n+m) exactness certificate for one distance vector.
* ``wcc``           -- weakly connected component labels.
* ``msbfs``         -- APSP-style batch: SOVM per source + ecc / sum / reached.
* ``wsssp_minplus`` -- weighted extension (Sec. 5, (min, +) future work): the
                       SOVM rounds of Alg. 3 over (min, +), non-negative int32
                       weights, int64 distances.
* ``dijkstra``      -- textbook Dijkstra (binary heap), pin for the above.
* ``wcertificate``  -- O(n+m) exactness certificate for weighted distances.

Every function is pinned by ``tests/test_oracle_pins.py`` to closed forms,
brute force, a library routine (scipy) and invariants; none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_DIR = Path(__file__).resolve().parent
_SRC = _DIR / "dawn_oracle.c"
_SO = _DIR / "_lib" / "libdawn_oracle.so"
_lib = None
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared"]


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (no GPU, no CUDA)."""
    if force or not _SO.exists() or _SO.stat().st_mtime < _SRC.stat().st_mtime:
        _SO.parent.mkdir(parents=True, exist_ok=True)
        tmp = _SO.with_suffix(".so.tmp")
        cmd = ["gcc", *CFLAGS, "-o", str(tmp), str(_SRC)]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"oracle build failed:\n{res.stderr}")
        tmp.replace(_SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        # DAWN_ORACLE_SO lets the mutation test point the pin suite at a copy of
        # the oracle with a planted mistake.
        override = os.environ.get("DAWN_ORACLE_SO")
        lib = ctypes.CDLL(override if override else str(build()))
        i32, i64, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        sig = {
            "oracle_sssp_sovm": [i32, vp, vp, i32, vp, vp, vp],
            "oracle_sssp_bovm": [i32, vp, vp, i32, vp, vp],
            "oracle_bfs_queue": [i32, vp, vp, i32, vp],
            "oracle_apsp_floyd": [i32, vp, vp, vp],
            "oracle_apsp_powers": [i32, vp, vp, vp],
            "oracle_certificate": [i32, vp, vp, i32, vp, vp],
            "oracle_wcc": [i32, vp, vp, vp],
            "oracle_msbfs": [i32, vp, vp, vp, i32, vp, vp, vp, vp],
            "oracle_parents": [i32, vp, vp, vp, vp],
            "oracle_centrality": [i32, vp, vp, vp, i32, vp, vp, vp, vp, vp, vp],
            "oracle_wsssp_minplus": [i32, vp, vp, vp, i32, vp, vp, vp],
            "oracle_dijkstra": [i32, vp, vp, vp, i32, vp],
            "oracle_wcertificate": [i32, vp, vp, vp, i32, vp, vp],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _csr(row_ptr, col_idx):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    if ci.size == 0:
        ci = np.zeros(1, dtype=np.int32)  # valid pointer for m = 0
    return rp, ci


def _p(a):
    return a.ctypes.data


def sssp_sovm(row_ptr, col_idx, src: int, with_stats: bool = False):
    """Alg. 3.  Returns dist (int32[n], -1 = unreachable) [, edge_visits, levels]."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    dist = np.empty(n, dtype=np.int32)
    visits = ctypes.c_int64(0)
    levels = ctypes.c_int32(0)
    rc = _load().oracle_sssp_sovm(n, _p(rp), _p(ci), int(src), _p(dist),
                                  ctypes.addressof(visits), ctypes.addressof(levels))
    if rc != 0:
        raise ValueError("oracle_sssp_sovm: bad input")
    return (dist, visits.value, levels.value) if with_stats else dist


def sssp_bovm(csc_ptr, csc_row, src: int, with_levels: bool = False):
    """Alg. 1 on the in-adjacency (CSC).  Returns dist [, levels]."""
    cp, cr = _csr(csc_ptr, csc_row)
    n = cp.size - 1
    dist = np.empty(n, dtype=np.int32)
    levels = ctypes.c_int32(0)
    rc = _load().oracle_sssp_bovm(n, _p(cp), _p(cr), int(src), _p(dist), ctypes.addressof(levels))
    if rc != 0:
        raise ValueError("oracle_sssp_bovm: bad input")
    return (dist, levels.value) if with_levels else dist


def bfs_queue(row_ptr, col_idx, src: int):
    """Alg. 2 (FIFO BFS)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    dist = np.empty(n, dtype=np.int32)
    if _load().oracle_bfs_queue(n, _p(rp), _p(ci), int(src), _p(dist)) != 0:
        raise ValueError("oracle_bfs_queue: bad input")
    return dist


def apsp_floyd(row_ptr, col_idx):
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    d = np.empty((n, n), dtype=np.int32)
    if _load().oracle_apsp_floyd(n, _p(rp), _p(ci), _p(d)) != 0:
        raise ValueError("oracle_apsp_floyd: n out of range")
    return d


def apsp_powers(row_ptr, col_idx):
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    d = np.empty((n, n), dtype=np.int32)
    if _load().oracle_apsp_powers(n, _p(rp), _p(ci), _p(d)) != 0:
        raise ValueError("oracle_apsp_powers: n out of range")
    return d


def certificate(row_ptr, col_idx, src: int, dist) -> tuple[int, int]:
    """(0, -1) when dist is exact; else (failed item 1/2/3, offending vertex)."""
    rp, ci = _csr(row_ptr, col_idx)
    d = np.ascontiguousarray(dist, dtype=np.int32)
    bad = ctypes.c_int32(-1)
    rc = _load().oracle_certificate(rp.size - 1, _p(rp), _p(ci), int(src), _p(d), ctypes.addressof(bad))
    return rc, bad.value


def wcc(row_ptr, col_idx):
    rp, ci = _csr(row_ptr, col_idx)
    lab = np.empty(rp.size - 1, dtype=np.int32)
    if _load().oracle_wcc(rp.size - 1, _p(rp), _p(ci), _p(lab)) != 0:
        raise MemoryError("oracle_wcc")
    return lab


def parents(row_ptr, col_idx, dist):
    """Smallest-id shortest-path tree for the exact distances `dist` (Fact 1)."""
    rp, ci = _csr(row_ptr, col_idx)
    d = np.ascontiguousarray(dist, dtype=np.int32)
    par = np.empty(rp.size - 1, dtype=np.int32)
    if _load().oracle_parents(rp.size - 1, _p(rp), _p(ci), _p(d), _p(par)) != 0:
        raise ValueError("oracle_parents: bad input")
    return par


def centrality(row_ptr, col_idx, sources):
    """Per source ecc, dsum, reached, closeness, harmonic; whole-run summary
    {diameter, radius, pairs, dist_total}."""
    rp, ci = _csr(row_ptr, col_idx)
    src = np.ascontiguousarray(sources, dtype=np.int32)
    k = src.size
    out = {"ecc": np.empty(k, dtype=np.int32), "dsum": np.empty(k, dtype=np.int64),
           "reached": np.empty(k, dtype=np.int32), "closeness": np.empty(k, dtype=np.float64),
           "harmonic": np.empty(k, dtype=np.float64)}
    summ = np.empty(4, dtype=np.int64)
    rc = _load().oracle_centrality(rp.size - 1, _p(rp), _p(ci), _p(src), k, _p(out["ecc"]), _p(out["dsum"]),
                                   _p(out["reached"]), _p(out["closeness"]), _p(out["harmonic"]), _p(summ))
    if rc != 0:
        raise ValueError("oracle_centrality: bad input")
    out["summary"] = dict(zip(("diameter", "radius", "pairs", "dist_total"), (int(x) for x in summ)))
    return out


def msbfs(row_ptr, col_idx, sources, keep_dist: bool = True):
    """SOVM per source.  Returns (dist_block [k,n] or None, ecc, dsum, reached)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    src = np.ascontiguousarray(sources, dtype=np.int32)
    k = src.size
    block = np.empty((k, n), dtype=np.int32) if keep_dist else None
    ecc = np.empty(k, dtype=np.int32)
    dsum = np.empty(k, dtype=np.int64)
    reached = np.empty(k, dtype=np.int32)
    rc = _load().oracle_msbfs(n, _p(rp), _p(ci), _p(src), k,
                              _p(block) if keep_dist else None, _p(ecc), _p(dsum), _p(reached))
    if rc != 0:
        raise ValueError("oracle_msbfs: bad input")
    return block, ecc, dsum, reached


def _w(weights, m):
    w = np.ascontiguousarray(weights, dtype=np.int32)
    if w.size != m:
        raise ValueError(f"need {m} weights, got {w.size}")
    return w if w.size else np.zeros(1, dtype=np.int32)


def wsssp_minplus(row_ptr, col_idx, weights, src: int, with_stats: bool = False):
    """(min, +) SOVM rounds.  Returns dist (int64[n], -1 = no path) [, rounds, arcs offered]."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    w = _w(weights, int(rp[-1]))
    dist = np.empty(n, dtype=np.int64)
    rounds = ctypes.c_int32(0)
    relax = ctypes.c_int64(0)
    rc = _load().oracle_wsssp_minplus(n, _p(rp), _p(ci), _p(w), int(src), _p(dist),
                                      ctypes.addressof(rounds), ctypes.addressof(relax))
    if rc != 0:
        raise ValueError(f"oracle_wsssp_minplus failed ({rc})")
    return (dist, rounds.value, relax.value) if with_stats else dist


def dijkstra(row_ptr, col_idx, weights, src: int):
    """Textbook Dijkstra.  Returns dist (int64[n], -1 = no path)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    w = _w(weights, int(rp[-1]))
    dist = np.empty(n, dtype=np.int64)
    if _load().oracle_dijkstra(n, _p(rp), _p(ci), _p(w), int(src), _p(dist)) != 0:
        raise ValueError("oracle_dijkstra failed")
    return dist


def wcertificate(row_ptr, col_idx, weights, src: int, dist) -> tuple[int, int]:
    """(1, -1) when dist is the exact weighted distance vector from src, else (0, bad vertex)."""
    rp, ci = _csr(row_ptr, col_idx)
    n = rp.size - 1
    w = _w(weights, int(rp[-1]))
    d = np.ascontiguousarray(dist, dtype=np.int64)
    bad = ctypes.c_int32(-1)
    ok = _load().oracle_wcertificate(n, _p(rp), _p(ci), _p(w), int(src), _p(d), ctypes.addressof(bad))
    return int(ok), int(bad.value)
