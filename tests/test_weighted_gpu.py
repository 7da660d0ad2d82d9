"""Weighted extension parity: dawn_wsssp ((min, +) rounds of Alg. 3, through
the C ABI) against the CPU oracle's (min, +) iteration and its textbook
Dijkstra, element by element, bit-exact (int64 distances, -1 = no path).

Covers random digraphs with self-loops, repeated arcs and zero weights (every
source), the directed ER workload (n = 1024, sources 0-3), symmetric and
directed RMAT graphs (hub rows longer than one warp, spread over warps by the
arc split), a percolated lattice (hundreds of rounds), weights up to 2^31 - 1
(distances past int32), all-zero weights, isolated and single-vertex cases,
host and device outputs, the stream-ordered variant, the full-size RMAT
scale-20 graph with the weighted certificate on sampled sources, and bad
arguments (no weights, negative weights, a source out of range).
"""
import numpy as np
import pytest

import oracle
from paper_2208_04514_b300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def upload(dawn, g, w):
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx,
                               flags=dawn.DAWN_SYMMETRIC if g.symmetric else dawn.DAWN_DIRECTED)
    dawn.dawn_graph_set_weights(h, np.ascontiguousarray(w, dtype=np.int32))
    return h


def run_host(dawn, h, n, s):
    dist = np.full(n, 77, dtype=np.int64)
    st = dawn.dawn_wsssp(h, s, dist)
    return dist, st


def run_device(dawn, h, n, s):
    dist = torch.full((n,), 77, dtype=torch.int64, device="cuda")
    st = dawn.dawn_wsssp(h, s, dist)
    return dist.cpu().numpy(), st


def check(g, w, s, dist, st):
    want, rounds, _ = oracle.wsssp_minplus(g.row_ptr, g.col_idx, w, s, with_stats=True)
    np.testing.assert_array_equal(dist, want, err_msg=f"source {s}")
    assert st["reached"] == int((want >= 0).sum())
    # values lowered during a round are offered at once: never more rounds
    # than the synchronous iteration
    assert 0 <= st["rounds"] <= rounds
    assert st["improvements"] >= st["reached"] - 1


@pytest.mark.parametrize("seed", range(8))
def test_small_digraphs_every_source(dawn, seed):
    from test_oracle_pins import random_weighted
    g, w = random_weighted(5100 + seed, n=int(np.random.default_rng(seed).integers(1, 60)))
    h = upload(dawn, g, w)
    try:
        for s in range(g.n):
            d, st = run_host(dawn, h, g.n, s)
            check(g, w, s, d, st)
            np.testing.assert_array_equal(d, oracle.dijkstra(g.row_ptr, g.col_idx, w, s))
    finally:
        dawn.dawn_graph_free(h)


WORKLOADS = {
    "er1024": lambda: (gg.erdos_renyi(1024, 8.0, seed=1), (1, 100)),
    "rmat12": lambda: (gg.rmat(12, seed=2), (1, 255)),
    "rmat12_dir": lambda: (gg.rmat(12, seed=2, symmetrise=False), (0, 255)),
    "lattice64": lambda: (gg.lattice(64, 64, 0.1, seed=3), (1, 100)),
    "rmat14_zero_heavy": lambda: (gg.rmat(14, seed=8), (0, 2)),
}


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_workloads(dawn, name):
    g, (lo, hi) = WORKLOADS[name]()
    w = gg.arc_weights(g, lo, hi, seed=7)
    h = upload(dawn, g, w)
    try:
        sources = [0, 1, 2, 3] if name == "er1024" else list(gg.sample_sources(g, 4, seed=5))
        for s in sources:
            d, st = run_device(dawn, h, g.n, s)
            check(g, w, s, d, st)
    finally:
        dawn.dawn_graph_free(h)


def test_large_weights_and_zero_weights(dawn):
    g = gg.rmat(11, seed=2)
    for lo, hi in [(2**31 - 64, 2**31 - 1), (0, 0)]:
        w = gg.arc_weights(g, lo, hi, seed=11)
        h = upload(dawn, g, w)
        try:
            for s in gg.sample_sources(g, 3, seed=5):
                d, st = run_host(dawn, h, g.n, s)
                check(g, w, s, d, st)
                if hi == 0:
                    np.testing.assert_array_equal(d, np.where(oracle.sssp_sovm(g.row_ptr, g.col_idx, s) >= 0, 0, -1))
                else:
                    assert d.max() > 2**31
        finally:
            dawn.dawn_graph_free(h)


def test_unit_weights_match_unweighted(dawn):
    g = gg.rmat(13, seed=2)
    h = upload(dawn, g, np.ones(g.m, dtype=np.int32))
    try:
        for s in gg.sample_sources(g, 3, seed=9):
            d, _ = run_device(dawn, h, g.n, s)
            d32 = np.empty(g.n, dtype=np.int32)
            dawn.dawn_sssp(h, int(s), d32)
            np.testing.assert_array_equal(d, d32.astype(np.int64))
    finally:
        dawn.dawn_graph_free(h)


def test_isolated_single_and_edgeless(dawn):
    g = gg.from_arcs(5, [0, 1], [1, 2])
    h = upload(dawn, g, np.array([3, 4], dtype=np.int32))
    try:
        d, st = run_host(dawn, h, 5, 4)
        np.testing.assert_array_equal(d, [-1, -1, -1, -1, 0])
        assert st["rounds"] == 0 and st["reached"] == 1
        d, _ = run_host(dawn, h, 5, 0)
        np.testing.assert_array_equal(d, [0, 3, 7, -1, -1])
    finally:
        dawn.dawn_graph_free(h)
    one = gg.from_arcs(1, [0], [0])
    h = upload(dawn, one, np.array([9], dtype=np.int32))
    try:
        np.testing.assert_array_equal(run_host(dawn, h, 1, 0)[0], [0])
    finally:
        dawn.dawn_graph_free(h)
    empty = gg.from_arcs(3, [], [])
    h = upload(dawn, empty, np.zeros(0, dtype=np.int32))
    try:
        np.testing.assert_array_equal(run_host(dawn, h, 3, 1)[0], [-1, 0, -1])
    finally:
        dawn.dawn_graph_free(h)


def test_async_stream_ordered_many_sources(dawn):
    g = gg.rmat(12, seed=2)
    w = gg.arc_weights(g)
    h = upload(dawn, g, w)
    try:
        srcs = gg.sample_sources(g, 6, seed=13)
        out = torch.empty((len(srcs), g.n), dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        for i, s in enumerate(srcs):
            dawn.dawn_wsssp_async(h, int(s), out[i], None, stream)
        dawn.dawn_graph_sync(h, stream)
        got = out.cpu().numpy()
        for i, s in enumerate(srcs):
            np.testing.assert_array_equal(got[i], oracle.dijkstra(g.row_ptr, g.col_idx, w, s))
    finally:
        dawn.dawn_graph_free(h)


def test_weights_replaced(dawn):
    g = gg.rmat(10, seed=2)
    h = upload(dawn, g, gg.arc_weights(g, 1, 9, seed=1))
    try:
        w2 = gg.arc_weights(g, 5, 500, seed=2)
        dawn.dawn_graph_set_weights(h, w2)
        d, st = run_host(dawn, h, g.n, 3)
        check(g, w2, 3, d, st)
    finally:
        dawn.dawn_graph_free(h)


def test_rmat20_full_size_certificate(dawn):
    """The weighted workload at full size (RMAT scale 20, weights 1-255): the
    weighted certificate (complete at any size) on sampled sources, plus one
    source against the oracle's Dijkstra element by element."""
    g = gg.rmat(20, seed=2)
    w = gg.arc_weights(g, 1, 255, seed=7)
    h = upload(dawn, g, w)
    try:
        srcs = gg.sample_sources(g, 3, seed=5)
        for i, s in enumerate(srcs):
            d, st = run_device(dawn, h, g.n, s)
            assert oracle.wcertificate(g.row_ptr, g.col_idx, w, s, d) == (1, -1)
            assert st["reached"] == int((d >= 0).sum())
            if i == 0:
                np.testing.assert_array_equal(d, oracle.dijkstra(g.row_ptr, g.col_idx, w, s))
    finally:
        dawn.dawn_graph_free(h)


def test_bad_arguments(dawn):
    g = gg.rmat(8, seed=2)
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC)
    try:
        dist = np.zeros(g.n, dtype=np.int64)
        with pytest.raises(dawn.DawnError) as e:
            dawn.dawn_wsssp(h, 0, dist)
        assert e.value.code == dawn.DAWN_E_INVALID
        bad = gg.arc_weights(g)
        bad[g.m // 2] = -5
        with pytest.raises(dawn.DawnError) as e:
            dawn.dawn_graph_set_weights(h, bad)
        assert e.value.code == dawn.DAWN_E_INVALID and str(g.m // 2) in str(e.value)
        with pytest.raises(dawn.DawnError):
            dawn.dawn_wsssp(h, 0, dist)  # rejected weights leave none attached
        good = gg.arc_weights(g)
        dawn.dawn_graph_set_weights(h, good)
        with pytest.raises(dawn.DawnError) as e:
            dawn.dawn_wsssp(h, g.n, dist)
        assert e.value.code == dawn.DAWN_E_INVALID
        d, st = run_host(dawn, h, g.n, 0)
        check(g, good, 0, d, st)
    finally:
        dawn.dawn_graph_free(h)
