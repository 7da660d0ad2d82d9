"""Single-source parity: the CUDA path (through the C ABI) against the CPU
oracle, element by element.  Distances are integers: the bar is bit-exact.

Sizes: tiny hand-derived and random digraphs (all three traversal modes),
the 1024-vertex directed ER graph with sources 0-3, RMAT graphs of growing
scale with isolated and hub sources, ragged n (not a multiple of 32),
at full size the RMAT scale-20 graph (sampled sources against Alg. 3, all
64 against the certificate) and the 4096^2 lattice (against Alg. 2), and
RMAT scale 21, whose pulls test against the bitmap in global memory.
"""
import numpy as np
import pytest

import oracle
from paper_2208_04514_b300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# traversal modes (auto, push only = Alg. 3, pull only = Alg. 1) on both
# engines (the grid-wide loop and the single-cluster loop, push only), and the
# automatic choice of both
MODES = [{"mode": 0, "engine": 1}, {"mode": 1, "engine": 1}, {"mode": 2, "engine": 1},
         {"mode": 0, "engine": 2}, {"mode": 1, "engine": 2}, {"mode": 0, "engine": 0}]


def upload(dawn, g):
    flags = dawn.DAWN_SYMMETRIC if g.symmetric else dawn.DAWN_DIRECTED
    return dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=flags)


def gpu_sssp(dawn, h, n, src, opts=None, host=False):
    opts = opts or {}
    if host:
        d = np.full(n, -7, dtype=np.int32)
        st = dawn.dawn_sssp_ex(h, src, d, opts)
        return d, st
    d = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    st = dawn.dawn_sssp_ex(h, src, d, opts)
    return d.cpu().numpy(), st


def check_stats(g, d, st):
    deg = g.out_degree()
    assert st["reached"] == int((d >= 0).sum())
    assert st["edges"] == int(deg[d >= 0].sum())  # E_r, the SOVM cost of Sec. 3.3
    assert st["levels"] == int(d.max())


def test_golden_fixtures(dawn):
    from test_oracle_pins import parse_golden
    from pathlib import Path
    for f in sorted((Path(__file__).parent / "golden").glob("hand_*.txt")):
        n, arcs, cases = parse_golden(f)
        g = gg.from_arcs(n, [a for a, _ in arcs], [b for _, b in arcs])
        h = upload(dawn, g)
        try:
            for src, want in cases:
                for mode in MODES:
                    d, st = gpu_sssp(dawn, h, n, src, mode)
                    np.testing.assert_array_equal(d, want, err_msg=f"{f.name} src={src} mode={mode}")
        finally:
            dawn.dawn_graph_free(h)


@pytest.mark.parametrize("seed", range(12))
def test_random_small_digraphs(dawn, seed):
    from test_oracle_pins import random_digraph
    g = random_digraph(5000 + seed, n=int(np.random.default_rng(seed).integers(1, 70)))
    h = upload(dawn, g)
    try:
        for src in range(g.n):
            want = oracle.sssp_sovm(g.row_ptr, g.col_idx, src)
            for mode in MODES:
                d, st = gpu_sssp(dawn, h, g.n, src, mode)
                np.testing.assert_array_equal(d, want, err_msg=f"src={src} mode={mode}")
                check_stats(g, d, st)
    finally:
        dawn.dawn_graph_free(h)


def test_er_1024_sources_0_to_3(dawn):
    g = gg.erdos_renyi(1024, 8.0, seed=1)
    h = upload(dawn, g)
    try:
        for src in range(4):
            want = oracle.sssp_sovm(g.row_ptr, g.col_idx, src)
            for mode in MODES:
                for host in (False, True):
                    d, st = gpu_sssp(dawn, h, g.n, src, mode, host)
                    np.testing.assert_array_equal(d, want)
                    check_stats(g, d, st)
    finally:
        dawn.dawn_graph_free(h)


@pytest.mark.parametrize("scale", [8, 12, 16])
def test_rmat_scales(dawn, scale):
    g = gg.rmat(scale, seed=2)
    deg = g.out_degree()
    h = upload(dawn, g)
    try:
        srcs = list(gg.sample_sources(g, 6, seed=scale))
        srcs.append(int(np.argmax(deg)))                       # the largest hub
        iso = np.nonzero(deg == 0)[0]
        if iso.size:
            srcs.append(int(iso[0]))                           # an isolated source
        for src in srcs:
            want = oracle.sssp_sovm(g.row_ptr, g.col_idx, src)
            for mode in MODES:
                d, st = gpu_sssp(dawn, h, g.n, src, mode)
                np.testing.assert_array_equal(d, want, err_msg=f"src={src} mode={mode}")
                check_stats(g, d, st)
    finally:
        dawn.dawn_graph_free(h)


def test_directed_rmat_uses_in_adjacency(dawn):
    g = gg.rmat(12, seed=9, symmetrise=False)
    h = upload(dawn, g)
    try:
        deg = g.out_degree()
        srcs = list(gg.sample_sources(g, 5, seed=1)) + [int(np.nonzero(deg == 0)[0][0])]
        for src in srcs:
            want = oracle.sssp_sovm(g.row_ptr, g.col_idx, src)
            for mode in MODES:
                d, _ = gpu_sssp(dawn, h, g.n, src, mode)
                np.testing.assert_array_equal(d, want, err_msg=f"src={src} mode={mode}")
    finally:
        dawn.dawn_graph_free(h)


@pytest.mark.parametrize("n", [1, 2, 31, 33, 63, 65, 1000, 4097])
def test_ragged_sizes_paths_and_stars(dawn, n):
    # undirected path: one vertex per level, the longest level chain for n
    s = np.arange(max(n - 1, 0))
    g = gg.from_arcs(n, np.r_[s, s + 1], np.r_[s + 1, s], symmetric=True)
    h = upload(dawn, g)
    try:
        for src in {0, n // 2, n - 1}:
            for mode in MODES:
                d, st = gpu_sssp(dawn, h, n, src, mode)
                np.testing.assert_array_equal(d, np.abs(np.arange(n) - src))
                check_stats(g, d, st)
    finally:
        dawn.dawn_graph_free(h)


def test_empty_graph_and_self_loops(dawn):
    g = gg.from_arcs(5, [], [])
    h = upload(dawn, g)
    try:
        for mode in MODES:
            d, st = gpu_sssp(dawn, h, 5, 3, mode)
            np.testing.assert_array_equal(d, [-1, -1, -1, 0, -1])
            assert st["levels"] == 0 and st["reached"] == 1 and st["edges"] == 0
    finally:
        dawn.dawn_graph_free(h)
    g = gg.from_arcs(4, [0, 0, 1, 1, 2, 3, 3], [0, 1, 1, 2, 2, 3, 0])  # loops + dup-free chain
    h = upload(dawn, g)
    try:
        for mode in MODES:
            d, _ = gpu_sssp(dawn, h, 4, 0, mode)
            np.testing.assert_array_equal(d, [0, 1, 2, -1])
            d, _ = gpu_sssp(dawn, h, 4, 3, mode)
            np.testing.assert_array_equal(d, [1, 2, 3, 0])
    finally:
        dawn.dawn_graph_free(h)


def test_invalid_inputs(dawn):
    rp = np.array([0, 2, 1], dtype=np.int32)  # decreasing
    ci = np.array([1, 0], dtype=np.int32)
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_graph_upload(rp, ci)
    assert ei.value.code == dawn.DAWN_E_INVALID and "row_ptr[2]" in str(ei.value)
    rp = np.array([0, 1, 2], dtype=np.int32)
    ci = np.array([1, 5], dtype=np.int32)  # out of range
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_graph_upload(rp, ci)
    assert "col_idx[1]" in str(ei.value)
    g = gg.erdos_renyi(64, 2.0, seed=3)
    h = upload(dawn, g)
    try:
        d = np.zeros(64, dtype=np.int32)
        for bad in (-1, 64, 1 << 30):
            with pytest.raises(dawn.DawnError) as ei:
                dawn.dawn_sssp(h, bad, d)
            assert ei.value.code == dawn.DAWN_E_INVALID
        with pytest.raises(dawn.DawnError):
            dawn.dawn_sssp_ex(h, 0, d, {"mode": 7})
        with pytest.raises(dawn.DawnError):
            dawn.dawn_sssp_ex(h, 0, d, {"engine": 7})
        with pytest.raises(dawn.DawnError):
            dawn.dawn_sssp_ex(h, 0, d, {"engine": 2, "mode": 2})
    finally:
        dawn.dawn_graph_free(h)


def test_barrier_timeout_is_reported_and_recoverable(dawn):
    """A one-cycle spin budget makes the first grid-barrier wait run out: the
    call must return DAWN_E_TIMEOUT, and the next call must work."""
    g = gg.rmat(12, seed=2)
    h = upload(dawn, g)
    try:
        d = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_sssp_ex(h, 0, d, {"spin_limit": 1})
        assert ei.value.code == dawn.DAWN_E_TIMEOUT
        src = int(gg.sample_sources(g, 1, seed=4)[0])
        dawn.dawn_sssp(h, src, d)
        np.testing.assert_array_equal(d.cpu().numpy(), oracle.sssp_sovm(g.row_ptr, g.col_idx, src))
    finally:
        dawn.dawn_graph_free(h)


def test_async_queue_of_sources(dawn):
    g = gg.rmat(14, seed=2)
    h = upload(dawn, g)
    try:
        srcs = gg.sample_sources(g, 16, seed=3)
        out = torch.zeros((len(srcs), g.n), dtype=torch.int32, device="cuda")
        stats = torch.zeros((len(srcs), dawn.STATS_WORDS), dtype=torch.int64, device="cuda")
        for i, s in enumerate(srcs):
            dawn.dawn_sssp_async(h, int(s), out[i], None, stats[i])
        dawn.dawn_graph_sync(h)
        out = out.cpu().numpy()
        stats = stats.cpu().numpy()
        for i, s in enumerate(srcs):
            d = out[i]
            np.testing.assert_array_equal(d, oracle.sssp_sovm(g.row_ptr, g.col_idx, int(s)))
            check_stats(g, d, dawn.stats_from_words(stats[i]))
    finally:
        dawn.dawn_graph_free(h)


@pytest.fixture(scope="module")
def rmat20():
    return gg.rmat(20, seed=2)


def test_rmat20_full_size(dawn, rmat20):
    """Full-size RMAT scale 20: 8 sampled sources element by element against
    Alg. 3, all 64 bench sources against the certificate (Thm 1 + Fact 1)."""
    g = rmat20
    h = upload(dawn, g)
    try:
        srcs = gg.sample_sources(g, 64, seed=5)
        d = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        for i, s in enumerate(srcs):
            st = dawn.dawn_sssp_ex(h, int(s), d)
            dh = d.cpu().numpy()
            assert oracle.certificate(g.row_ptr, g.col_idx, int(s), dh) == (0, -1)
            check_stats(g, dh, st)
            if i < 8:
                np.testing.assert_array_equal(dh, oracle.sssp_sovm(g.row_ptr, g.col_idx, int(s)))
        iso = int(np.nonzero(g.out_degree() == 0)[0][0])
        st = dawn.dawn_sssp_ex(h, iso, d)
        dh = d.cpu().numpy()
        assert dh[iso] == 0 and (dh >= 0).sum() == 1 and st["levels"] == 0
    finally:
        dawn.dawn_graph_free(h)


def test_lattice_4096_full_size(dawn):
    """Full-size 4096^2 lattice (p = 0.1), ~10^4 levels: all 16 sources the
    benchmark times (uniform, seed 7) against Alg. 2 (the oracle's queue BFS)
    and the certificate; the grid-wide engine on two of them as well."""
    g = gg.lattice(4096, 4096, 0.1, seed=3)
    h = upload(dawn, g)
    try:
        d = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        srcs = gg.uniform_vertices(g.n, 16, seed=7)
        # the 16 sources in one call as well: several clusters side by side
        rows = torch.full((16, g.n), -7, dtype=torch.int32, device="cuda")
        mstats = torch.zeros((16, dawn.STATS_WORDS), dtype=torch.int64, device="cuda")
        dawn.dawn_sssp_many(h, torch.from_numpy(srcs.astype(np.int32)).cuda(), dist=rows, stats=mstats)
        mst = mstats.cpu().numpy()
        for i, s in enumerate(srcs):
            st = dawn.dawn_sssp_ex(h, int(s), d)
            dh = d.cpu().numpy()
            np.testing.assert_array_equal(dh, oracle.bfs_queue(g.row_ptr, g.col_idx, int(s)))
            assert oracle.certificate(g.row_ptr, g.col_idx, int(s), dh) == (0, -1)
            check_stats(g, dh, st)
            assert st["levels"] > 4000
            np.testing.assert_array_equal(rows[i].cpu().numpy(), dh)
            check_stats(g, dh, dawn.stats_from_words(mst[i]))
            if i < 2:
                # the grid-wide engine on the same source (AUTO takes the cluster here)
                st = dawn.dawn_sssp_ex(h, int(s), d, {"engine": 1})
                np.testing.assert_array_equal(d.cpu().numpy(), dh)
                check_stats(g, dh, st)
    finally:
        dawn.dawn_graph_free(h)


@pytest.mark.parametrize("where", ["host_pinned", "host_pageable", "device"])
def test_many_sources_rows(dawn, where):
    """dawn_sssp_many: every row equals the oracle (and the single-source
    call), for pinned / pageable host rows and device rows, with statistics;
    an odd k exercises both staging buffers unevenly."""
    g = gg.rmat(13, seed=7)
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC)
    try:
        srcs = gg.sample_sources(g, 7, seed=3)
        if where == "device":
            dist = torch.full((7, g.n), 99, dtype=torch.int32, device="cuda")
            stats = torch.zeros((7, dawn.STATS_WORDS), dtype=torch.int64, device="cuda")
            dawn.dawn_sssp_many(h, torch.from_numpy(srcs).cuda(), dist=dist, stats=stats)
            rows, st = dist.cpu().numpy(), stats.cpu().numpy()
        else:
            dist = torch.full((7, g.n), 99, dtype=torch.int32, pin_memory=(where == "host_pinned"))
            stats = np.zeros((7, dawn.STATS_WORDS), dtype=np.int64)
            dawn.dawn_sssp_many(h, srcs, dist=dist, stats=stats)
            rows, st = dist.numpy(), stats
        for i, s in enumerate(srcs):
            want = oracle.sssp_sovm(g.row_ptr, g.col_idx, int(s))
            np.testing.assert_array_equal(rows[i], want)
            assert dawn.stats_from_words(st[i])["reached"] == int((want >= 0).sum())
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_sssp_many(h, np.array([0, g.n], dtype=np.int32), dist=np.zeros((2, g.n), dtype=np.int32))
        assert ei.value.code == dawn.DAWN_E_INVALID
    finally:
        dawn.dawn_graph_free(h)


def test_cluster_engine_graphs_of_different_sizes(dawn):
    """The cluster engine's shared-memory limit belongs to the kernel: setting
    up a smaller graph after a larger one must not break the larger one's
    launches (they need more dynamic shared memory)."""
    big = gg.lattice(1024, 1024, 0.1, seed=3)
    small = gg.lattice(40, 40, 0.1, seed=4)
    hb, hs = upload(dawn, big), upload(dawn, small)
    try:
        opts = {"engine": 2}
        for h, g, s in ((hb, big, 0), (hs, small, 0), (hb, big, 777), (hs, small, 99)):
            d, st = gpu_sssp(dawn, h, g.n, s, opts)
            np.testing.assert_array_equal(d, oracle.bfs_queue(g.row_ptr, g.col_idx, s))
            check_stats(g, d, st)
    finally:
        dawn.dawn_graph_free(hb)
        dawn.dawn_graph_free(hs)


def test_many_device_rows_graph_replay(dawn):
    """Device rows on the grid engine: the first call captures the launches as
    a CUDA graph, a repeated call replays it.  A direct launch in between
    changes the barrier-counter parity, so the next call must not replay a
    graph captured on the other parity: every result stays exact."""
    g = gg.rmat(14, seed=2)  # high degree: grid engine
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC)
    try:
        srcs = gg.sample_sources(g, 9, seed=8)
        src_dev = torch.from_numpy(srcs).cuda()
        want = np.stack([oracle.sssp_sovm(g.row_ptr, g.col_idx, int(s)) for s in srcs])
        dist = torch.full((9, g.n), -7, dtype=torch.int32, device="cuda")
        one = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for rep in range(5):
            dist.fill_(-7)
            dawn.dawn_sssp_many(h, src_dev, dist=dist)
            np.testing.assert_array_equal(dist.cpu().numpy(), want, err_msg=f"call {rep}")
            if rep in (1, 3):
                dawn.dawn_sssp(h, int(srcs[0]), one)  # one direct launch: the parity flips
                np.testing.assert_array_equal(one.cpu().numpy(), want[0])
    finally:
        dawn.dawn_graph_free(h)


def test_symmetric_components_stop_when_reached(dawn):
    """On a symmetric graph the loop stops as soon as the source's connected
    component (found at upload) is reached: distances and statistics are as
    before, and the levels run are exactly those that reached a vertex."""
    src, dst = [], []
    def edge(a, b):
        src.extend([a, b])
        dst.extend([b, a])
    for i in range(49):          # path 0..49
        edge(i, i + 1)
    for i in range(51, 70):      # star: centre 50, leaves 51..69
        edge(50, i)
    for i in range(30):          # cycle 70..99
        edge(70 + i, 70 + (i + 1) % 30)
    edge(0, 0)                   # a self-loop; 100..104 isolated
    g = gg.from_arcs(105, src, dst, symmetric=True)
    h = upload(dawn, g)
    try:
        for s in [0, 25, 49, 50, 57, 70, 85, 102]:
            d, st = gpu_sssp(dawn, h, g.n, s, {"engine": 1})  # the grid engine (AUTO picks the cluster here)
            np.testing.assert_array_equal(d, oracle.sssp_sovm(g.row_ptr, g.col_idx, s))
            check_stats(g, d, st)
            if st["levels"] > 0:
                assert st["push_steps"] + st["pull_steps"] == st["levels"]
    finally:
        dawn.dawn_graph_free(h)


@pytest.mark.parametrize("symmetric", [True, False])
def test_pulls_against_a_bitmap_in_global_memory(dawn, symmetric):
    """n = 2^21: the visited bitmap (256 KB) is larger than a CTA copies into
    shared memory, so the pull levels test in-neighbours against the bitmap
    in global memory, the other pull path.  RMAT scale 21, edge factor 4,
    symmetric and directed, AUTO and pull only, against the oracle."""
    g = gg.rmat(21, edge_factor=4, seed=12, symmetrise=symmetric)
    assert (g.n + 31) // 32 * 4 > 200 * 1024
    h = upload(dawn, g)
    try:
        for src in gg.sample_sources(g, 3, seed=21):
            want = oracle.sssp_sovm(g.row_ptr, g.col_idx, int(src))
            for opts in ({"mode": 0, "engine": 1}, {"mode": 2, "engine": 1}):
                d, st = gpu_sssp(dawn, h, g.n, int(src), opts)
                np.testing.assert_array_equal(d, want, err_msg=f"src={src} opts={opts}")
                check_stats(g, d, st)
                if opts["mode"] == 2:
                    assert st["pull_steps"] >= 1 and st["push_steps"] == 0
    finally:
        dawn.dawn_graph_free(h)


def test_symmetric_flag_is_checked_at_upload(dawn):
    """DAWN_SYMMETRIC makes the CSR its own in-adjacency, so the upload checks
    that the arc multiset equals its reverse and rejects a graph that is not
    symmetric with DAWN_E_INVALID naming an arc without a matching reverse
    (through the binding and through the raw C ABI)."""
    import ctypes
    # a directed ER graph uploaded as symmetric
    g = gg.erdos_renyi(500, 4.0, seed=3)
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC)
    assert ei.value.code == dawn.DAWN_E_INVALID and "DAWN_SYMMETRIC" in str(ei.value)
    # a symmetric RMAT graph with one arc (u, v) taken out: the arc left without a reverse, (v, u), is named
    s = gg.rmat(12, seed=5)
    u = int(np.nonzero(s.out_degree() >= 3)[0][0])
    j = int(s.row_ptr[u]) + 1
    v = int(s.col_idx[j])
    src = np.repeat(np.arange(s.n), s.out_degree())
    keep = np.ones(s.m, dtype=bool)
    keep[j] = False
    cut = gg.from_arcs(s.n, src[keep], s.col_idx[keep])
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_graph_upload(cut.row_ptr, cut.col_idx, flags=dawn.DAWN_SYMMETRIC)
    msg = str(ei.value)
    assert ei.value.code == dawn.DAWN_E_INVALID and f"arc ({v}, {u})" in msg, msg
    # the raw C ABI returns the same status
    lib = dawn.load()
    h = ctypes.c_void_p()
    rc = lib.dawn_graph_upload(cut.row_ptr.ctypes.data, cut.col_idx.ctypes.data, cut.n, cut.m,
                               dawn.DAWN_SYMMETRIC, None, ctypes.byref(h))
    assert rc == dawn.DAWN_E_INVALID and "DAWN_SYMMETRIC" in dawn.dawn_last_error()
    # symmetric graphs with self-loops and duplicated edges (both arcs) pass,
    # and give the oracle's distances
    a = np.array([0, 1, 1, 2, 3, 3, 0], dtype=np.int64)
    b = np.array([1, 2, 2, 3, 3, 0, 1], dtype=np.int64)
    ok = gg.from_arcs(4, np.r_[a, b], np.r_[b, a], symmetric=True)
    h2 = dawn.dawn_graph_upload(ok.row_ptr, ok.col_idx, flags=dawn.DAWN_SYMMETRIC)
    try:
        d = np.zeros(4, dtype=np.int32)
        dawn.dawn_sssp(h2, 0, d)
        np.testing.assert_array_equal(d, oracle.sssp_sovm(ok.row_ptr, ok.col_idx, 0))
    finally:
        dawn.dawn_graph_free(h2)


@pytest.mark.parametrize("where", ["device", "host"])
def test_many_sources_on_the_cluster_engine(dawn, where):
    """dawn_sssp_many on a low-degree graph runs its sources on several
    clusters at once, each taking the next source: more sources than clusters
    the device holds, device and host rows, every row against Alg. 2 and the
    per-source statistics against the rows."""
    g = gg.lattice(300, 220, 0.1, seed=5)
    h = upload(dawn, g)
    try:
        srcs = gg.uniform_vertices(g.n, 41, seed=3).astype(np.int32)
        if where == "device":
            rows_t = torch.full((41, g.n), -7, dtype=torch.int32, device="cuda")
            st_t = torch.zeros((41, dawn.STATS_WORDS), dtype=torch.int64, device="cuda")
            dawn.dawn_sssp_many(h, torch.from_numpy(srcs).cuda(), dist=rows_t, stats=st_t)
            rows, st = rows_t.cpu().numpy(), st_t.cpu().numpy()
        else:
            rows = np.full((41, g.n), -7, dtype=np.int32)
            st = np.zeros((41, dawn.STATS_WORDS), dtype=np.int64)
            dawn.dawn_sssp_many(h, srcs, dist=rows, stats=st)
        for i, s in enumerate(srcs):
            np.testing.assert_array_equal(rows[i], oracle.bfs_queue(g.row_ptr, g.col_idx, int(s)))
            check_stats(g, rows[i], dawn.stats_from_words(st[i]))
    finally:
        dawn.dawn_graph_free(h)


def _trace_levels(dawn, h, g, src):
    """dawn_sssp_ex with the per-level trace: the distances, the statistics and
    the trace records {kind, step, count, time} (kind 5 = a list pull)."""
    tr = torch.zeros((64, 4), dtype=torch.int64, device="cuda")
    d, st = gpu_sssp(dawn, h, g.n, src, {"engine": 1, "trace": tr.data_ptr(), "trace_cap": 64})
    recs = [r for r in tr.cpu().numpy() if r[3] != 0]
    return d, st, recs


def test_lookahead_stop_folds_the_last_level(dawn):
    """A list pull on a symmetric graph tests the candidates it leaves
    unreached one level further (through their first two in-neighbours and
    theirs), and two levels further for vertices whose rows and whose
    in-neighbours' rows are short.  When that shows every vertex left in the
    source's component, the loop stops there and the last levels are not run:
    the trace then ends with a list pull one or two steps short of the
    eccentricity.  Distances and
    statistics (reached, E_r, levels, push + pull levels) stay those of the
    oracle whether or not it folds.  The second graph hangs a K4 off a path:
    the K4's far vertices have a first two in-neighbours that lie at their own
    level or the one before, so no two-hop test can place them and the level
    that finds them runs."""
    base = gg.rmat(16, seed=2)
    folded = 0
    h = upload(dawn, base)
    try:
        for src in gg.sample_sources(base, 24, seed=21):
            src = int(src)
            d, st, recs = _trace_levels(dawn, h, base, src)
            np.testing.assert_array_equal(d, oracle.sssp_sovm(base.row_ptr, base.col_idx, src), err_msg=f"src={src}")
            check_stats(base, d, st)
            assert st["push_steps"] + st["pull_steps"] == st["levels"]
            last = recs[-1]
            if last[0] == 5 and last[1] in (st["levels"] - 1, st["levels"] - 2):
                folded += 1
            else:
                assert last[1] == st["levels"], (src, recs[-1], st)
    finally:
        dawn.dawn_graph_free(h)
    assert folded >= 1

    # the RMAT graph with a path to a K4 from its largest hub
    rp, ci, n = base.row_ptr, base.col_idx, base.n
    src_l = list(np.repeat(np.arange(n), np.diff(rp)))
    dst_l = list(ci)
    hub = int(np.argmax(base.out_degree()))

    def edge(a, b):
        src_l.extend([a, b])
        dst_l.extend([b, a])
    path = list(range(n, n + 5))
    edge(hub, path[0])
    for a, b in zip(path, path[1:]):
        edge(a, b)
    k4 = [n + 5, n + 6, n + 7, n + 8]
    edge(path[-1], k4[0])
    for i in range(4):
        for j in range(i + 1, 4):
            edge(k4[i], k4[j])
    g = gg.from_arcs(n + 9, src_l, dst_l, symmetric=True)
    h = upload(dawn, g)
    try:
        for src in list(gg.sample_sources(base, 8, seed=22)) + [hub, path[2], k4[3]]:
            src = int(src)
            d, st, recs = _trace_levels(dawn, h, g, src)
            np.testing.assert_array_equal(d, oracle.sssp_sovm(g.row_ptr, g.col_idx, src), err_msg=f"src={src}")
            check_stats(g, d, st)
            assert st["push_steps"] + st["pull_steps"] == st["levels"]
            if set(np.nonzero(d == d.max())[0].tolist()) <= set(k4[1:]):
                assert recs[-1][1] == st["levels"], (src, recs[-1], st)  # the last level ran
    finally:
        dawn.dawn_graph_free(h)


def test_lookahead_two_levels_on_tails(dawn):
    """An RMAT graph with a two-vertex tail hung on every vertex of degree 1:
    a tail's first vertex has two in-arcs and its end one, so a list pull at
    the level of the leaf the tail hangs on places the first vertex one level
    ahead (two-hop test) and the end two levels ahead (both rows short, the
    leaf's neighbour reached before the level).  When the farthest base level
    is a list pull, both tail levels fold into it: the trace ends two steps
    short of the eccentricity.  Every source's distances and statistics are
    the oracle's whether or not it folds."""
    base = gg.rmat(14, seed=4)
    rp, ci, n = base.row_ptr, base.col_idx, base.n
    deg = np.diff(rp)
    src_l = list(np.repeat(np.arange(n), deg))
    dst_l = list(ci)
    nn = n
    for leaf in np.nonzero(deg == 1)[0]:
        t1, t2 = nn, nn + 1
        nn += 2
        src_l += [int(leaf), t1, t1, t2]
        dst_l += [t1, int(leaf), t2, t1]
    g = gg.from_arcs(nn, src_l, dst_l, symmetric=True)
    h = upload(dawn, g)
    double = 0
    try:
        for src in gg.sample_sources(base, 24, seed=31):
            src = int(src)
            d, st, recs = _trace_levels(dawn, h, g, src)
            np.testing.assert_array_equal(d, oracle.sssp_sovm(g.row_ptr, g.col_idx, src), err_msg=f"src={src}")
            check_stats(g, d, st)
            assert st["push_steps"] + st["pull_steps"] == st["levels"]
            last = recs[-1]
            if last[0] == 5 and last[1] == st["levels"] - 2:
                double += 1
            elif not (last[0] == 5 and last[1] == st["levels"] - 1):
                assert last[1] == st["levels"], (src, recs[-1], st)
    finally:
        dawn.dawn_graph_free(h)
    assert double >= 1


def test_lookahead_two_levels_needs_short_second_hop(dawn):
    """The two-level test needs every in-neighbour of v's in-neighbours read:
    with a fork on every leaf (t1 joined to the leaf and to two ends t2, t3),
    t1 has three in-arcs, so the ends cannot be placed two levels ahead.  When
    the farthest vertices are such ends, the level before them runs and its
    one-level look-ahead folds the last level: the trace ends one step short
    of the eccentricity, never two.  Distances and statistics are the
    oracle's."""
    base = gg.rmat(14, seed=4)
    rp, ci, n = base.row_ptr, base.col_idx, base.n
    deg = np.diff(rp)
    src_l = list(np.repeat(np.arange(n), deg))
    dst_l = list(ci)
    nn = n
    ends = set()
    for leaf in np.nonzero(deg == 1)[0]:
        t1, t2, t3 = nn, nn + 1, nn + 2
        nn += 3
        for x, y in ((int(leaf), t1), (t1, t2), (t1, t3)):
            src_l += [x, y]
            dst_l += [y, x]
        ends.update((t2, t3))
    g = gg.from_arcs(nn, src_l, dst_l, symmetric=True)
    h = upload(dawn, g)
    checked = 0
    try:
        for src in gg.sample_sources(base, 24, seed=31):
            src = int(src)
            d, st, recs = _trace_levels(dawn, h, g, src)
            np.testing.assert_array_equal(d, oracle.sssp_sovm(g.row_ptr, g.col_idx, src), err_msg=f"src={src}")
            check_stats(g, d, st)
            assert st["push_steps"] + st["pull_steps"] == st["levels"]
            if st["levels"] > 0 and set(np.nonzero(d == d.max())[0].tolist()) <= ends:
                assert recs[-1][1] >= st["levels"] - 1, (src, recs[-1], st)
                checked += 1
    finally:
        dawn.dawn_graph_free(h)
    assert checked >= 1
