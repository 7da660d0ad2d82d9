"""Continuous-batching server: every request's distance rows against the CPU
oracle, bit-exact, and the same request alone and inside a mix of requests
of uneven source counts on several resident graphs.  Also admission by the
device-memory budget, device outputs, the int16 overflow report and bad
arguments."""
import time

import numpy as np
import pytest

import oracle
from paper_2208_04514_b300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graphs():
    return [gg.rmat(10, seed=21), gg.erdos_renyi(1024, 8.0, seed=1), gg.lattice(32, 32, 0.1, seed=3),
            gg.rmat(12, seed=22, symmetrise=False)]


@pytest.fixture(scope="module")
def handles(dawn, graphs):
    hs = [dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC if g.symmetric else dawn.DAWN_DIRECTED)
          for g in graphs]
    yield hs
    for h in hs:
        dawn.dawn_graph_free(h)


def want_rows(g, srcs):
    return oracle.msbfs(g.row_ptr, g.col_idx, np.asarray(srcs, dtype=np.int32))[0]


def wait_done(dawn, s, rid, timeout=60.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        if dawn.dawn_serve_poll(s, rid) == dawn.DAWN_REQ_DONE:
            return
        time.sleep(0.001)
    raise AssertionError(f"request {rid} not done after {timeout} s")


@pytest.mark.parametrize("modes", ["auto", "dense", "frontier", "mixed"])
def test_alone_and_in_the_mix(dawn, graphs, handles, modes):
    """The same stream under each per-graph step: the dense pull, the frontier
    push, the automatic choice, and the two alternating across graphs."""
    if modes == "auto":
        s = dawn.dawn_serve_create(handles, 0, 256)
    else:
        pick = {"dense": [dawn.DAWN_SERVE_DENSE] * 4, "frontier": [dawn.DAWN_SERVE_FRONTIER] * 4,
                "mixed": [dawn.DAWN_SERVE_FRONTIER, dawn.DAWN_SERVE_DENSE] * 2}[modes]
        s = dawn.dawn_serve_create_ex(handles, 0, 256, pick)
    try:
        probe_srcs = np.array([3, 17, 200, 511, 1000], dtype=np.int32)
        alone = np.full((5, graphs[0].n), 99, dtype=np.int16)
        rid = dawn.dawn_serve_submit(s, 0, probe_srcs, dist_bytes=2, dist_out=alone)
        wait_done(dawn, s, rid)
        np.testing.assert_array_equal(alone, want_rows(graphs[0], probe_srcs))

        rng = np.random.default_rng(7)
        reqs = []
        for i in range(120):
            gi = int(rng.integers(0, len(graphs)))
            k = int(min(300, max(1, np.floor(256 ** rng.random()))))
            srcs = rng.integers(0, graphs[gi].n, k).astype(np.int32)
            db = 2 if rng.random() < 0.5 else 4
            out = np.full((k, graphs[gi].n), 99, dtype=np.int16 if db == 2 else np.int32)
            reqs.append((dawn.dawn_serve_submit(s, gi, srcs, dist_bytes=db, dist_out=out), gi, srcs, out))
            if i == 60:  # the probe again, in the middle of the stream
                mixed = np.full((5, graphs[0].n), 99, dtype=np.int16)
                mid = dawn.dawn_serve_submit(s, 0, probe_srcs, dist_bytes=2, dist_out=mixed)
            if i % 10 == 0:
                time.sleep(0.002)  # arrivals spread while earlier requests run
        dawn.dawn_serve_drain(s, 120000)
        wait_done(dawn, s, mid)
        np.testing.assert_array_equal(mixed, alone)
        for rid, gi, srcs, out in reqs:
            assert dawn.dawn_serve_poll(s, rid) == dawn.DAWN_REQ_DONE
            np.testing.assert_array_equal(out.astype(np.int64), want_rows(graphs[gi], srcs), err_msg=f"request {rid}")
            t_sub, t_done = dawn.dawn_serve_times(s, rid)
            assert t_done >= t_sub > 0
    finally:
        dawn.dawn_serve_destroy(s)


def test_memory_budget_admission_and_device_outputs(dawn, graphs, handles):
    g = graphs[1]
    block = 64 * g.n * 4
    s = dawn.dawn_serve_create(handles, block + 1024, 64)  # room for one 64-source int32 block at a time
    try:
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_serve_submit(s, 1, np.arange(65, dtype=np.int32), dist_bytes=4,
                                   dist_out=np.zeros((65, g.n), dtype=np.int32))
        assert ei.value.code == dawn.DAWN_E_NOMEM
        outs = []
        for r in range(6):
            srcs = np.arange(r, r + 64, dtype=np.int32)
            out = np.zeros((64, g.n), dtype=np.int32)
            outs.append((dawn.dawn_serve_submit(s, 1, srcs, dist_bytes=4, dist_out=out), srcs, out))
        dev_srcs = np.array([5, 6, 7], dtype=np.int32)
        dev_out = torch.full((3, graphs[2].n), 99, dtype=torch.int32, device="cuda")
        rd = dawn.dawn_serve_submit(s, 2, dev_srcs, dist_bytes=4, dist_out=dev_out)
        dawn.dawn_serve_drain(s, 60000)
        for rid, srcs, out in outs:
            np.testing.assert_array_equal(out, want_rows(g, srcs))
        assert dawn.dawn_serve_poll(s, rd) == dawn.DAWN_REQ_DONE
        np.testing.assert_array_equal(dev_out.cpu().numpy(), want_rows(graphs[2], dev_srcs))
    finally:
        dawn.dawn_serve_destroy(s)


@pytest.mark.parametrize("mode", ["dense", "frontier"])
def test_overflow_and_bad_arguments(dawn, mode):
    """A 40,000-vertex path: levels past 32767 overflow an int16 row (the
    request fails with DAWN_E_OVERFLOW), the int32 request on the same path
    completes exactly."""
    n = 40000
    s_ = np.arange(n - 1)
    path = gg.from_arcs(n, np.r_[s_, s_ + 1], np.r_[s_ + 1, s_], symmetric=True)
    h = dawn.dawn_graph_upload(path.row_ptr, path.col_idx, flags=dawn.DAWN_SYMMETRIC)
    s = dawn.dawn_serve_create_ex([h], 0, 64, [dawn.DAWN_SERVE_DENSE if mode == "dense" else dawn.DAWN_SERVE_FRONTIER])
    try:
        out16 = np.zeros((1, n), dtype=np.int16)
        r16 = dawn.dawn_serve_submit(s, 0, np.array([0], dtype=np.int32), dist_bytes=2, dist_out=out16)
        out32 = np.zeros((1, n), dtype=np.int32)
        r32 = dawn.dawn_serve_submit(s, 0, np.array([0], dtype=np.int32), dist_bytes=4, dist_out=out32)
        dawn.dawn_serve_drain(s, 120000)  # returns once every request is done or failed
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_serve_poll(s, r16)
        assert ei.value.code == dawn.DAWN_E_OVERFLOW
        assert dawn.dawn_serve_poll(s, r32) == dawn.DAWN_REQ_DONE
        np.testing.assert_array_equal(out32[0], np.arange(n))
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_serve_poll(s, 987654)
        assert ei.value.code == dawn.DAWN_E_STATE
        for bad in [dict(graph_idx=1), dict(sources=np.array([n], dtype=np.int32)), dict(dist_bytes=3)]:
            args = dict(graph_idx=0, sources=np.array([0], dtype=np.int32), dist_bytes=4)
            args.update(bad)
            with pytest.raises(dawn.DawnError) as ei:
                dawn.dawn_serve_submit(s, args["graph_idx"], args["sources"], dist_bytes=args["dist_bytes"],
                                       dist_out=np.zeros((1, n), dtype=np.int32))
            assert ei.value.code == dawn.DAWN_E_INVALID
    finally:
        dawn.dawn_serve_destroy(s)
        dawn.dawn_graph_free(h)
    with pytest.raises(dawn.DawnError):
        dawn.dawn_serve_create([h], 0, 100)


@pytest.mark.parametrize("mode", ["dense", "frontier"])
def test_lane_reuse_on_long_lattice(dawn, mode):
    """64 lanes, many more sources than lanes on a high-diameter lattice and a
    directed graph: every lane is re-admitted many times, so stale visited
    bits of finished lanes must never leak into a new lane's search."""
    lat = gg.lattice(96, 96, 0.25, seed=8)
    dg = gg.rmat(11, seed=31, symmetrise=False)
    hs = [dawn.dawn_graph_upload(lat.row_ptr, lat.col_idx, flags=dawn.DAWN_SYMMETRIC),
          dawn.dawn_graph_upload(dg.row_ptr, dg.col_idx, flags=dawn.DAWN_DIRECTED)]
    md = dawn.DAWN_SERVE_DENSE if mode == "dense" else dawn.DAWN_SERVE_FRONTIER
    s = dawn.dawn_serve_create_ex(hs, 0, 64, [md, md])
    try:
        rng = np.random.default_rng(11)
        reqs = []
        for i in range(40):
            gi = i % 2
            g = (lat, dg)[gi]
            k = int(rng.integers(1, 40))
            srcs = rng.integers(0, g.n, k).astype(np.int32)
            out = np.full((k, g.n), 99, dtype=np.int32)
            reqs.append((dawn.dawn_serve_submit(s, gi, srcs, dist_bytes=4, dist_out=out), g, srcs, out))
            if i % 8 == 7:
                time.sleep(0.003)
        dawn.dawn_serve_drain(s, 120000)
        for rid, g, srcs, out in reqs:
            assert dawn.dawn_serve_poll(s, rid) == dawn.DAWN_REQ_DONE
            np.testing.assert_array_equal(out, want_rows(g, srcs), err_msg=f"request {rid}")
    finally:
        dawn.dawn_serve_destroy(s)
        for h in hs:
            dawn.dawn_graph_free(h)


def test_bad_serve_modes(dawn, handles):
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_serve_create_ex(handles, 0, 64, [0, 1, 2, 3])
    assert ei.value.code == dawn.DAWN_E_INVALID


@pytest.mark.parametrize("mode", ["frontier", "dense"])
def test_serving_graphs_at_full_size(dawn, mode):
    """The serving workload's largest resident graphs: the 4096^2 lattice
    (p = 0.1, ~10^4 levels) and RMAT scale 22, both resident in one server, a
    few requests each (a 1-source and a 3-source request per graph, int16
    rows on the device), every served row against Alg. 2 (the oracle's FIFO
    BFS), under the frontier push and under the dense pull."""
    lat = gg.lattice(4096, 4096, 0.1, seed=3)
    rm = gg.rmat(22, seed=122)
    hs = [dawn.dawn_graph_upload(lat.row_ptr, lat.col_idx, flags=dawn.DAWN_SYMMETRIC),
          dawn.dawn_graph_upload(rm.row_ptr, rm.col_idx, flags=dawn.DAWN_SYMMETRIC)]
    step = dawn.DAWN_SERVE_FRONTIER if mode == "frontier" else dawn.DAWN_SERVE_DENSE
    s = dawn.dawn_serve_create_ex(hs, 0, 64, [step, step])
    try:
        reqs = []
        for gi, g in enumerate((lat, rm)):
            pool = gg.sample_sources(g, 4, seed=31 + gi)
            for srcs in (pool[:1], pool[1:]):
                out = torch.full((len(srcs), g.n), 77, dtype=torch.int16, device="cuda")
                rid = dawn.dawn_serve_submit(s, gi, np.ascontiguousarray(srcs, dtype=np.int32), dist_bytes=2,
                                             dist_out=out)
                reqs.append((g, srcs, out, rid))
        dawn.dawn_serve_drain(s, 600000)
        for g, srcs, out, rid in reqs:
            assert dawn.dawn_serve_poll(s, rid) == dawn.DAWN_REQ_DONE
            got = out.cpu().numpy()
            for i, src in enumerate(srcs):
                want = oracle.bfs_queue(g.row_ptr, g.col_idx, int(src)).astype(np.int16)
                np.testing.assert_array_equal(got[i], want)
    finally:
        dawn.dawn_serve_destroy(s)
        for h in hs:
            dawn.dawn_graph_free(h)


@pytest.mark.parametrize("dist_bytes", [2, 4])
def test_idle_fast_path_on_a_low_degree_graph(dawn, dist_bytes):
    """A lone request of at most four sources on a graph served in AUTO mode
    whose average out-degree is below 8 runs, while the server is idle, as
    single-source searches on thread-block clusters; requests that arrive
    together run in the serving loop.  Either way every row is the oracle's
    (Alg. 2), in int16 or int32, to host or device memory, and the same
    sources give the same rows both ways."""
    lat = gg.lattice(1024, 1024, 0.1, seed=3)   # m < 8n: the fast path's kind of graph
    rm = gg.rmat(12, seed=22)
    hs = [dawn.dawn_graph_upload(lat.row_ptr, lat.col_idx, flags=dawn.DAWN_SYMMETRIC),
          dawn.dawn_graph_upload(rm.row_ptr, rm.col_idx, flags=dawn.DAWN_SYMMETRIC)]
    s = dawn.dawn_serve_create(hs, 0, 64)
    dt = np.int16 if dist_bytes == 2 else np.int32
    tdt = torch.int16 if dist_bytes == 2 else torch.int32
    try:
        pool = gg.sample_sources(lat, 8, seed=41)
        lone = {}
        for i, where in enumerate(("device", "host", "device")):
            srcs = pool[i:i + 1 + i]   # 1, 2, 3 sources
            if where == "device":
                out = torch.full((len(srcs), lat.n), 77, dtype=tdt, device="cuda")
            else:
                out = np.full((len(srcs), lat.n), 77, dtype=dt)
            rid = dawn.dawn_serve_submit(s, 0, np.ascontiguousarray(srcs, dtype=np.int32), dist_bytes=dist_bytes,
                                         dist_out=out)
            wait_done(dawn, s, rid)
            got = out.cpu().numpy() if where == "device" else out
            for j, src in enumerate(srcs):
                want = oracle.bfs_queue(lat.row_ptr, lat.col_idx, int(src)).astype(dt)
                np.testing.assert_array_equal(got[j], want)
                lone[int(src)] = got[j].copy()
        # a burst: requests on both graphs at once (the loop), lattice rows as when alone
        reqs = []
        for gi, g in enumerate((lat, rm)):
            for r in range(3):
                srcs = pool[r:r + 2] if gi == 0 else gg.sample_sources(g, 2, seed=50 + r)
                out = torch.full((len(srcs), g.n), 77, dtype=tdt, device="cuda")
                rid = dawn.dawn_serve_submit(s, gi, np.ascontiguousarray(srcs, dtype=np.int32),
                                             dist_bytes=dist_bytes, dist_out=out)
                reqs.append((g, srcs, out, rid))
        dawn.dawn_serve_drain(s, 120000)
        for g, srcs, out, rid in reqs:
            assert dawn.dawn_serve_poll(s, rid) == dawn.DAWN_REQ_DONE
            got = out.cpu().numpy()
            for j, src in enumerate(srcs):
                want = oracle.bfs_queue(g.row_ptr, g.col_idx, int(src)).astype(dt)
                np.testing.assert_array_equal(got[j], want)
                if g is lat and int(src) in lone:
                    np.testing.assert_array_equal(got[j], lone[int(src)])
    finally:
        dawn.dawn_serve_destroy(s)
        for h in hs:
            dawn.dawn_graph_free(h)


def test_idle_fast_path_overflow_and_int32(dawn):
    """The idle fast path keeps the loop's int16 rule: on a 40,000-vertex
    path served in AUTO mode, a lone int16 request from one end fails with
    DAWN_E_OVERFLOW (levels past 32767), a lone int32 request completes
    exactly, and so do int16 requests whose levels all fit."""
    n = 40000
    s_ = np.arange(n - 1)
    path = gg.from_arcs(n, np.r_[s_, s_ + 1], np.r_[s_ + 1, s_], symmetric=True)
    h = dawn.dawn_graph_upload(path.row_ptr, path.col_idx, flags=dawn.DAWN_SYMMETRIC)
    s = dawn.dawn_serve_create([h], 0, 64)
    try:
        out16 = np.zeros((1, n), dtype=np.int16)
        r16 = dawn.dawn_serve_submit(s, 0, np.array([0], dtype=np.int32), dist_bytes=2, dist_out=out16)
        dawn.dawn_serve_drain(s, 120000)
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_serve_poll(s, r16)
        assert ei.value.code == dawn.DAWN_E_OVERFLOW
        out32 = torch.zeros((1, n), dtype=torch.int32, device="cuda")
        r32 = dawn.dawn_serve_submit(s, 0, np.array([0], dtype=np.int32), dist_bytes=4, dist_out=out32)
        wait_done(dawn, s, r32)
        np.testing.assert_array_equal(out32[0].cpu().numpy(), np.arange(n))
        mid = np.array([n // 2, n // 2 + 7], dtype=np.int32)  # farthest levels 20,000 and 20,006: they fit
        out_m = np.zeros((2, n), dtype=np.int16)
        rm = dawn.dawn_serve_submit(s, 0, mid, dist_bytes=2, dist_out=out_m)
        wait_done(dawn, s, rm)
        for j, src in enumerate(mid):
            np.testing.assert_array_equal(out_m[j], np.abs(np.arange(n) - int(src)).astype(np.int16))
    finally:
        dawn.dawn_serve_destroy(s)
        dawn.dawn_graph_free(h)
