"""Shortest-path tree parity: dawn_sssp_tree (through the C ABI) against the
CPU oracle's distances and its smallest-id predecessor tree (Fact 1),
element by element, bit-exact.

Covers random digraphs with self-loops and duplicate arcs (every source),
the directed ER workload (n = 1024, sources 0-3), symmetric and directed RMAT
graphs (hub rows longer than one warp), a percolated lattice, isolated and
single-vertex cases, host and device outputs, the stream-ordered variant, the
full-size RMAT scale-20 graph on sampled sources, and bad arguments.
"""
import numpy as np
import pytest

import oracle
from paper_2208_04514_b300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def upload(dawn, g):
    return dawn.dawn_graph_upload(g.row_ptr, g.col_idx,
                                  flags=dawn.DAWN_SYMMETRIC if g.symmetric else dawn.DAWN_DIRECTED)


def want(g, s):
    d = oracle.sssp_sovm(g.row_ptr, g.col_idx, s)
    return d, oracle.parents(g.row_ptr, g.col_idx, d)


def run_host(dawn, h, n, s):
    dist = np.full(n, 77, dtype=np.int32)
    par = np.full(n, 77, dtype=np.int32)
    dawn.dawn_sssp_tree(h, s, dist, par)
    return dist, par


def run_device(dawn, h, n, s):
    dist = torch.full((n,), 77, dtype=torch.int32, device="cuda")
    par = torch.full((n,), 77, dtype=torch.int32, device="cuda")
    dawn.dawn_sssp_tree(h, s, dist, par)
    return dist.cpu().numpy(), par.cpu().numpy()


@pytest.mark.parametrize("seed", range(6))
def test_small_digraphs_every_source(dawn, seed):
    from test_oracle_pins import random_digraph
    g = random_digraph(4100 + seed, n=int(np.random.default_rng(seed).integers(1, 60)))
    h = upload(dawn, g)
    try:
        for s in range(g.n):
            d, p = run_host(dawn, h, g.n, s)
            wd, wp = want(g, s)
            np.testing.assert_array_equal(d, wd)
            np.testing.assert_array_equal(p, wp, err_msg=f"source {s}")
    finally:
        dawn.dawn_graph_free(h)


@pytest.mark.parametrize("name", ["er1024", "rmat12", "rmat12_dir", "lattice64"])
def test_workload_graphs(dawn, name):
    g = {"er1024": lambda: gg.erdos_renyi(1024, 8.0, seed=1),
         "rmat12": lambda: gg.rmat(12, seed=2),
         "rmat12_dir": lambda: gg.rmat(12, seed=9, symmetrise=False),
         "lattice64": lambda: gg.lattice(64, 64, 0.1, seed=3)}[name]()
    h = upload(dawn, g)
    try:
        deg = g.out_degree()
        srcs = [0, 1, 2, 3, int(np.argmax(deg))]
        if (deg == 0).any():
            srcs.append(int(np.nonzero(deg == 0)[0][0]))  # isolated: the tree is empty
        for i, s in enumerate(srcs):
            run = run_device if i % 2 else run_host
            d, p = run(dawn, h, g.n, s)
            wd, wp = want(g, s)
            np.testing.assert_array_equal(d, wd)
            np.testing.assert_array_equal(p, wp, err_msg=f"{name} source {s}")
    finally:
        dawn.dawn_graph_free(h)


def test_async_matches_sync_and_single_vertex(dawn):
    g = gg.rmat(11, seed=4)
    h = upload(dawn, g)
    try:
        stream = torch.cuda.current_stream()
        d = torch.empty((3, g.n), dtype=torch.int32, device="cuda")
        p = torch.empty((3, g.n), dtype=torch.int32, device="cuda")
        for i, s in enumerate((5, 50, 500)):
            dawn.dawn_sssp_tree_async(h, s, d[i], p[i], stream)
        dawn.dawn_graph_sync(h, stream)
        for i, s in enumerate((5, 50, 500)):
            wd, wp = want(g, s)
            np.testing.assert_array_equal(d[i].cpu().numpy(), wd)
            np.testing.assert_array_equal(p[i].cpu().numpy(), wp)
    finally:
        dawn.dawn_graph_free(h)
    one = gg.from_arcs(1, np.array([0]), np.array([0]))  # a self-loop only
    h = upload(dawn, one)
    try:
        d, p = run_host(dawn, h, 1, 0)
        assert d.tolist() == [0] and p.tolist() == [-1]
    finally:
        dawn.dawn_graph_free(h)


def test_rmat20_full_size_sampled_sources(dawn):
    g = gg.rmat(20, seed=2)
    h = upload(dawn, g)
    try:
        srcs = gg.sample_sources(g, 2, seed=2)
        for s in srcs:
            d, p = run_device(dawn, h, g.n, int(s))
            wd, wp = want(g, int(s))
            np.testing.assert_array_equal(d, wd)
            np.testing.assert_array_equal(p, wp)
    finally:
        dawn.dawn_graph_free(h)


def test_bad_arguments(dawn):
    g = gg.rmat(8, seed=1)
    h = upload(dawn, g)
    try:
        dist = np.zeros(g.n, dtype=np.int32)
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_sssp_tree(h, g.n, dist, np.zeros(g.n, dtype=np.int32))
        assert ei.value.code == dawn.DAWN_E_INVALID
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_sssp_tree_async(h, 0, dist, np.zeros(g.n, dtype=np.int32))  # host memory
        assert ei.value.code == dawn.DAWN_E_INVALID
    finally:
        dawn.dawn_graph_free(h)


def shuffled_rows(g, seed):
    """The same graph with every CSR row in a random order (rows no longer ascending)."""
    rng = np.random.default_rng(seed)
    ci = g.col_idx.copy()
    for v in range(g.n):
        a, b = g.row_ptr[v], g.row_ptr[v + 1]
        ci[a:b] = rng.permutation(ci[a:b])
    return gg.Graph(g.name + "_shuffled", g.row_ptr.copy(), ci, g.symmetric)


@pytest.mark.parametrize("shuffle", [False, True])
def test_hub_row_with_late_predecessor(dawn, shuffle):
    """A hub H with 3,000 in-arcs whose only in-neighbour one level closer is
    the largest id: the CTA-wide scan must reach the end of the row (rows in
    order), or read the whole row (rows shuffled).  Also a symmetric RMAT
    graph with shuffled rows (no early stop on a symmetric upload)."""
    n = 3005
    hub, far = 1, n - 1
    leaves = np.arange(2, 2 + 3000)
    src = np.r_[0, far, leaves, np.full(3000, hub)]
    dst = np.r_[far, hub, np.full(3000, hub), leaves]
    g = gg.from_arcs(n, np.r_[src, dst], np.r_[dst, src], symmetric=True)
    if shuffle:
        g = shuffled_rows(g, 3)
    graphs = [g, shuffled_rows(gg.rmat(12, seed=2), 5) if shuffle else gg.rmat(12, seed=2)]
    for gr in graphs:
        h = upload(dawn, gr)
        try:
            for s in (0, int(np.argmax(gr.out_degree())), 7):
                d, p = run_device(dawn, h, gr.n, s)
                wd, wp = want(gr, s)
                np.testing.assert_array_equal(d, wd)
                np.testing.assert_array_equal(p, wp, err_msg=f"{gr.name} source {s}")
        finally:
            dawn.dawn_graph_free(h)


@pytest.mark.parametrize("row_len", [10, 40])
def test_level2_from_a_wide_source_row(dawn, row_len):
    """A source with about 2,000 level-1 neighbours (some arcs repeated) whose
    out-rows overlap, repeat arcs and reach back into level 1, directed.  With
    10 arcs per neighbour row the level-1 rows hold few enough arcs for the
    level-2 push; with 40 they hold more than the push takes and the level-2
    vertices scan their in-rows.  Parents against oracle.parents either way."""
    rng = np.random.default_rng(row_len)
    n1, n2, n3 = 2000, 3000, 500
    n = 1 + n1 + n2 + n3
    lv1 = np.arange(1, 1 + n1)
    lv2 = np.arange(1 + n1, 1 + n1 + n2)
    lv3 = np.arange(1 + n1 + n2, n)
    dup = rng.choice(lv1, 40, replace=False)                    # 2,040 arcs in the source row
    src = [np.zeros(n1 + dup.size, np.int64)]
    dst = [np.r_[lv1, dup]]
    u = np.repeat(lv1, row_len)                                  # level 1 -> level 2 (overlapping, repeats)
    v = rng.choice(lv2, u.size)
    v[::7] = rng.choice(lv1, v[::7].size)                         # and some back into level 1
    src.append(u); dst.append(v)
    w = rng.choice(lv2, 4000)                                    # level 2 -> level 3
    src.append(w); dst.append(rng.choice(lv3, w.size))
    g = gg.from_arcs(n, np.concatenate(src), np.concatenate(dst))
    assert g.row_ptr[1] - g.row_ptr[0] == n1 + dup.size <= 2048
    h = upload(dawn, g)
    try:
        d_want, p_want = want(g, 0)
        assert (d_want == 2).sum() > 1000
        for run in (run_host, run_device):
            dist, par = run(dawn, h, n, 0)
            np.testing.assert_array_equal(dist, d_want)
            np.testing.assert_array_equal(par, p_want)
    finally:
        dawn.dawn_graph_free(h)
