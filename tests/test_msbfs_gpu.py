"""Bit-lane multi-source parity: dawn_msbfs (through the C ABI) against the CPU
oracle's SOVM-per-source batch (Sec. 3.3, APSP as one SSSP per source),
element by element.  Distances are integers: bit-exact.

Covers both kernels (DAWN_MSBFS_SLICED and DAWN_MSBFS_PER_LEVEL), every lane
width (64/128/256), int16 and int32 blocks, both layouts, host and device
outputs, ragged source counts (not a multiple of 64), duplicate and isolated
sources, directed graphs (pull over the in-adjacency), rows split into pieces
(a star's hub), more levels than the sliced kernel's first planes hold, the
full-size RMAT scale-16 all-sources workload (1,024 sampled rows bit-exact,
every source's reached count = its component size), the int16 overflow
report and the bounded-wait timeout.
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


KERNELS = [1, 2]  # DAWN_MSBFS_SLICED, DAWN_MSBFS_PER_LEVEL


def run(dawn, h, n, srcs, lanes, dist_bytes=2, layout=0, device=True, with_block=True, kernel=0):
    k = len(srcs)
    dt = torch.int16 if dist_bytes == 2 else torch.int32
    shape = (k, n) if layout == 0 else (n, k)
    if device:
        block = torch.full(shape, 77, dtype=dt, device="cuda") if with_block else None
        ecc = torch.zeros(k, dtype=torch.int32, device="cuda")
        dsum = torch.zeros(k, dtype=torch.int64, device="cuda")
        reached = torch.zeros(k, dtype=torch.int32, device="cuda")
        src = torch.from_numpy(np.asarray(srcs, dtype=np.int32)).cuda()
    else:
        block = np.full(shape, 77, dtype=np.int16 if dist_bytes == 2 else np.int32) if with_block else None
        ecc = np.zeros(k, dtype=np.int32)
        dsum = np.zeros(k, dtype=np.int64)
        reached = np.zeros(k, dtype=np.int32)
        src = np.asarray(srcs, dtype=np.int32)
    dawn.dawn_msbfs_ex(h, src, k, block, dist_bytes, layout, ecc, dsum, reached, {"lanes": lanes, "kernel": kernel})
    conv = (lambda x: x.cpu().numpy()) if device else (lambda x: x)
    b = None
    if with_block:
        b = conv(block).astype(np.int64)
        if layout == 1:
            b = b.T
    return b, conv(ecc), conv(dsum), conv(reached)


def check(g, srcs, got, with_block=True):
    want_block, want_ecc, want_dsum, want_reached = oracle.msbfs(g.row_ptr, g.col_idx, srcs, keep_dist=with_block)
    b, ecc, dsum, reached = got
    if with_block:
        np.testing.assert_array_equal(b, want_block)
    np.testing.assert_array_equal(ecc, want_ecc)
    np.testing.assert_array_equal(dsum, want_dsum)
    np.testing.assert_array_equal(reached, want_reached)


@pytest.mark.parametrize("seed", range(4))
def test_small_digraphs_all_sources(dawn, seed):
    from test_oracle_pins import random_digraph
    g = random_digraph(7000 + seed, n=int(np.random.default_rng(seed).integers(2, 70)))
    h = upload(dawn, g)
    try:
        srcs = np.arange(g.n, dtype=np.int32)
        for kernel in KERNELS:
            for lanes in (64, 128, 256):
                check(g, srcs, run(dawn, h, g.n, srcs, lanes, kernel=kernel))
    finally:
        dawn.dawn_graph_free(h)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("lanes", [64, 128, 256])
@pytest.mark.parametrize("dist_bytes,layout,device", [(2, 0, True), (4, 0, True), (2, 1, True),
                                                       (4, 1, False), (2, 0, False)])
def test_rmat12_ragged_batches(dawn, lanes, dist_bytes, layout, device, kernel):
    g = gg.rmat(12, seed=2)
    deg = g.out_degree()
    rng = np.random.default_rng(lanes + dist_bytes)
    srcs = rng.integers(0, g.n, 300).astype(np.int32)        # 300: not a multiple of 64
    srcs[:3] = srcs[3]                                        # duplicates
    srcs[10] = int(np.nonzero(deg == 0)[0][0])                # an isolated source
    srcs[11] = int(np.argmax(deg))                            # the largest hub
    h = upload(dawn, g)
    try:
        check(g, srcs, run(dawn, h, g.n, srcs, lanes, dist_bytes, layout, device, kernel=kernel))
    finally:
        dawn.dawn_graph_free(h)


def test_directed_graph_batches(dawn):
    g = gg.rmat(11, seed=9, symmetrise=False)
    h = upload(dawn, g)
    try:
        srcs = np.arange(0, g.n, 7, dtype=np.int32)
        # alternating kernels on one handle: each starts from what the other left
        for kernel in (2, 1, 2, 1):
            for lanes in (64, 256):
                check(g, srcs, run(dawn, h, g.n, srcs, lanes, kernel=kernel))
    finally:
        dawn.dawn_graph_free(h)


def test_split_rows_and_short_rows(dawn):
    """A star whose hub has 5,000 in-arcs (a row cut into pieces), leaves of
    in-degree 1..3 (one vertex per lane), a tail of 20 mid-degree rows and
    isolated vertices, directed: the pieces' shared-memory OR and the slices
    against the oracle, from hub, leaf, tail and isolated sources."""
    rng = np.random.default_rng(3)
    nleaf, ntail = 5000, 20
    n = 1 + nleaf + ntail + 7
    leaves = np.arange(1, nleaf + 1)
    tail = np.arange(nleaf + 1, nleaf + 1 + ntail)
    src = [leaves, np.zeros(nleaf, np.int64)]  # leaf -> hub
    dst = [np.zeros(nleaf, np.int64), leaves]  # hub -> leaf
    extra = rng.integers(1, nleaf + 1, (3000, 2))  # leaf -> leaf, in-degree up to a few
    src.append(extra[:, 0]); dst.append(extra[:, 1])
    for i, t in enumerate(tail):  # tail vertex t: in-arcs from 40 + i leaves, out-arc to the next
        fr = rng.choice(leaves, 40 + i, replace=False)
        src.append(fr); dst.append(np.full(fr.size, t))
        if i + 1 < ntail:
            src.append([t]); dst.append([t + 1])
    g = gg.from_arcs(n, np.concatenate(src), np.concatenate(dst))
    h = upload(dawn, g)
    try:
        srcs = np.r_[0, 1, 2, tail[0], tail[-1], n - 1, rng.integers(0, n, 100)].astype(np.int32)
        for kernel in KERNELS:
            check(g, srcs, run(dawn, h, g.n, srcs, 128, kernel=kernel))
    finally:
        dawn.dawn_graph_free(h)


def test_more_levels_than_first_planes(dawn):
    """A path of 700 vertices: 699 levels, past the 255 that the sliced
    kernel's first planes hold; it widens them and runs the call again."""
    n = 700
    s = np.arange(n - 1)
    g = gg.from_arcs(n, np.r_[s, s + 1], np.r_[s + 1, s], symmetric=True)
    h = upload(dawn, g)
    try:
        srcs = np.array([0, 350, n - 1, 5], dtype=np.int32)
        for dist_bytes in (2, 4):
            check(g, srcs, run(dawn, h, n, srcs, 64, dist_bytes, kernel=1))
    finally:
        dawn.dawn_graph_free(h)


def test_reductions_without_block(dawn):
    g = gg.rmat(12, seed=5)
    h = upload(dawn, g)
    try:
        srcs = np.random.default_rng(1).integers(0, g.n, 700).astype(np.int32)
        check(g, srcs, run(dawn, h, g.n, srcs, 256, with_block=False), with_block=False)
    finally:
        dawn.dawn_graph_free(h)


def test_lattice_closed_form(dawn):
    """Bond-complete lattice: dist = Manhattan distance, ecc from a corner 2(W-1)."""
    w = 40
    g = gg.lattice(w, w, 0.0, seed=0)
    h = upload(dawn, g)
    try:
        srcs = np.arange(0, g.n, 13, dtype=np.int32)
        b, ecc, dsum, reached = run(dawn, h, g.n, srcs, 128, 4)
        r, c = np.divmod(np.arange(g.n), w)
        for i, s in enumerate(srcs):
            sr, sc = divmod(int(s), w)
            np.testing.assert_array_equal(b[i], np.abs(r - sr) + np.abs(c - sc))
        assert ecc[0] == 2 * (w - 1)
        assert (reached == g.n).all()
    finally:
        dawn.dawn_graph_free(h)


def test_int16_overflow_is_reported(dawn):
    n = 40000
    s = np.arange(n - 1)
    g = gg.from_arcs(n, np.r_[s, s + 1], np.r_[s + 1, s], symmetric=True)
    h = upload(dawn, g)
    try:
        with pytest.raises(dawn.DawnError) as ei:
            run(dawn, h, n, np.array([0], dtype=np.int32), 64, 2)
        assert ei.value.code == dawn.DAWN_E_OVERFLOW
        b, ecc, dsum, reached = run(dawn, h, n, np.array([0, n - 1], dtype=np.int32), 64, 4)
        assert ecc.tolist() == [n - 1, n - 1]
        assert dsum[0] == n * (n - 1) // 2
        np.testing.assert_array_equal(b[1], n - 1 - np.arange(n))
    finally:
        dawn.dawn_graph_free(h)


def test_bad_arguments_and_timeout(dawn):
    g = gg.rmat(10, seed=3)
    h = upload(dawn, g)
    try:
        src = np.array([0, 1, 2], dtype=np.int32)
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_msbfs_ex(h, np.array([0, g.n], dtype=np.int32), 2, None, 2, 0, None, None, None)
        assert ei.value.code == dawn.DAWN_E_INVALID
        for bad in ({"lanes": 96}, {"lanes": 512}):
            with pytest.raises(dawn.DawnError):
                dawn.dawn_msbfs_ex(h, src, 3, None, 2, 0, None, None, None, bad)
        with pytest.raises(dawn.DawnError):
            dawn.dawn_msbfs_ex(h, src, 3, None, 3, 0, None, None, None)
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_msbfs_ex(h, src, 3, None, 2, 0, None, None, None, {"kernel": 3})
        assert ei.value.code == dawn.DAWN_E_INVALID
        for kernel in KERNELS:
            with pytest.raises(dawn.DawnError) as ei:
                dawn.dawn_msbfs_ex(h, src, 3, None, 2, 0, None, None, None, {"spin_limit": 1, "kernel": kernel})
            assert ei.value.code == dawn.DAWN_E_TIMEOUT
            check(g, src, run(dawn, h, g.n, src, 64, kernel=kernel))  # usable again afterwards
    finally:
        dawn.dawn_graph_free(h)


def test_rmat16_all_sources_full_size(dawn):
    """The batched all-sources workload: RMAT scale 16, every vertex a source,
    256 lanes per pass.  1,024 sampled rows bit-exact against the oracle; for
    every source, reached = size of its (weak = strong, symmetric) component."""
    g = gg.rmat(16, seed=4)
    n = g.n
    h = upload(dawn, g)
    try:
        srcs = np.arange(n, dtype=np.int32)
        ecc = np.zeros(n, dtype=np.int32)
        dsum = np.zeros(n, dtype=np.int64)
        reached = np.zeros(n, dtype=np.int32)
        dawn.dawn_msbfs_ex(h, torch.from_numpy(srcs).cuda(), n, None, 2, 0, ecc, dsum, reached, {"lanes": 256})
        lab = oracle.wcc(g.row_ptr, g.col_idx)
        comp = np.bincount(lab, minlength=n)
        np.testing.assert_array_equal(reached, comp[lab])
        sample = np.random.default_rng(5).choice(n, 1024, replace=False).astype(np.int32)
        b, e2, d2, r2 = run(dawn, h, n, sample, 256, 2)
        check(g, sample, (b, e2, d2, r2))
        np.testing.assert_array_equal(ecc[sample], e2)
        np.testing.assert_array_equal(dsum[sample], d2)
    finally:
        dawn.dawn_graph_free(h)


def test_rmat20_sliced_long_pieces(dawn):
    """RMAT scale 20: the sliced kernel's row pieces are longer than on the
    small graphs (the piece length grows with the arcs per warp) and CTAs own
    many split rows.  256 sampled sources: every source's reached count is the
    size of its component, and 4 rows against Alg. 2 (FIFO BFS), bit-exact,
    for both kernels."""
    g = gg.rmat(20, 16, 0.57, 0.19, 0.19, seed=2, symmetrise=True)
    n = g.n
    h = upload(dawn, g)
    try:
        srcs = gg.sample_sources(g, 256, seed=9).astype(np.int32)
        lab = oracle.wcc(g.row_ptr, g.col_idx)
        comp = np.bincount(lab, minlength=n)
        for kernel in KERNELS:
            block = torch.full((256, n), 77, dtype=torch.int16, device="cuda")
            reached = torch.zeros(256, dtype=torch.int32, device="cuda")
            ecc = torch.zeros(256, dtype=torch.int32, device="cuda")
            dawn.dawn_msbfs_ex(h, torch.from_numpy(srcs).cuda(), 256, block, 2, 0, ecc, None, reached,
                               {"lanes": 256, "kernel": kernel})
            np.testing.assert_array_equal(reached.cpu().numpy(), comp[lab[srcs]])
            rows = block[:4].cpu().numpy().astype(np.int32)
            for i in range(4):
                want = oracle.bfs_queue(g.row_ptr, g.col_idx, int(srcs[i]))
                np.testing.assert_array_equal(rows[i], want)
                assert ecc[i].item() == want.max()
            del block
    finally:
        dawn.dawn_graph_free(h)
