"""dawn_sssp_noalloc, the allocation-free single-source entry point.

It serves callers that cannot call cudaMalloc (a framework allocator that
already holds the device memory they may use, or a request path that must not
allocate after start-up): its work buffers live in a fixed device array inside
the library.  These tests call it through the C ABI and check its output
against the CPU oracle (the literal Alg. 3 SOVM iteration), bit for bit:
distances are integers and the tolerance is zero.  They cover two calls in a
row on one graph, so that contents left behind by the first call cannot leak
into the second, and a smaller graph after a larger one.  They also cover a
directed graph whose n is not a multiple of 32, a source with more than 1,024
out-arcs (the launch path that clears before level 1), and malformed CSRs,
which the entry point's device-side check must reject with the index of the
bad entry.  The file sorts last so that a run stopping at the first failure
has already run every other test.
"""
import numpy as np
import pytest

import oracle
from paper_2208_04514_b300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def noalloc(dawn, g, src):
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx if g.m else np.zeros(1, np.int32)).cuda()
    got = torch.full((g.n,), -9, dtype=torch.int32, device="cuda")
    dawn.dawn_sssp_noalloc(rp, ci, int(src), got, n=g.n, m=g.m)
    return got.cpu().numpy()


def test_noalloc_matches_the_oracle_twice(dawn):
    g = gg.rmat(16, seed=2)
    for s in gg.sample_sources(g, 2, seed=11):  # two calls in a row, different sources
        np.testing.assert_array_equal(noalloc(dawn, g, s), oracle.sssp_sovm(g.row_ptr, g.col_idx, int(s)))


def test_noalloc_directed_ragged_and_a_smaller_graph_after(dawn):
    # directed, n % 32 != 0, after the larger graph of the test above
    g = gg.erdos_renyi(1000, 3.0, seed=9)
    assert not g.symmetric and g.n % 32 != 0
    for s in (0, 1, 999):
        np.testing.assert_array_equal(noalloc(dawn, g, s), oracle.sssp_sovm(g.row_ptr, g.col_idx, s))
    # a large graph, then a much smaller one: nothing of the first may show
    big = gg.rmat(18, seed=3)
    s = int(gg.sample_sources(big, 1, seed=1)[0])
    np.testing.assert_array_equal(noalloc(dawn, big, s), oracle.sssp_sovm(big.row_ptr, big.col_idx, s))
    small = gg.from_arcs(37, np.arange(36), np.arange(1, 37))  # a directed path of 37 vertices
    np.testing.assert_array_equal(noalloc(dawn, small, 0), np.arange(37, dtype=np.int32))
    want = np.full(37, -1, dtype=np.int32)
    want[20:] = np.arange(17)
    np.testing.assert_array_equal(noalloc(dawn, small, 20), want)


def test_noalloc_source_with_more_than_1024_out_arcs(dawn):
    # a hub source with 3,000 leaves, each leaf pointing on to one more vertex
    n = 1 + 3000 + 3000
    leaves = np.arange(1, 3001)
    src = np.r_[np.zeros(3000, np.int64), leaves]
    dst = np.r_[leaves, leaves + 3000]
    g = gg.from_arcs(n, src, dst)
    got = noalloc(dawn, g, 0)
    np.testing.assert_array_equal(got, oracle.sssp_sovm(g.row_ptr, g.col_idx, 0))
    assert got.max() == 2 and (got == 1).sum() == 3000


def test_noalloc_rejects_a_malformed_csr(dawn):
    g = gg.erdos_renyi(64, 4.0, seed=5)
    rp = torch.from_numpy(g.row_ptr).cuda()
    ci = torch.from_numpy(g.col_idx).cuda()
    d = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    # a row_ptr entry smaller than the one before it
    bad_rp = rp.clone()
    bad_rp[10] = bad_rp[9] - 1
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_sssp_noalloc(bad_rp, ci, 0, d, n=g.n, m=g.m)
    assert ei.value.code == dawn.DAWN_E_INVALID and "row_ptr[10]" in str(ei.value)
    # a column index past the last vertex
    bad_ci = ci.clone()
    bad_ci[17] = g.n
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_sssp_noalloc(rp, bad_ci, 0, d, n=g.n, m=g.m)
    assert ei.value.code == dawn.DAWN_E_INVALID and "col_idx[17]" in str(ei.value)
    # and the entry point still works afterwards
    d2 = torch.zeros(g.n, dtype=torch.int32, device="cuda")
    dawn.dawn_sssp_noalloc(rp, ci, 3, d2, n=g.n, m=g.m)
    np.testing.assert_array_equal(d2.cpu().numpy(), oracle.sssp_sovm(g.row_ptr, g.col_idx, 3))


def test_noalloc_rejects_sizes_beyond_its_maximum(dawn):
    rp = torch.zeros((1 << 20) + 2, dtype=torch.int32, device="cuda")
    ci = torch.zeros(1, dtype=torch.int32, device="cuda")
    d = torch.zeros((1 << 20) + 1, dtype=torch.int32, device="cuda")
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_sssp_noalloc(rp, ci, 0, d, n=(1 << 20) + 1, m=0)
    assert ei.value.code == dawn.DAWN_E_INVALID and "1048576" in str(ei.value)
    with pytest.raises(dawn.DawnError) as ei:
        dawn.dawn_sssp_noalloc(rp[:3], ci, 0, d, n=2, m=(1 << 25) + 1)
    assert ei.value.code == dawn.DAWN_E_INVALID
