"""dawn_sssp_noalloc, the allocation-free single-source entry point.

It serves callers that cannot call cudaMalloc (a framework allocator that
already holds the device memory they may use, or a request path that must not
allocate after start-up): its work buffers live in a fixed device array inside
the library.  This test calls it through the C ABI and checks its output
against dawn_sssp on the same graph, bit for bit (distances are integers, the
tolerance is zero), on two calls in a row, so that contents left behind by the
first call cannot leak into the second.  The file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2208_04514_b300 import graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_matches_dawn_sssp_twice(dawn):
    g = gg.rmat(16, seed=2)
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC)
    try:
        rp = torch.from_numpy(g.row_ptr).cuda()
        ci = torch.from_numpy(g.col_idx).cuda()
        srcs = gg.sample_sources(g, 2, seed=11)
        ref = torch.empty(g.n, dtype=torch.int32, device="cuda")
        got = torch.full((g.n,), -9, dtype=torch.int32, device="cuda")
        for s in srcs:  # two calls in a row, different sources
            dawn.dawn_sssp(h, int(s), ref)
            dawn.dawn_sssp_noalloc(rp, ci, int(s), got)
            np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())
    finally:
        dawn.dawn_graph_free(h)


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
