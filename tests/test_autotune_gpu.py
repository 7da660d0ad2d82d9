"""Autotuner: settings are measured, stored on the handle, cached per graph
class and GPU, and never change a result."""
import numpy as np
import pytest

import oracle
from paper_2208_04514_b300 import autotune, graphgen as gg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_autotune_cache_and_results_unchanged(dawn, tmp_path):
    g = gg.rmat(14, seed=2)
    h = dawn.dawn_graph_upload(g.row_ptr, g.col_idx, flags=dawn.DAWN_SYMMETRIC)
    try:
        sample = gg.sample_sources(g, 8, seed=1)
        t = autotune.tuned(h, g.row_ptr, g.col_idx, True, sample, cache=tmp_path / "t.json")
        assert t["cached"] is False and t["lanes"] in (64, 128, 256) and t["alpha"] > 0 and t["sssp_us"] > 0
        t2 = autotune.tuned(h, g.row_ptr, g.col_idx, True, sample, cache=tmp_path / "t.json")
        assert t2["cached"] is True and t2["alpha"] == t["alpha"] and t2["lanes"] == t["lanes"]
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for s in sample[:4]:
            dawn.dawn_sssp(h, int(s), d)
            np.testing.assert_array_equal(d.cpu().numpy(), oracle.sssp_sovm(g.row_ptr, g.col_idx, int(s)))
        ecc = np.zeros(8, dtype=np.int32)
        dawn.dawn_msbfs_ex(h, sample, 8, None, 2, 0, ecc, None, None)
        _, want_ecc, _, _ = oracle.msbfs(g.row_ptr, g.col_idx, sample, keep_dist=False)
        np.testing.assert_array_equal(ecc, want_ecc)
        with pytest.raises(dawn.DawnError):
            dawn.dawn_set_tuning(h, {"lanes": 100})
    finally:
        dawn.dawn_graph_free(h)
