"""Centrality parity: dawn_centrality (through the C ABI) against the CPU
oracle.  ecc, distance sums, reached counts and the whole-run summary
(diameter, radius, pairs, distance total) are integers: bit-exact.
Closeness and harmonic centrality are IEEE doubles computed on both sides by
the same operations in the same order (harmonic: vertices at distance d over
d, added in ascending d), so they are compared bit for bit as well.

Covers both batched kernels (the sliced one, which counts each pass's
levels from its level bits, and the per-level one), every lane width, ragged
source counts, duplicate and isolated sources, directed graphs, a
high-diameter lattice and a path past int16 (levels beyond the sliced
kernel's level arrays: the call moves to the per-level kernel), host and
device outputs, the all-sources RMAT scale-16 workload, and bad arguments.
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


def run(dawn, h, srcs, lanes=0, device=False, kernel=0):
    k = len(srcs)
    if device:
        out = {"ecc": torch.zeros(k, dtype=torch.int32, device="cuda"),
               "dsum": torch.zeros(k, dtype=torch.int64, device="cuda"),
               "reached": torch.zeros(k, dtype=torch.int32, device="cuda"),
               "closeness": torch.zeros(k, dtype=torch.float64, device="cuda"),
               "harmonic": torch.zeros(k, dtype=torch.float64, device="cuda")}
        src = torch.from_numpy(np.asarray(srcs, dtype=np.int32)).cuda()
    else:
        out = {"ecc": np.zeros(k, np.int32), "dsum": np.zeros(k, np.int64), "reached": np.zeros(k, np.int32),
               "closeness": np.zeros(k, np.float64), "harmonic": np.zeros(k, np.float64)}
        src = np.asarray(srcs, dtype=np.int32)
    summ = dawn.dawn_centrality(h, src, k, out["ecc"], out["dsum"], out["reached"], out["closeness"],
                                out["harmonic"], {"lanes": lanes, "kernel": kernel})
    if device:
        out = {key: v.cpu().numpy() for key, v in out.items()}
    out["summary"] = summ
    return out


def check(g, srcs, got):
    want = oracle.centrality(g.row_ptr, g.col_idx, np.asarray(srcs, dtype=np.int32))
    for key in ("ecc", "dsum", "reached"):
        np.testing.assert_array_equal(got[key], want[key], err_msg=key)
    for key in ("closeness", "harmonic"):  # same IEEE operations in the same order
        np.testing.assert_array_equal(got[key].view(np.int64), want[key].view(np.int64), err_msg=key)
    assert got["summary"] == want["summary"]


@pytest.mark.parametrize("seed", range(3))
def test_small_digraphs_all_sources(dawn, seed):
    from test_oracle_pins import random_digraph
    g = random_digraph(5200 + seed, n=int(np.random.default_rng(seed).integers(2, 80)))
    h = upload(dawn, g)
    try:
        srcs = np.arange(g.n, dtype=np.int32)
        for kernel in KERNELS:
            for lanes in (64, 128, 256):
                check(g, srcs, run(dawn, h, srcs, lanes, kernel=kernel))
    finally:
        dawn.dawn_graph_free(h)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("device", [False, True])
def test_rmat_and_directed_ragged(dawn, device, kernel):
    for g in (gg.rmat(12, seed=2), gg.rmat(11, seed=9, symmetrise=False)):
        h = upload(dawn, g)
        try:
            deg = g.out_degree()
            srcs = np.random.default_rng(3).integers(0, g.n, 300).astype(np.int32)
            srcs[:3] = srcs[3]
            if (deg == 0).any():
                srcs[10] = int(np.nonzero(deg == 0)[0][0])
            srcs[11] = int(np.argmax(deg))
            check(g, srcs, run(dawn, h, srcs, 256, device, kernel))
        finally:
            dawn.dawn_graph_free(h)


def test_long_path_past_int16(dawn):
    """40,000-vertex path: distances past 32767 are fine (no rows stored)."""
    n = 40000
    s = np.arange(n - 1)
    g = gg.from_arcs(n, np.r_[s, s + 1], np.r_[s + 1, s], symmetric=True)
    h = upload(dawn, g)
    try:
        srcs = np.array([0, n // 2, n - 1], dtype=np.int32)
        got = run(dawn, h, srcs, 64)  # the sliced kernel stops at level 16 and the per-level one runs
        check(g, srcs, got)
        assert got["ecc"].tolist() == [n - 1, n // 2, n - 1]
        with pytest.raises(dawn.DawnError) as ei:  # asked for by name, the sliced kernel reports it
            run(dawn, h, srcs, 64, kernel=1)
        assert ei.value.code == dawn.DAWN_E_INVALID
    finally:
        dawn.dawn_graph_free(h)


def test_lattice_all_sources_summary(dawn):
    w = 48
    g = gg.lattice(w, w, 0.0, seed=0)
    h = upload(dawn, g)
    try:
        srcs = np.arange(g.n, dtype=np.int32)
        got = run(dawn, h, srcs, 256)
        check(g, srcs, got)
        assert got["summary"]["diameter"] == 2 * (w - 1)
        assert got["summary"]["radius"] == 2 * (w // 2)  # centre of an even lattice: (w/2) + (w/2)
    finally:
        dawn.dawn_graph_free(h)


def test_rmat16_all_sources(dawn):
    """All 65,536 sources of the RMAT scale-16 workload: integers against the
    component sizes and 1,024 sampled sources against the oracle."""
    g = gg.rmat(16, seed=4)
    h = upload(dawn, g)
    try:
        srcs = np.arange(g.n, dtype=np.int32)
        got = run(dawn, h, srcs, 256, device=True)
        lab = oracle.wcc(g.row_ptr, g.col_idx)
        np.testing.assert_array_equal(got["reached"], np.bincount(lab, minlength=g.n)[lab])
        sample = np.random.default_rng(5).choice(g.n, 1024, replace=False).astype(np.int32)
        want = oracle.centrality(g.row_ptr, g.col_idx, sample)
        for key in ("ecc", "dsum", "reached"):
            np.testing.assert_array_equal(got[key][sample], want[key])
        for key in ("closeness", "harmonic"):
            np.testing.assert_array_equal(got[key][sample].view(np.int64), want[key].view(np.int64))
        assert got["summary"]["pairs"] == int((got["reached"].astype(np.int64) - 1).sum())
    finally:
        dawn.dawn_graph_free(h)


def test_bad_arguments(dawn):
    g = gg.rmat(9, seed=1)
    h = upload(dawn, g)
    try:
        with pytest.raises(dawn.DawnError) as ei:
            dawn.dawn_centrality(h, np.array([0, g.n], dtype=np.int32))
        assert ei.value.code == dawn.DAWN_E_INVALID
        with pytest.raises(dawn.DawnError):
            dawn.dawn_centrality(h, np.array([0], dtype=np.int32), opts={"lanes": 32})
    finally:
        dawn.dawn_graph_free(h)
