"""Pins for the CPU oracle: each check ties it to something other than itself.

* closed forms (path, directed cycle, star, complete graph, bond-complete
  lattice with Manhattan distance, binary tree, empty graph, n = 1);
* brute force on tiny digraphs: Floyd-Warshall and scipy's unweighted
  shortest_path (a library routine), both against Alg. 3, Alg. 1 and Alg. 2;
* Thm 1 / Lemma 1 evaluated independently with numpy integer matrix powers
  (path counts), against the oracle's Boolean-power routine;
* the SOVM cost identity of Sec. 3.3: edges examined = sum of out-degrees of
  the reached vertices;
* the certificate: accepts exact vectors, rejects every planted off-by-one;
* WCC labels against scipy's connected_components.

Run against a mutant (``DAWN_ORACLE_SO``) by ``test_oracle_mutants.py``.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components, csgraph_from_dense, shortest_path

import oracle
from paper_2208_04514_b300 import graphgen as gg

RNG_SEEDS = list(range(40))


def random_digraph(seed, n=None, p=None, loops=True, dups=True):
    rng = np.random.default_rng(seed)
    n = n or int(rng.integers(1, 48))
    p = p if p is not None else float(rng.uniform(0.0, 0.25))
    mask = rng.random((n, n)) < p
    if not loops:
        np.fill_diagonal(mask, False)
    src, dst = np.nonzero(mask)
    if dups and src.size:
        k = int(rng.integers(0, src.size + 1))
        pick = rng.integers(0, src.size, k)
        src = np.concatenate([src, src[pick]])
        dst = np.concatenate([dst, dst[pick]])
    return gg.from_arcs(n, src, dst, f"rand{seed}")


def scipy_dist(g, src):
    n = g.n
    a = sp.csr_matrix((np.ones(g.m), g.col_idx, g.row_ptr), shape=(n, n))
    d = shortest_path(a, directed=True, unweighted=True, indices=[src])[0]
    out = np.where(np.isinf(d), -1, d).astype(np.int64)
    return out


def all_oracle_sssp(g, src):
    t = gg.transpose(g)
    return (oracle.sssp_sovm(g.row_ptr, g.col_idx, src),
            oracle.sssp_bovm(t.row_ptr, t.col_idx, src),
            oracle.bfs_queue(g.row_ptr, g.col_idx, src))


# ------------------------------------------------------------ closed forms --

def path_graph(n, directed):
    s = np.arange(n - 1)
    if directed:
        return gg.from_arcs(n, s, s + 1)
    return gg.from_arcs(n, np.r_[s, s + 1], np.r_[s + 1, s], symmetric=True)


@pytest.mark.parametrize("n", [1, 2, 7, 33])
def test_path_closed_form(n):
    g = path_graph(n, directed=False)
    for src in {0, n // 2, n - 1}:
        want = np.abs(np.arange(n) - src)
        for d in all_oracle_sssp(g, src):
            np.testing.assert_array_equal(d, want)
    gd = path_graph(n, directed=True)
    for src in {0, n // 2, n - 1}:
        want = np.where(np.arange(n) >= src, np.arange(n) - src, -1)
        for d in all_oracle_sssp(gd, src):
            np.testing.assert_array_equal(d, want)


@pytest.mark.parametrize("n", [2, 5, 40])
def test_directed_cycle_closed_form(n):
    s = np.arange(n)
    g = gg.from_arcs(n, s, (s + 1) % n)
    for src in range(0, n, max(1, n // 5)):
        want = (np.arange(n) - src) % n
        for d in all_oracle_sssp(g, src):
            np.testing.assert_array_equal(d, want)


def test_star_and_complete():
    n = 17
    leaves = np.arange(1, n)
    star = gg.from_arcs(n, np.r_[np.zeros(n - 1, int), leaves], np.r_[leaves, np.zeros(n - 1, int)], symmetric=True)
    for d in all_oracle_sssp(star, 0):
        np.testing.assert_array_equal(d, np.r_[0, np.ones(n - 1, int)])
    for d in all_oracle_sssp(star, 5):
        want = np.full(n, 2)
        want[0], want[5] = 1, 0
        np.testing.assert_array_equal(d, want)
    i, j = np.nonzero(~np.eye(n, dtype=bool))
    comp = gg.from_arcs(n, i, j, symmetric=True)
    for d in all_oracle_sssp(comp, 3):
        want = np.ones(n, int)
        want[3] = 0
        np.testing.assert_array_equal(d, want)


@pytest.mark.parametrize("w", [1, 2, 9, 24])
def test_bond_complete_lattice_is_manhattan(w):
    g = gg.lattice(w, w, p_delete=0.0, seed=0)
    assert g.m == 4 * w * (w - 1)
    r, c = np.divmod(np.arange(w * w), w)
    for src in {0, w * w - 1, (w // 2) * w + w // 3}:
        sr, sc = divmod(src, w)
        want = np.abs(r - sr) + np.abs(c - sc)
        for d in all_oracle_sssp(g, src):
            np.testing.assert_array_equal(d, want)
    _, ecc, dsum, reached = oracle.msbfs(g.row_ptr, g.col_idx, [0], keep_dist=False)
    assert ecc[0] == 2 * (w - 1)
    assert dsum[0] == w * w * (w - 1)  # sum over r,c of r + c
    assert reached[0] == w * w


def test_binary_tree_depths():
    n = 100
    child = np.arange(1, n)
    parent = (child - 1) // 2
    g = gg.from_arcs(n, np.r_[parent, child], np.r_[child, parent], symmetric=True)
    want = np.floor(np.log2(np.arange(n) + 1)).astype(int)
    for d in all_oracle_sssp(g, 0):
        np.testing.assert_array_equal(d, want)


def test_empty_and_single():
    g = gg.from_arcs(6, [], [])
    for d in all_oracle_sssp(g, 4):
        np.testing.assert_array_equal(d, [-1, -1, -1, -1, 0, -1])
    g1 = gg.from_arcs(1, [0], [0])  # one vertex with a self-loop
    for d in all_oracle_sssp(g1, 0):
        np.testing.assert_array_equal(d, [0])


# -------------------------------------------------- brute force, n <= 48 --

@pytest.mark.parametrize("seed", RNG_SEEDS)
def test_random_digraphs_vs_floyd_and_scipy(seed):
    g = random_digraph(seed)
    fw = oracle.apsp_floyd(g.row_ptr, g.col_idx)
    for src in range(g.n):
        ref = scipy_dist(g, src)
        np.testing.assert_array_equal(fw[src], ref)
        for d in all_oracle_sssp(g, src):
            np.testing.assert_array_equal(d, ref)


def numpy_path_count_distances(g):
    """Thm 1 from Lemma 1: (A^k)_ij counts i->j walks of length k; the
    distance is the first k >= 1 with a non-zero count (i != j)."""
    n = g.n
    a = np.zeros((n, n), dtype=np.float64)
    np.add.at(a, (np.repeat(np.arange(n), g.out_degree()), g.col_idx), 1.0)
    a = (a > 0).astype(np.float64)
    d = np.full((n, n), -1, dtype=np.int64)
    np.fill_diagonal(d, 0)
    p = a.copy()
    for k in range(1, n):
        hit = (p > 0) & (d == -1)
        d[hit] = k
        p = np.minimum(p @ a, 1e6)  # counts capped: only non-zero-ness matters
    return d


@pytest.mark.parametrize("seed", RNG_SEEDS[:20])
def test_boolean_powers_definition(seed):
    g = random_digraph(1000 + seed, n=int(np.random.default_rng(seed).integers(2, 30)))
    want = numpy_path_count_distances(g)
    np.testing.assert_array_equal(oracle.apsp_powers(g.row_ptr, g.col_idx), want)
    for src in range(g.n):
        np.testing.assert_array_equal(oracle.sssp_sovm(g.row_ptr, g.col_idx, src), want[src])


# ----------------------------------------------------------- cost identity --

@pytest.mark.parametrize("seed", RNG_SEEDS[:10])
def test_sovm_edge_visits_identity(seed):
    g = random_digraph(2000 + seed, n=40)
    deg = g.out_degree()
    for src in range(0, g.n, 3):
        d, visits, levels = oracle.sssp_sovm(g.row_ptr, g.col_idx, src, with_stats=True)
        assert visits == int(deg[d >= 0].sum())
        assert levels == int(d.max())


def test_edge_visits_identity_er():
    g = gg.erdos_renyi(1024, 8.0, seed=1)
    deg = g.out_degree()
    for src in range(4):
        d, visits, levels = oracle.sssp_sovm(g.row_ptr, g.col_idx, src, with_stats=True)
        assert visits == int(deg[d >= 0].sum())


# ------------------------------------------------------------- certificate --

@pytest.mark.parametrize("seed", RNG_SEEDS[:15])
def test_certificate_accepts_exact_rejects_planted(seed):
    g = random_digraph(3000 + seed, n=45, p=0.06)
    rng = np.random.default_rng(seed)
    for src in range(0, g.n, 4):
        d = scipy_dist(g, src).astype(np.int32)
        assert oracle.certificate(g.row_ptr, g.col_idx, src, d) == (0, -1)
        for v in rng.choice(g.n, size=min(8, g.n), replace=False):
            for delta in (-1, 1):
                bad = d.copy()
                if bad[v] == -1 and delta == -1:
                    continue
                bad[v] = bad[v] + delta if bad[v] >= 0 else 1
                if v == src and bad[v] < 0:
                    bad[v] = 1
                assert oracle.certificate(g.row_ptr, g.col_idx, src, bad)[0] != 0
            if d[v] >= 0:
                bad = d.copy()
                bad[v] = -1
                assert oracle.certificate(g.row_ptr, g.col_idx, src, bad)[0] != 0


def test_certificate_on_er_and_lattice():
    for g in (gg.erdos_renyi(1024, 8.0, seed=1), gg.lattice(64, 64, 0.1, seed=3)):
        for src in range(3):
            d = oracle.bfs_queue(g.row_ptr, g.col_idx, src)
            np.testing.assert_array_equal(d, scipy_dist(g, src))
            assert oracle.certificate(g.row_ptr, g.col_idx, src, d)[0] == 0


# --------------------------------------------------------------------- WCC --

@pytest.mark.parametrize("seed", RNG_SEEDS[:10])
def test_wcc_vs_scipy(seed):
    g = random_digraph(4000 + seed, n=60, p=0.02)
    lab = oracle.wcc(g.row_ptr, g.col_idx)
    a = sp.csr_matrix((np.ones(g.m), g.col_idx, g.row_ptr), shape=(g.n, g.n))
    _, ref = connected_components(a, directed=True, connection="weak")
    # same partition: labels equal iff scipy labels equal
    assert ((lab[:, None] == lab[None, :]) == (ref[:, None] == ref[None, :])).all()
    # label is the smallest id in the component
    for c in np.unique(lab):
        assert c == np.nonzero(lab == c)[0].min()


def test_unreachable_outside_wcc_symmetric():
    g = gg.rmat(10, seed=7)
    lab = oracle.wcc(g.row_ptr, g.col_idx)
    for src in (0, 1, 2, 3, 4):
        d = oracle.sssp_sovm(g.row_ptr, g.col_idx, src)
        np.testing.assert_array_equal(d >= 0, lab == lab[src])


# ----------------------------------------------------------------- batches --

def test_msbfs_matches_scipy_rows():
    g = gg.rmat(9, seed=11)
    srcs = np.array([0, 5, 17, 100, 511], dtype=np.int32)
    block, ecc, dsum, reached = oracle.msbfs(g.row_ptr, g.col_idx, srcs)
    for i, s in enumerate(srcs):
        ref = scipy_dist(g, int(s))
        np.testing.assert_array_equal(block[i], ref)
        fin = ref[ref >= 0]
        assert ecc[i] == fin.max() and dsum[i] == fin.sum() and reached[i] == fin.size


# ---------------------------------------------------------- golden fixtures --

def test_golden_fixtures():
    """Small hand-derived graphs under tests/golden (derivations in the files)."""
    from pathlib import Path
    gdir = Path(__file__).parent / "golden"
    files = sorted(gdir.glob("hand_*.txt"))
    assert files, "no golden fixtures"
    for f in files:
        n, arcs, cases = parse_golden(f)
        g = gg.from_arcs(n, [a for a, _ in arcs], [b for _, b in arcs])
        for src, want in cases:
            for d in all_oracle_sssp(g, src):
                np.testing.assert_array_equal(d, want, err_msg=f"{f.name} src={src}")


def parse_golden(path):
    n, arcs, cases = None, [], []
    for line in path.read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, _, rest = line.partition(":")
        vals = [int(x) for x in rest.split()]
        if key == "n":
            n = vals[0]
        elif key == "arc":
            arcs.append((vals[0], vals[1]))
        elif key.startswith("dist"):
            cases.append((int(key.split()[1]), np.array(vals)))
    return n, arcs, cases


# ------------------------------------------------- shortest-path tree pins --

def lattice_parent_closed_form(w, src):
    """Full w x w lattice (id = r*w + c): the in-neighbours one step closer to
    src are the ones stepping toward it; the smallest id among them is
    id - w (from above) if r > sr, else id - 1 if c > sc, else id + 1 if
    c < sc, else id + w."""
    ids = np.arange(w * w)
    r, c = np.divmod(ids, w)
    sr, sc = divmod(src, w)
    want = np.where(r > sr, ids - w, np.where(c > sc, ids - 1, np.where(c < sc, ids + 1, ids + w)))
    want[src] = -1
    return want


def test_tree_closed_forms():
    # undirected path: the neighbour toward the source
    n = 12
    g = path_graph(n, directed=False)
    for s in (0, 5, n - 1):
        d = oracle.sssp_sovm(g.row_ptr, g.col_idx, s)
        v = np.arange(n)
        want = np.where(v > s, v - 1, v + 1)
        want[s] = -1
        np.testing.assert_array_equal(oracle.parents(g.row_ptr, g.col_idx, d), want)
    # star: from the centre every leaf hangs on 0; from a leaf, 0 hangs on it
    k = 9
    leaves = np.arange(1, k)
    star = gg.from_arcs(k, np.r_[np.zeros(k - 1, int), leaves], np.r_[leaves, np.zeros(k - 1, int)], symmetric=True)
    d = oracle.sssp_sovm(star.row_ptr, star.col_idx, 0)
    np.testing.assert_array_equal(oracle.parents(star.row_ptr, star.col_idx, d), np.r_[-1, np.zeros(k - 1, int)])
    d = oracle.sssp_sovm(star.row_ptr, star.col_idx, 4)
    want = np.zeros(k, int)
    want[0], want[4] = 4, -1
    np.testing.assert_array_equal(oracle.parents(star.row_ptr, star.col_idx, d), want)
    # complete graph: everything hangs on the source
    i, j = np.nonzero(~np.eye(k, dtype=bool))
    comp = gg.from_arcs(k, i, j, symmetric=True)
    d = oracle.sssp_sovm(comp.row_ptr, comp.col_idx, 6)
    want = np.full(k, 6)
    want[6] = -1
    np.testing.assert_array_equal(oracle.parents(comp.row_ptr, comp.col_idx, d), want)
    # binary heap tree from the root: (v - 1) // 2
    m = 60
    child = np.arange(1, m)
    t = gg.from_arcs(m, np.r_[(child - 1) // 2, child], np.r_[child, (child - 1) // 2], symmetric=True)
    d = oracle.sssp_sovm(t.row_ptr, t.col_idx, 0)
    np.testing.assert_array_equal(oracle.parents(t.row_ptr, t.col_idx, d), np.r_[-1, (child - 1) // 2])
    # bond-complete lattice, several sources (the tie-break matters everywhere off the axes)
    w = 11
    lat = gg.lattice(w, w, p_delete=0.0, seed=0)
    for s in (0, w * w - 1, 3 * w + 7, 5 * w + 5):
        d = oracle.sssp_sovm(lat.row_ptr, lat.col_idx, s)
        np.testing.assert_array_equal(oracle.parents(lat.row_ptr, lat.col_idx, d), lattice_parent_closed_form(w, s))


def brute_force_tree(g, s):
    """Enumerate every simple path from s (tiny graphs): for each v, the least
    length of a path s -> v and the set of vertices right before v on the
    paths of that length; the tree takes the smallest of that set."""
    adj = [sorted(set(g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]].tolist())) for u in range(g.n)]
    best = {s: (0, set())}

    def walk(path, on):
        u = path[-1]
        for v in adj[u]:
            if v in on:
                continue
            length = len(path)
            if v not in best or length < best[v][0]:
                best[v] = (length, {u})
            elif length == best[v][0]:
                best[v][1].add(u)
            on.add(v)
            path.append(v)
            walk(path, on)
            path.pop()
            on.discard(v)

    walk([s], {s})
    par = np.full(g.n, -1)
    for v, (_, pre) in best.items():
        if pre:
            par[v] = min(pre)
    return par


@pytest.mark.parametrize("seed", range(12))
def test_tree_vs_path_enumeration(seed):
    rng = np.random.default_rng(900 + seed)
    g = random_digraph(900 + seed, n=int(rng.integers(2, 9)), p=float(rng.uniform(0.15, 0.5)))
    for s in range(g.n):
        d = oracle.sssp_sovm(g.row_ptr, g.col_idx, s)
        np.testing.assert_array_equal(oracle.parents(g.row_ptr, g.col_idx, d), brute_force_tree(g, s),
                                      err_msg=f"seed {seed} source {s}")


def test_tree_walks_back_to_source():
    """Following parent from any reached vertex takes dist[v] arcs and ends at
    the source (on a directed ER graph and an RMAT graph)."""
    for g in (gg.erdos_renyi(1024, 8.0, seed=1), gg.rmat(10, seed=3, symmetrise=False)):
        arcs = set(zip(np.repeat(np.arange(g.n), np.diff(g.row_ptr)).tolist(), g.col_idx.tolist()))
        for s in (0, 17, 400):
            d = oracle.sssp_sovm(g.row_ptr, g.col_idx, s)
            par = oracle.parents(g.row_ptr, g.col_idx, d)
            assert par[s] == -1 and (par[d < 0] == -1).all()
            for v in np.nonzero(d > 0)[0][::7]:
                x, steps = int(v), 0
                while x != s:
                    p = int(par[x])
                    assert (p, x) in arcs
                    x, steps = p, steps + 1
                assert steps == d[v]


# ------------------------------------------------------------ centrality pins --

def test_centrality_closed_forms():
    n = 13
    allv = np.arange(n)
    # path: from an end, harmonic = H_(n-1), closeness = 2 / n; diameter n-1, radius ceil((n-1)/2)
    g = path_graph(n, directed=False)
    c = oracle.centrality(g.row_ptr, g.col_idx, allv)
    assert c["harmonic"][0] == pytest.approx(sum(1.0 / i for i in range(1, n)), rel=1e-15)
    assert c["closeness"][0] == pytest.approx(2.0 / n, rel=1e-15)
    assert c["summary"] == {"diameter": n - 1, "radius": (n - 1 + 1) // 2, "pairs": n * (n - 1),
                            "dist_total": int(sum(abs(i - j) for i in range(n) for j in range(n)))}
    # star: centre harmonic n-1 and closeness 1; leaf harmonic 1 + (n-2)/2; diameter 2, radius 1
    leaves = np.arange(1, n)
    star = gg.from_arcs(n, np.r_[np.zeros(n - 1, int), leaves], np.r_[leaves, np.zeros(n - 1, int)], symmetric=True)
    c = oracle.centrality(star.row_ptr, star.col_idx, allv)
    assert c["harmonic"][0] == n - 1 and c["closeness"][0] == 1.0
    assert c["harmonic"][5] == pytest.approx(1 + (n - 2) / 2, rel=1e-15)
    assert (c["summary"]["diameter"], c["summary"]["radius"]) == (2, 1)
    # complete graph: harmonic n-1, closeness 1, diameter = radius = 1
    i, j = np.nonzero(~np.eye(n, dtype=bool))
    comp = gg.from_arcs(n, i, j, symmetric=True)
    c = oracle.centrality(comp.row_ptr, comp.col_idx, allv)
    assert (c["harmonic"] == n - 1).all() and (c["closeness"] == 1.0).all()
    assert (c["summary"]["diameter"], c["summary"]["radius"]) == (1, 1)
    # odd undirected cycle n = 2m + 1: every vertex has two at each distance 1..m
    m = 6
    cyc_n = 2 * m + 1
    s_ = np.arange(cyc_n)
    cyc = gg.from_arcs(cyc_n, np.r_[s_, (s_ + 1) % cyc_n], np.r_[(s_ + 1) % cyc_n, s_], symmetric=True)
    c = oracle.centrality(cyc.row_ptr, cyc.col_idx, np.arange(cyc_n))
    assert np.allclose(c["harmonic"], 2 * sum(1.0 / d for d in range(1, m + 1)), rtol=1e-15)
    assert (c["summary"]["diameter"], c["summary"]["radius"]) == (m, m)
    # isolated sources are left out of the radius; no edges at all: radius -1
    iso = gg.from_arcs(4, np.array([0, 1]), np.array([1, 0]), symmetric=True)
    c = oracle.centrality(iso.row_ptr, iso.col_idx, np.arange(4))
    assert c["summary"] == {"diameter": 1, "radius": 1, "pairs": 2, "dist_total": 2}
    assert c["harmonic"][3] == 0.0 and c["closeness"][3] == 0.0
    empty = gg.from_arcs(3, np.array([], int), np.array([], int))
    assert oracle.centrality(empty.row_ptr, empty.col_idx, np.arange(3))["summary"]["radius"] == -1


@pytest.mark.parametrize("seed", range(8))
def test_centrality_vs_scipy(seed):
    g = random_digraph(1300 + seed)
    n = g.n
    a = sp.csr_matrix((np.ones(g.m), g.col_idx, g.row_ptr), shape=(n, n))
    d = shortest_path(a, directed=True, unweighted=True)
    c = oracle.centrality(g.row_ptr, g.col_idx, np.arange(n))
    fin = np.isfinite(d)
    np.fill_diagonal(fin, False)
    for s in range(n):
        ds = d[s][fin[s]]
        assert c["ecc"][s] == (int(ds.max()) if ds.size else 0)
        assert c["dsum"][s] == int(ds.sum())
        assert c["reached"][s] == ds.size + 1
        assert c["harmonic"][s] == pytest.approx(float((1.0 / ds).sum()) if ds.size else 0.0, rel=1e-12)
        assert c["closeness"][s] == pytest.approx(ds.size / ds.sum() if ds.size else 0.0, rel=1e-15)
    ecc = np.array([int(d[s][fin[s]].max()) if fin[s].any() else 0 for s in range(n)])
    reaching = fin.any(axis=1)
    assert c["summary"]["diameter"] == ecc.max()
    assert c["summary"]["radius"] == (ecc[reaching].min() if reaching.any() else -1)
    assert c["summary"]["pairs"] == fin.sum()
    assert c["summary"]["dist_total"] == int(d[fin].sum())


# ---------------------------------------- weighted (min, +) extension pins --

def weighted_from_arcs(n, arcs):
    """CSR + aligned weights from (u, v, w) triples (self-loops and repeats kept)."""
    arcs = sorted(arcs)
    g = gg.from_arcs(n, [a for a, _, _ in arcs], [b for _, b, _ in arcs])
    return g, np.array([c for _, _, c in arcs], dtype=np.int32)


def random_weighted(seed, n=None, wmax=None):
    g = random_digraph(seed, n=n)
    rng = np.random.default_rng(10_000 + seed)
    wmax = wmax if wmax is not None else int(rng.choice([0, 1, 3, 20, 1000]))
    return g, rng.integers(0, wmax + 1, g.m).astype(np.int32)


def scipy_wdist(g, w, src):
    """scipy's Dijkstra (a library routine).  Repeated arcs keep their smallest
    weight; the graph goes through a dense matrix with inf for 'no arc', so
    that zero-weight arcs stay arcs (csgraph_from_dense with null_value=inf)."""
    n = g.n
    dense = np.full((n, n), np.inf)
    src_of = np.repeat(np.arange(n), g.out_degree())
    for u, v, c in zip(src_of, g.col_idx, w):
        if c < dense[u, v]:
            dense[u, v] = c
    cg = csgraph_from_dense(dense, null_value=np.inf)
    d = shortest_path(cg, method="D", directed=True, indices=[src])[0]
    return np.where(np.isinf(d), -1, d).astype(np.int64)


def floyd_weighted(g, w):
    n = g.n
    d = np.full((n, n), np.inf)
    np.fill_diagonal(d, 0)
    src_of = np.repeat(np.arange(n), g.out_degree())
    for u, v, c in zip(src_of, g.col_idx, w):
        d[u, v] = min(d[u, v], c) if u != v else 0
    for k in range(n):
        d = np.minimum(d, d[:, [k]] + d[[k], :])
    return np.where(np.isinf(d), -1, d).astype(np.int64)


@pytest.mark.parametrize("seed", RNG_SEEDS)
def test_weighted_vs_scipy_and_floyd(seed):
    g, w = random_weighted(2000 + seed)
    fw = floyd_weighted(g, w)
    for src in range(0, g.n, max(1, g.n // 5)):
        want = scipy_wdist(g, w, src)
        np.testing.assert_array_equal(fw[src], want)
        np.testing.assert_array_equal(oracle.wsssp_minplus(g.row_ptr, g.col_idx, w, src), want)
        np.testing.assert_array_equal(oracle.dijkstra(g.row_ptr, g.col_idx, w, src), want)


def tight_hops(g, w, src, dist):
    """Fewest arcs on a shortest path to each reached vertex: BFS over the arcs
    u -> v with dist[u] + w = dist[v] (numpy / Python, independent of the oracle)."""
    n = g.n
    hops = np.full(n, -1)
    hops[src] = 0
    frontier = [src]
    while frontier:
        nxt = []
        for u in frontier:
            for j in range(g.row_ptr[u], g.row_ptr[u + 1]):
                v = int(g.col_idx[j])
                if hops[v] < 0 and dist[v] == dist[u] + int(w[j]):
                    hops[v] = hops[u] + 1
                    nxt.append(v)
        frontier = nxt
    return hops


@pytest.mark.parametrize("seed", range(16))
def test_weighted_rounds_are_shortest_path_hops(seed):
    """Round k of the (min, +) iteration holds the least weight over walks of at
    most k arcs, so the rounds that change something number the largest, over
    reached vertices, of the fewest arcs on a shortest path."""
    g, w = random_weighted(2100 + seed)
    for src in range(0, g.n, max(1, g.n // 3)):
        d, rounds, _ = oracle.wsssp_minplus(g.row_ptr, g.col_idx, w, src, with_stats=True)
        assert rounds == int(tight_hops(g, w, src, d).max())


def test_weighted_closed_forms():
    # weighted directed path: prefix sums
    n = 7
    wts = [3, 0, 5, 1, 1, 9]
    g, w = weighted_from_arcs(n, [(i, i + 1, wts[i]) for i in range(n - 1)])
    want = np.concatenate([[0], np.cumsum(wts)])
    np.testing.assert_array_equal(oracle.wsssp_minplus(g.row_ptr, g.col_idx, w, 0), want)
    np.testing.assert_array_equal(oracle.wsssp_minplus(g.row_ptr, g.col_idx, w, 3),
                                  [-1, -1, -1, 0, 1, 2, 11])
    # directed cycle with unit weights: (v - s) mod n
    c, wc = weighted_from_arcs(9, [(i, (i + 1) % 9, 1) for i in range(9)])
    np.testing.assert_array_equal(oracle.wsssp_minplus(c.row_ptr, c.col_idx, wc, 4), (np.arange(9) - 4) % 9)
    # a shortcut of weight 10 against a 4-arc path of weight 4: the path wins
    s, ws = weighted_from_arcs(5, [(0, 4, 10), (0, 1, 1), (1, 2, 1), (2, 3, 1), (3, 4, 1)])
    assert oracle.wsssp_minplus(s.row_ptr, s.col_idx, ws, 0)[4] == 4
    # all-zero weights: 0 on every reached vertex
    g2 = random_digraph(77, n=30, p=0.1)
    z = np.zeros(g2.m, dtype=np.int32)
    bfs = oracle.sssp_sovm(g2.row_ptr, g2.col_idx, 0)
    np.testing.assert_array_equal(oracle.wsssp_minplus(g2.row_ptr, g2.col_idx, z, 0), np.where(bfs >= 0, 0, -1))
    # n = 1, with and without a self-loop
    one, w1 = weighted_from_arcs(1, [(0, 0, 5)])
    np.testing.assert_array_equal(oracle.wsssp_minplus(one.row_ptr, one.col_idx, w1, 0), [0])
    # the largest weights: distances past int32
    big, wb = weighted_from_arcs(4, [(0, 1, 2**31 - 1), (1, 2, 2**31 - 1), (2, 3, 2**31 - 1)])
    assert oracle.wsssp_minplus(big.row_ptr, big.col_idx, wb, 0)[3] == 3 * (2**31 - 1)


@pytest.mark.parametrize("seed", range(8))
def test_unit_weights_reduce_to_bfs(seed):
    g = random_digraph(2200 + seed)
    ones = np.ones(g.m, dtype=np.int32)
    for src in range(0, g.n, max(1, g.n // 4)):
        bfs = oracle.sssp_sovm(g.row_ptr, g.col_idx, src)
        np.testing.assert_array_equal(oracle.wsssp_minplus(g.row_ptr, g.col_idx, ones, src), bfs)


def test_weighted_golden_fixture():
    from pathlib import Path
    path = Path(__file__).parent / "golden" / "hand_weighted_6.txt"
    n, arcs, cases = None, [], []
    for line in path.read_text().splitlines():
        line = line.split("#", 1)[0].strip()
        if not line:
            continue
        key, _, rest = line.partition(":")
        vals = [int(x) for x in rest.split()]
        if key == "n":
            n = vals[0]
        elif key == "warc":
            arcs.append(tuple(vals))
        elif key.startswith("wdist"):
            cases.append((int(key.split()[1]), np.array(vals)))
    g, w = weighted_from_arcs(n, arcs)
    assert cases
    for src, want in cases:
        np.testing.assert_array_equal(oracle.wsssp_minplus(g.row_ptr, g.col_idx, w, src), want)
        np.testing.assert_array_equal(oracle.dijkstra(g.row_ptr, g.col_idx, w, src), want)
        assert oracle.wcertificate(g.row_ptr, g.col_idx, w, src, want) == (1, -1)


@pytest.mark.parametrize("seed", range(12))
def test_wcertificate_accepts_exact_rejects_planted(seed):
    g, w = random_weighted(2300 + seed, wmax=5)
    src = 0
    d = scipy_wdist(g, w, src)
    assert oracle.wcertificate(g.row_ptr, g.col_idx, w, src, d) == (1, -1)
    reached = np.nonzero(d > 0)[0]
    for v in reached[:6]:
        for delta in (-1, +1):
            bad = d.copy()
            bad[v] += delta
            assert oracle.wcertificate(g.row_ptr, g.col_idx, w, src, bad)[0] == 0
    unreached = np.nonzero(d < 0)[0]
    if unreached.size:
        bad = d.copy()
        bad[unreached[0]] = 5
        assert oracle.wcertificate(g.row_ptr, g.col_idx, w, src, bad)[0] == 0


def test_wcertificate_rejects_zero_weight_mutual_support():
    """Vertices 2 and 3 are unreachable from 0 but support each other through
    zero-weight arcs; only the search over tight arcs from the source sees it."""
    g, w = weighted_from_arcs(4, [(0, 1, 1), (2, 3, 0), (3, 2, 0)])
    exact = np.array([0, 1, -1, -1])
    assert oracle.wcertificate(g.row_ptr, g.col_idx, w, 0, exact) == (1, -1)
    fake = np.array([0, 1, 5, 5])
    assert oracle.wcertificate(g.row_ptr, g.col_idx, w, 0, fake)[0] == 0


def test_weighted_rejects_negative_weights():
    g, w = weighted_from_arcs(3, [(0, 1, 1), (1, 2, -1)])
    with pytest.raises(ValueError):
        oracle.wsssp_minplus(g.row_ptr, g.col_idx, w, 0)


def test_wcertificate_rejects_tight_but_too_long():
    """d(2) is 2 through 1, but a claim of 3 is tight through 3 (d(3) = 2, w = 1):
    only the arc bound on 1 -> 2 rejects it."""
    g, w = weighted_from_arcs(4, [(0, 1, 1), (1, 2, 1), (0, 3, 2), (3, 2, 1)])
    assert oracle.wcertificate(g.row_ptr, g.col_idx, w, 0, np.array([0, 1, 2, 2])) == (1, -1)
    assert oracle.wcertificate(g.row_ptr, g.col_idx, w, 0, np.array([0, 1, 3, 2]))[0] == 0
