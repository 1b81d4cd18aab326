"""Pins of the oracle's search (Algorithm 1 with the plain or PEOs routing test) and
of the graph both paths read.

- Brute force: with efs >= N on a connected graph every node is reached, so
  recall@k = 1 against FP64 brute force (Sec. 2's K-NN definition).
- Routing disabled (every neighbour passes) gives the plain trajectory; the
  cut-only test (T = -inf: only A >= 1 rejects, and A >= 1 implies dist >= delta)
  gives the same R evolution.
- A lossy visited table (forgets nodes), in a second implementation of Algorithm 1
  that first reproduces the oracle, gives the same results and trajectory as the exact
  visited set: a forgotten node is already in R or lies at distance >= delta.
- The graph generator equals the oracle's graph builder; the pruning rule holds by
  brute force; every node is reachable from the entry.
"""
import numpy as np
import pytest

import lossy_search
import oracle
import workloads
from workloads.graph import build_graph


@pytest.fixture(scope="module")
def small():
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 3000, 40)
    X, Q = workloads.generate(cfg)
    nbrs, entry = oracle.build_graph(X, 32)
    ix = oracle.Index(X, nbrs, entry, 8, 16, cfg.proj_seed)
    return X, Q, nbrs, entry, ix


def test_knn_f64_is_brute_force():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((500, 24)).astype(np.float32)
    Q = rng.standard_normal((20, 24)).astype(np.float32)
    ids, dists = oracle.knn_f64(X, Q, 7)
    D = ((Q[:, None, :].astype(np.float64) - X[None].astype(np.float64)) ** 2).sum(-1)
    order = np.lexsort((np.broadcast_to(np.arange(500), D.shape), D), axis=1)[:, :7]
    assert np.array_equal(ids, order)
    assert np.allclose(dists, np.take_along_axis(D, order, 1), rtol=1e-12)
    # small integer rows: many equal distances, ordered by id
    Xi = rng.integers(0, 3, size=(500, 4)).astype(np.float32)
    Qi = rng.integers(0, 3, size=(20, 4)).astype(np.float32)
    ids, dists = oracle.knn_f64(Xi, Qi, 25)
    D = ((Qi[:, None, :].astype(np.float64) - Xi[None].astype(np.float64)) ** 2).sum(-1)
    order = np.lexsort((np.broadcast_to(np.arange(500), D.shape), D), axis=1)[:, :25]
    assert np.array_equal(ids, order) and np.array_equal(dists, np.take_along_axis(D, order, 1))
    assert np.any(np.diff(dists, axis=1) == 0)            # ties occurred


def test_full_ef_finds_exact_knn():
    cfg = workloads.scaled(workloads.CONFIGS["tiny"], 600, 20)
    X, Q = workloads.generate(cfg)
    nbrs, entry = oracle.build_graph(X, 16)
    gt, _ = oracle.knn_f64(X, Q, 10)
    r = oracle.search(X, nbrs, entry, Q, 10, 600, routing=0)
    assert oracle.recall_at_k(r["ids"], gt) == 1.0
    ix = oracle.Index(X, nbrs, entry, 8, 16, 1)
    p = ix.search(Q, 10, 600, routing=1, eps=0.1)
    assert oracle.recall_at_k(p["ids"], gt) == 1.0


@pytest.mark.parametrize("ef", [16, 64])
def test_disabled_test_equals_plain_trajectory(small, ef):
    X, Q, nbrs, entry, ix = small
    a = oracle.search(X, nbrs, entry, Q, 10, ef, routing=0, trace_cap=4096)
    b = ix.search(Q, 10, ef, routing=1, test_mode=2, trace_cap=4096)
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["dists"], b["dists"])
    assert np.array_equal(a["trace_v"], b["trace_v"])
    assert np.array_equal(a["counters"][:, 7], b["counters"][:, 7])


@pytest.mark.parametrize("ef", [16, 64])
def test_cut_only_keeps_plain_trajectory(small, ef):
    X, Q, nbrs, entry, ix = small
    a = oracle.search(X, nbrs, entry, Q, 10, ef, routing=0, trace_cap=4096)
    b = ix.search(Q, 10, ef, routing=1, test_mode=1, trace_cap=4096)
    assert np.array_equal(a["ids"], b["ids"])
    assert np.array_equal(a["trace_v"], b["trace_v"])
    assert b["counters"][:, 5].sum() == 0       # no edge reached the H >= T stage


@pytest.mark.parametrize("routing", [0, 1])
@pytest.mark.parametrize("cap", [64, 256])
def test_lossy_visited_table_changes_nothing(small, routing, cap):
    """A second implementation of Algorithm 1 (tests/lossy_search.py) reproduces the
    oracle's trajectory with an exact visited set, and with a lossy table that forgets
    nodes it keeps the same trajectory and results (the GPU's table is lossy)."""
    X, Q, nbrs, entry, ix = small
    test = None
    if routing == 1:
        def test(v, dv, delta2, q=None):
            return ix.edge_stats(q, v, dv, delta2, eps=0.2)["passed"].astype(bool)
    orc = ix.search(Q[:12], 10, 48, routing=routing, eps=0.2, trace_cap=4096)
    grew = 0
    for qi in range(12):
        t = None if test is None else (lambda v, dv, d2, q=Q[qi]: test(v, dv, d2, q=q))
        a = lossy_search.search(X, nbrs, entry, Q[qi], 10, 48, cap=0, test=t)
        b = lossy_search.search(X, nbrs, entry, Q[qi], 10, 48, cap=cap, test=t)
        n_exp = int(orc["counters"][qi, 0])
        assert a[2] == orc["trace_v"][qi, :n_exp].tolist()
        assert np.array_equal(a[0], orc["ids"][qi]) and np.array_equal(a[1], orc["dists"][qi])
        assert a[3] == orc["counters"][qi, 7]
        assert b[2] == a[2] and np.array_equal(b[0], a[0]) and np.array_equal(b[1], a[1])
        assert b[3] >= a[3]                      # forgetting only adds evaluations
        grew += b[3] > a[3]
    if cap == 64:
        assert grew > 0                          # the small table did forget nodes


@pytest.mark.parametrize("routing", [0, 1])
@pytest.mark.parametrize("beam", [2, 4])
def test_beam_width_follows_its_definition(small, routing, beam):
    """Beam width W (W nodes expanded per iteration) against the second implementation of
    the iteration in tests/lossy_search.py: same trajectory, results and distance count."""
    X, Q, nbrs, entry, ix = small
    test = None
    if routing == 1:
        def test(v, dv, delta2, q=None):
            return ix.edge_stats(q, v, dv, delta2, eps=0.2)["passed"].astype(bool)
    orc = ix.search(Q[:12], 10, 48, routing=routing, eps=0.2, trace_cap=4096, beam=beam)
    for qi in range(12):
        t = None if test is None else (lambda v, dv, d2, q=Q[qi]: test(v, dv, d2, q=q))
        ids, dists, trace, nd = lossy_search.search(X, nbrs, entry, Q[qi], 10, 48, test=t, beam=beam)
        n_exp = int(orc["counters"][qi, 0])
        assert trace == orc["trace_v"][qi, :n_exp].tolist()
        assert np.array_equal(ids, orc["ids"][qi]) and np.array_equal(dists, orc["dists"][qi])
        assert nd == orc["counters"][qi, 7]


@pytest.mark.parametrize("beam", [1, 2, 4, 8])
def test_beam_width_special_cases(small, beam):
    """Any W: efs >= N reaches every node (exact K-NN); the always-pass test is plain
    routing with the same W; W = 1 is the default."""
    X, Q, nbrs, entry, ix = small
    gt, _ = oracle.knn_f64(X, Q, 10)
    full = ix.search(Q[:8], 10, len(X), routing=1, eps=0.2, beam=beam)
    assert np.array_equal(full["ids"], gt[:8])
    a = oracle.search(X, nbrs, entry, Q, 10, 32, routing=0, beam=beam, trace_cap=4096)
    b = ix.search(Q, 10, 32, routing=1, test_mode=2, beam=beam, trace_cap=4096)
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["trace_v"], b["trace_v"])
    if beam == 1:
        c = oracle.search(X, nbrs, entry, Q, 10, 32, routing=0, trace_cap=4096)
        assert np.array_equal(a["trace_v"], c["trace_v"])
    with pytest.raises(ValueError):
        ix.search(Q[:2], 10, 32, routing=1, beam=9)


def test_peos_saves_distances_at_similar_recall(small):
    X, Q, nbrs, entry, ix = small
    gt, _ = oracle.knn_f64(X, Q, 10)
    a = oracle.search(X, nbrs, entry, Q, 10, 64, routing=0)
    b = ix.search(Q, 10, 64, routing=1, eps=0.2)
    assert b["counters"][:, 7].mean() < 0.85 * a["counters"][:, 7].mean()
    assert oracle.recall_at_k(b["ids"], gt) >= oracle.recall_at_k(a["ids"], gt) - 0.05
    # the paper-literal frame (q' projected once per query) runs and finds neighbours too
    c = ix.search(Q, 10, 64, routing=1, eps=0.2, frame=1)
    assert oracle.recall_at_k(c["ids"], gt) >= oracle.recall_at_k(a["ids"], gt) - 0.1


def test_results_sorted_and_exact(small):
    X, Q, nbrs, entry, ix = small
    r = ix.search(Q, 10, 32, routing=1)
    assert np.all(np.diff(r["dists"], axis=1) >= 0)
    for qi in range(len(Q)):
        for j in range(10):
            assert r["dists"][qi, j] == oracle.dist2_f32(Q[qi], X[r["ids"][qi, j]])


def test_lazy_index_equals_eager(small):
    X, Q, nbrs, entry, ix = small
    lazy = oracle.Index(X, nbrs, entry, 8, 16, ix.seed, lazy=True)
    a = ix.search(Q, 10, 32, routing=1, trace_cap=2048)
    b = lazy.search(Q, 10, 32, routing=1, trace_cap=2048)
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["trace_v"], b["trace_v"])
    built = lazy.ready == 2
    assert built.sum() < len(X)
    assert np.array_equal(lazy.codes[built], ix.codes[built]) and np.array_equal(lazy.wreg[built], ix.wreg[built])


@pytest.mark.parametrize("name,n", [("tiny", 2000), ("sift", 3000)])
def test_generator_graph_equals_oracle_graph(name, n):
    cfg = workloads.scaled(workloads.CONFIGS[name], n, 1)
    X, _ = workloads.generate(cfg)
    g1, e1 = oracle.build_graph(X, 32)
    g2, e2 = build_graph(X, 32)
    assert e1 == e2
    assert np.array_equal(g1, g2)


def test_graph_properties_brute_force(small):
    X, Q, nbrs, entry, ix = small
    n = len(X)
    X64 = X.astype(np.float64)
    # lists sorted by (distance, id), no self loops, no duplicates
    for v in range(0, n, 7):
        lst = nbrs[v][nbrs[v] >= 0]
        assert v not in lst and len(set(lst.tolist())) == len(lst)
        d = ((X64[lst] - X64[v]) ** 2).sum(1)
        assert np.all((np.diff(d) > 0) | ((np.diff(d) == 0) & (np.diff(lst) > 0)))
    # reachability from the entry
    seen = np.zeros(n, bool)
    seen[entry] = True
    frontier = [entry]
    while frontier:
        nb = nbrs[frontier].ravel()
        nb = np.unique(nb[nb >= 0])
        nb = nb[~seen[nb]]
        seen[nb] = True
        frontier = nb.tolist()
    assert seen.all()
    # the entry is the point nearest the centroid
    c = X64.mean(0)
    assert entry == int(np.argmin(((X64 - c) ** 2).sum(1)))


def test_ties_with_the_list_bound_are_not_inserted():
    """Algorithm 1 inserts into a full list only a candidate strictly closer than δ, and
    takes candidates in ascending (dist, id).  Worked by hand on a star: node 0 at the
    origin (the entry, also the query) and nodes 1..4 at distance 1 around it, all of them
    node 0's neighbours.  With efs = 2 the list is [(0, 0)] when node 0 is expanded; its
    four neighbours all have distance 1, so (1, 1) fills the list and the other three
    equal the bound δ = 1 and stay out; node 1 is expanded next (its only neighbour, node
    0, was visited) and the search ends: results [0, 1], trajectory [0, 1], five exact
    distances (the entry and the four neighbours)."""
    X = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1]], dtype=np.float32)
    nbrs = np.array([[1, 2, 3, 4], [0, -1, -1, -1], [0, -1, -1, -1], [0, -1, -1, -1], [0, -1, -1, -1]],
                    dtype=np.int32)
    r = oracle.search(X, nbrs, 0, X[:1], 2, 2, routing=0, trace_cap=8)
    assert r["ids"][0].tolist() == [0, 1] and r["dists"][0].tolist() == [0.0, 1.0]
    assert r["trace_v"][0, :int(r["counters"][0, 0])].tolist() == [0, 1]
    assert int(r["counters"][0, 7]) == 5
    # the second implementation of Algorithm 1 agrees
    ids, dists, trace, nd = lossy_search.search(X, nbrs, 0, X[0], 2, 2)
    assert ids.tolist() == [0, 1] and trace == [0, 1] and nd == 5
    # a list longer than the reachable nodes: the five nodes, then empty slots (id -1, +inf)
    r = oracle.search(X, nbrs, 0, X[:1], 8, 8, routing=0)
    assert r["ids"][0].tolist() == [0, 1, 2, 3, 4, -1, -1, -1]
    assert r["dists"][0].tolist() == [0.0, 1.0, 1.0, 1.0, 1.0] + [float("inf")] * 3
