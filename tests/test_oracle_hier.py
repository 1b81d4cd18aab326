"""Pins of the oracle's hierarchical entry (greedy descent through HNSW-style upper
layers, the paper's HNSW indexes of Sec. 6.1) and of searches with per-query entries.

Greedy descent with a list of one is fixed by special cases: on a complete layer one
hop reaches the exact nearest node; on a path over points of a line it walks to the
point nearest the query; in general it ends at a local minimum no farther than its
start.  A search whose per-query entries all equal the graph's entry is the plain
search, and a search with efs = 1 started at the exact nearest node returns it."""
import numpy as np
import pytest

import oracle
import workloads
from workloads.graph import build_graph
from workloads.hier import build_hierarchy


def test_complete_layer_reaches_exact_nn():
    rng = np.random.default_rng(1)
    n, d = 300, 16
    X = rng.integers(0, 50, size=(n, d)).astype(np.float32)
    Q = rng.integers(0, 50, size=(40, d)).astype(np.float32)
    ids = np.arange(n, dtype=np.int32)
    nbrs = np.array([[u for u in range(n) if u != v] for v in range(n)], dtype=np.int32)
    start = rng.integers(0, n, size=len(Q)).astype(np.int32)
    end, hops = oracle.greedy_layer(X, Q, ids, nbrs, start)
    D = ((Q[:, None, :].astype(np.float64) - X[None]) ** 2).sum(-1)
    nn = np.lexsort((np.arange(n)[None].repeat(len(Q), 0), D), axis=1)[:, 0]
    assert np.array_equal(end, nn)
    assert np.all(hops == (start != nn))


def test_path_over_a_line_walks_to_the_nearest_point():
    n = 101
    X = np.zeros((n, 4), dtype=np.float32)
    X[:, 0] = np.arange(n) * 2.0          # points 0, 2, 4, ... on a line
    nbrs = np.full((n, 2), -1, dtype=np.int32)
    nbrs[1:, 0] = np.arange(n - 1)
    nbrs[:-1, 1] = np.arange(1, n)
    Q = np.zeros((5, 4), dtype=np.float32)
    Q[:, 0] = [0.4, 37.0, 121.2, 199.9, 500.0]
    start = np.array([50, 0, 100, 3, 7], dtype=np.int32)
    end, hops = oracle.greedy_layer(X, Q, np.arange(n, dtype=np.int32), nbrs, start)
    want = np.clip(np.floor(Q[:, 0] / 2 + 0.5), 0, n - 1).astype(np.int32)
    want[1] = 18  # 37 is halfway between 36 and 38: equal distances keep the lower id
    assert np.array_equal(end, want)
    assert np.array_equal(hops, np.abs(want - start))


def test_equal_neighbours_take_the_lower_id():
    """Two neighbours at the same distance from q, both closer than the current node: the
    descent takes the one with the lower id, whatever their slot order.  Worked by hand:
    node 0 at (0, 0), nodes 1 at (1, 1) and 2 at (1, -1), q at (2, 0): distances 4, 2 and
    2; from node 0 (neighbours listed 2 then 1) one hop to node 1, which has no closer
    neighbour."""
    X = np.array([[0, 0], [1, 1], [1, -1]], dtype=np.float32)
    nbrs = np.array([[2, 1], [0, -1], [0, -1]], dtype=np.int32)
    Q = np.array([[2, 0]], dtype=np.float32)
    end, hops = oracle.greedy_layer(X, Q, np.arange(3, dtype=np.int32), nbrs, np.zeros(1, dtype=np.int32))
    assert end.tolist() == [1] and hops.tolist() == [1]


@pytest.fixture(scope="module")
def small():
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 6000, 60)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 16)
    layers, top = build_hierarchy(X, 16, seed=3, M=6, min_nodes=20)
    return cfg, X, Q, nbrs, entry, layers, top


def test_descent_ends_at_a_local_minimum(small):
    cfg, X, Q, nbrs, entry, layers, top = small
    assert len(layers) >= 2 and len(layers[0]["ids"]) < len(layers[-1]["ids"])
    cur = np.full(len(Q), top, dtype=np.int32)
    for i, lay in enumerate(layers):
        start = cur.copy()
        cur, _ = oracle.greedy_layer(X, Q, lay["ids"], lay["nbrs"], cur)
        Xl = X[lay["ids"]].astype(np.float64)
        for qi in range(len(Q)):
            dq = ((Xl - Q[qi]) ** 2).sum(1)
            c = cur[qi]
            nb = lay["nbrs"][c][lay["nbrs"][c] >= 0]
            assert dq[c] <= dq[start[qi]]
            assert np.all(dq[nb] >= dq[c])
        if i + 1 < len(layers):
            cur = lay["down"][cur]
    ent, hops = oracle.hier_entries(X, Q, layers, top)
    assert np.array_equal(ent, layers[-1]["ids"][cur])
    assert np.all(hops >= 0)


def test_hierarchy_structure(small):
    cfg, X, Q, nbrs, entry, layers, top = small
    for hi, lo in zip(layers[:-1], layers[1:]):
        assert np.all(np.isin(hi["ids"], lo["ids"]))          # nested node sets
        assert np.array_equal(lo["ids"][hi["down"]], hi["ids"])  # down maps to the same node
    for lay in layers:
        nb = lay["nbrs"]
        assert nb.max() < len(lay["ids"]) and np.all(nb[nb >= 0] != np.nonzero(nb >= 0)[0])
    # about n / M^l nodes on layer l (M = 6)
    assert abs(len(layers[-1]["ids"]) - len(X) / 6) < 5 * np.sqrt(len(X) / 6)


def test_per_query_entries(small):
    cfg, X, Q, nbrs, entry, layers, top = small
    ix = oracle.Index(X, nbrs, entry, cfg.L, cfg.m, cfg.proj_seed)
    for routing in (0, 1):
        a = ix.search(Q, 10, 32, routing=routing, eps=0.2)
        b = ix.search(Q, 10, 32, routing=routing, eps=0.2, entries=np.full(len(Q), entry, dtype=np.int32))
        assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["counters"], b["counters"])
    nn, _ = oracle.knn_f64(X, Q, 1)
    r = ix.search(Q, 1, 1, routing=0, entries=nn[:, 0])
    assert np.array_equal(r["ids"][:, 0], nn[:, 0])
    with pytest.raises(ValueError):
        ix.search(Q, 10, 32, routing=0, entries=np.full(len(Q), len(X), dtype=np.int32))
