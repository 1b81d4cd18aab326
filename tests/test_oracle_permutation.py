"""Pins of the oracle's dimension permutation (Appendix D.1) and of an index built in
permuted coordinates.

The permutation is checked against examples worked by hand from the appendix's steps,
against invariants its greedy rounds guarantee (a permutation; one coordinate of each
rank group per subspace; final subspace sums within the largest in-round spread of
each other), and the permuted index against the two special cases that fix it: the
identity permutation changes nothing, and an index with permutation p answers exactly
like an unpermuted index built on X[:, p] queried with q[p] (integer-valued data, so
exact distances do not depend on summation order)."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dim_permutation.txt")


def _examples():
    ex = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            name, field = k.split(".")
            ex.setdefault(name, {})[field] = [float(t) for t in v.split()]
    return ex


def _one_edge(edge):
    d = len(edge)
    X = np.zeros((2, d), dtype=np.float32)
    X[1] = edge
    nbrs = np.array([[1], [-1]], dtype=np.int32)
    return X, nbrs


@pytest.mark.parametrize("name", ["ex1", "ex2"])
def test_worked_examples(name):
    ex = _examples()[name]
    L = int(ex["L"][0])
    X, nbrs = _one_edge(ex["edge"])
    perm = oracle.dim_permutation(X, nbrs, L)
    assert perm.tolist() == [int(v) for v in ex["perm"]]
    avg = np.asarray(ex["edge"]) ** 2
    sums = avg[perm].reshape(L, -1).sum(axis=1)
    assert sums.tolist() == ex["sums"]


def _avg(X, nbrs):
    v, s = np.nonzero(nbrs >= 0)
    E = X[nbrs[v, s]].astype(np.float64) - X[v].astype(np.float64)
    return (E * E).sum(axis=0) / len(v)


@pytest.mark.parametrize("d,L,seed", [(32, 4, 0), (96, 8, 1), (960, 24, 2), (100, 10, 3)])
def test_greedy_round_invariants(d, L, seed):
    rng = np.random.default_rng(seed)
    n, R = 300, 6
    # unequal per-coordinate spread, as in real data (some coordinates carry most energy)
    scale = rng.gamma(0.7, size=d).astype(np.float32)
    X = np.round(rng.standard_normal((n, d)) * scale * 20).astype(np.float32)
    nbrs = rng.integers(0, n, size=(n, R)).astype(np.int32)
    nbrs[rng.random((n, R)) < 0.2] = -1
    perm = oracle.dim_permutation(X, nbrs, L)
    assert sorted(perm.tolist()) == list(range(d))
    avg = _avg(X, nbrs)
    dp = d // L
    rank = np.empty(d, dtype=np.int64)
    rank[np.lexsort((np.arange(d), avg))] = np.arange(d)
    blocks = perm.reshape(L, dp)
    # the t-th coordinate of every subspace comes from the t-th round's rank group,
    # and within a subspace the rounds are in order
    assert np.all(rank[blocks] // L == np.arange(dp)[None, :])
    # the greedy keeps the subspace sums within the largest spread of any round's values
    rounds = np.sort(avg)[: d].reshape(dp, L)
    spread = (rounds[:, -1] - rounds[:, 0]).max()
    sums = avg[blocks].sum(axis=1)
    assert sums.max() - sums.min() <= spread * (1 + 1e-12)
    # and in each round the heaviest subspace so far receives the smallest value
    run = np.zeros(L)
    for l in range(dp):
        got = avg[blocks[:, l]]
        order = np.lexsort((np.arange(L), -run))
        assert np.all(np.diff(got[order]) >= 0)
        run += got


def test_empty_graph_and_bad_L():
    X = np.arange(8, dtype=np.float32).reshape(2, 4)
    nbrs = np.full((2, 3), -1, dtype=np.int32)
    # no edge: every Avg is 0, ties by coordinate, subspaces served in index order
    assert oracle.dim_permutation(X, nbrs, 2).tolist() == [0, 2, 1, 3]
    with pytest.raises(ValueError):
        oracle.dim_permutation(X, nbrs, 3)


@pytest.fixture(scope="module")
def small():
    rng = np.random.default_rng(7)
    n, d, R = 2000, 64, 12
    scale = np.linspace(0.2, 3.0, d)[rng.permutation(d)]
    X = np.round(rng.standard_normal((n, d)) * scale * 10).astype(np.float32)
    Q = np.round(rng.standard_normal((40, d)) * scale * 10).astype(np.float32)
    nbrs, entry = oracle.build_graph(X, R)
    return X, Q, nbrs, entry


def test_identity_permutation_changes_nothing(small):
    X, Q, nbrs, entry = small
    a = oracle.Index(X, nbrs, entry, 8, 16, 5)
    b = oracle.Index(X, nbrs, entry, 8, 16, 5, perm=np.arange(X.shape[1]))
    for f in ("codes", "enorm", "wreg", "cres", "tv"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    ra = a.search(Q, 10, 64, routing=1, eps=0.2)
    rb = b.search(Q, 10, 64, routing=1, eps=0.2)
    assert np.array_equal(ra["ids"], rb["ids"]) and np.array_equal(ra["counters"], rb["counters"])


def test_permutation_equals_permuted_data_and_queries(small):
    X, Q, nbrs, entry = small
    perm = oracle.dim_permutation(X, nbrs, 8)
    assert not np.array_equal(perm, np.arange(X.shape[1]))
    a = oracle.Index(X, nbrs, entry, 8, 16, 5, perm=perm)
    b = oracle.Index(np.ascontiguousarray(X[:, perm]), nbrs, entry, 8, 16, 5)
    for f in ("codes", "enorm", "wreg", "cres", "tv"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    Qp = np.ascontiguousarray(Q[:, perm])
    ra = a.search(Q, 10, 64, routing=1, eps=0.2)
    rb = b.search(Qp, 10, 64, routing=1, eps=0.2)
    assert np.array_equal(ra["ids"], rb["ids"]) and np.array_equal(ra["dists"], rb["dists"])
    assert np.array_equal(ra["counters"], rb["counters"])
    sa = a.edge_stats(Q[0], entry, 50.0, 4000.0, eps=0.2)
    sb = b.edge_stats(Qp[0], entry, 50.0, 4000.0, eps=0.2)
    for f in ("A", "H", "T", "passed", "kind"):
        assert np.array_equal(sa[f], sb[f]), f
    # the inverse permutation is a different index (the direction matters)
    inv = np.argsort(perm).astype(np.int32)
    if not np.array_equal(inv, perm):
        c = oracle.Index(X, nbrs, entry, 8, 16, 5, perm=inv)
        assert not np.array_equal(c.codes, a.codes)


def test_lazy_permuted_index_equals_eager(small):
    X, Q, nbrs, entry = small
    perm = oracle.dim_permutation(X, nbrs, 8)
    a = oracle.Index(X, nbrs, entry, 8, 16, 5, perm=perm)
    b = oracle.Index(X, nbrs, entry, 8, 16, 5, perm=perm, lazy=True)
    ra = a.search(Q, 10, 64, routing=1, eps=0.2)
    rb = b.search(Q, 10, 64, routing=1, eps=0.2)
    assert np.array_equal(ra["ids"], rb["ids"]) and np.array_equal(ra["counters"], rb["counters"])
