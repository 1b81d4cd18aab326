"""The oracle's search on many small random inputs built to hit the corners of Algorithm 1:
integer-valued rows (equal distances everywhere, so the (dist, id) order decides), rows
that repeat an id, self loops, empty slots, nodes unreachable from the entry, lists of one
entry and lists longer than the graph.

- Plain routing, and PEOs routing with the test decided by the oracle's own edge
  statistics (pinned against FP64 definitions elsewhere), against the second
  implementation of Algorithm 1 (tests/lossy_search.py): the same trajectory, results
  and number of exact distances, for beam widths 1 and 2.
- With efs >= N every node reachable from the entry is reached: the results are the
  k nearest reachable nodes in (distance, id) order, by brute force."""
import numpy as np
import pytest

import lossy_search
import oracle


def _case(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 41))
    d = int(rng.choice([4, 8]))
    R = int(rng.integers(1, 7))
    X = rng.integers(0, 4, size=(n, d)).astype(np.float32)
    nbrs = rng.integers(0, n, size=(n, R)).astype(np.int32)
    nbrs[rng.random((n, R)) < 0.25] = -1
    entry = int(rng.integers(0, n))
    Q = rng.integers(0, 4, size=(3, d)).astype(np.float32)
    ef = int(rng.integers(1, n + 3))
    k = int(rng.integers(1, ef + 1))
    return X, nbrs, entry, Q, ef, k


def _reachable(nbrs, entry):
    seen = {entry}
    frontier = [entry]
    while frontier:
        nxt = []
        for v in frontier:
            for u in nbrs[v].tolist():
                if u >= 0 and u not in seen:
                    seen.add(u)
                    nxt.append(u)
        frontier = nxt
    return sorted(seen)


@pytest.mark.parametrize("beam", [1, 2])
def test_plain_search_equals_second_implementation(beam):
    for seed in range(80):
        X, nbrs, entry, Q, ef, k = _case(seed)
        r = oracle.search(X, nbrs, entry, Q, k, ef, routing=0, beam=beam, trace_cap=4096)
        for qi in range(len(Q)):
            ids, dists, trace, nd = lossy_search.search(X, nbrs, entry, Q[qi], k, ef, beam=beam)
            n_exp = int(r["counters"][qi, 0])
            assert trace == r["trace_v"][qi, :n_exp].tolist(), seed
            assert np.array_equal(ids, r["ids"][qi]) and np.array_equal(dists, r["dists"][qi]), seed
            assert nd == int(r["counters"][qi, 7]), seed


@pytest.mark.parametrize("beam", [1, 2])
def test_peos_search_equals_second_implementation(beam):
    tested = 0
    for seed in range(80):
        X, nbrs, entry, Q, ef, k = _case(1000 + seed)
        ix = oracle.Index(X, nbrs, entry, 2, 16, seed)
        r = ix.search(Q, k, ef, routing=1, eps=0.2, beam=beam, trace_cap=4096)
        for qi in range(len(Q)):
            def test(v, dv, d2, q=Q[qi]):
                return ix.edge_stats(q, v, dv, d2, eps=0.2)["passed"].astype(bool)
            ids, dists, trace, nd = lossy_search.search(X, nbrs, entry, Q[qi], k, ef, test=test, beam=beam)
            n_exp = int(r["counters"][qi, 0])
            assert trace == r["trace_v"][qi, :n_exp].tolist(), seed
            assert np.array_equal(ids, r["ids"][qi]) and np.array_equal(dists, r["dists"][qi]), seed
            assert nd == int(r["counters"][qi, 7]), seed
            tested += int(r["counters"][qi, 5])
    assert tested > 50                       # the H >= T stage decided edges


def test_full_list_returns_the_nearest_reachable_nodes():
    for seed in range(80):
        X, nbrs, entry, Q, _, k = _case(2000 + seed)
        n = len(X)
        k = min(k, n)
        reach = np.array(_reachable(nbrs, entry))
        r = oracle.search(X, nbrs, entry, Q, k, n, routing=0)
        for qi in range(len(Q)):
            dd = ((X[reach].astype(np.float64) - Q[qi]) ** 2).sum(1)
            order = reach[np.lexsort((reach, dd))][:k]
            want = np.full(k, -1, dtype=np.int32)
            want[:len(order)] = order
            assert np.array_equal(r["ids"][qi], want), seed
            got = r["dists"][qi]
            assert np.all(np.isinf(got[len(order):]))
            assert np.array_equal(got[:len(order)], np.sort(dd)[:len(order)].astype(np.float32))
