"""A second, deliberately simple implementation of Algorithm 1 (pure Python, small
inputs only) whose visited set is either exact or a lossy direct-mapped table of `cap`
slots that can forget nodes, as the GPU's per-query table in shared memory does.

It exists to check one claim about that table: forgetting a node never changes the
result list R, the trajectory (the sequence of expanded nodes) or the results, because a
forgotten node is either still in R (its second insertion is dropped as a duplicate) or
was evicted or never entered, so its distance is >= the list bound then and, the bound
only decreasing, it is rejected again.  Only the number of exact distances can grow.

With the exact set it must reproduce the oracle's own trajectory (which pins it); the
routing test, when given, is a callback returning the pass decisions of v's edges.

`beam` = W expands the W unexpanded entries with the smallest (dist, id) per iteration,
with the list bound frozen for the iteration, the nodes taken in list order, each node's
edges in slot order, and the passes of the whole iteration inserted in ascending
(dist, id) order (W = 1: Algorithm 1's pop-one loop).
"""
from __future__ import annotations

import numpy as np


def _dist2(q, x) -> np.float32:
    acc = np.float32(0.0)
    for a, b in zip(q.tolist(), x.tolist()):
        t = np.float32(np.float32(a) - np.float32(b))
        acc = np.float32(acc + np.float32(t * t))
    return acc


def search(X, nbrs, entry: int, q, k: int, ef: int, cap: int = 0, test=None, beam: int = 1,
           bound_node: bool = False):
    """Returns (ids [k], dists [k], trace [expansions], n_dist).  cap = 0: exact visited
    set; cap = 2^b: lossy table.  test(v, dv, delta2) -> bool array over v's slots, used
    only while R is full (the oracle's convention: a list that is not full passes all);
    with bound_node the test also gets p = the id of R's efs-th entry (frame Q's p)."""
    n = X.shape[0]
    exact = set()
    table = np.full(cap, -1, dtype=np.int64) if cap else None

    def slot(u):
        return ((u * 0x9E3779B1) & 0xFFFFFFFF) >> (32 - (cap.bit_length() - 1))

    def seen(u):
        return (u in exact) if not cap else table[slot(u)] == u

    def mark(u):
        if cap:
            table[slot(u)] = u
        else:
            exact.add(u)

    R = [[_dist2(q, X[entry]), int(entry), False]]
    mark(int(entry))
    n_dist = 1
    trace = []
    while True:
        batch = [r for r in R if not r[2]][:beam]
        if not batch:
            break
        for r in batch:
            r[2] = True
        full = len(R) == ef
        delta2 = R[-1][0] if full else np.float32(np.inf)
        cand = []
        for dv, v, _ in batch:
            trace.append(v)
            passes = None
            if test is not None and full:
                passes = (test(v, float(dv), float(delta2), p=int(R[-1][1])) if bound_node
                          else test(v, float(dv), float(delta2)))
            for s, u in enumerate(nbrs[v].tolist()):
                if u < 0 or u >= n or seen(u):
                    continue
                if passes is not None and not passes[s]:
                    continue
                mark(u)
                cand.append((_dist2(q, X[u]), u))
                n_dist += 1
        for du, u in sorted(cand):
            if any(r[1] == u for r in R):
                continue            # already in R: only a forgotten node can come back
            if len(R) == ef and not du < R[-1][0]:
                continue
            pos = len(R)
            while pos > 0 and (R[pos - 1][0], R[pos - 1][1]) > (du, u):
                pos -= 1
            R.insert(pos, [du, u, False])
            if len(R) > ef:
                R.pop()
    ids = [r[1] for r in R[:k]] + [-1] * max(0, k - len(R))
    dists = [r[0] for r in R[:k]] + [np.float32(np.inf)] * max(0, k - len(R))
    return np.array(ids, dtype=np.int32), np.array(dists, dtype=np.float32), trace, n_dist
