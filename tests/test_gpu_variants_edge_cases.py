"""Edge cases of the search variants (SimHash test, frame Q, permuted codes, per-query
entries) against the oracle: duplicated vectors (degenerate edges), queries equal to
base points, ragged degrees, the smallest and largest lists, empty batches, and the
two-edges-per-lane shape (R = 48) on float data.  Bars: tests/parity.py (plain routing
on these integer-valued rows: bit for bit)."""
import numpy as np
import pytest
import torch

import oracle
import parity
import workloads
from workloads.graph import build_graph
from workloads.hier import build_hierarchy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module")
def ragged(P):
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 3000, 37)
    X, Q = workloads.generate(cfg)
    X[100:110] = X[200]
    Q[:5] = X[[0, 200, 1234, 2999, 105]]
    nbrs, entry = build_graph(X, 32)
    rng = np.random.default_rng(5)
    drop = rng.random(nbrs.shape) < 0.3
    drop[:, 0] = False
    nbrs = np.where(drop, -1, nbrs).astype(np.int32)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    return X, Q, nbrs, entry, Xt, Qt, G


LISTS = ((1, 1), (1, 8), (10, 10), (10, 512), (100, 1024))


def test_simhash_ragged(P, ragged):
    X, Q, nbrs, entry, Xt, Qt, G = ragged
    codes = P.build_simhash(G, Xt, 64, 3)
    sh = oracle.SimHash(X, nbrs, 64, 3)
    for k, ef in LISTS:
        ids, dists, cnt = P.search(G, codes, Xt, Qt, k, ef, routing=2, eps=0.2, counters=True)
        want = oracle.search(X, nbrs, entry, Q, k, ef, routing=2, simhash=sh, eps=0.2)
        parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, what=f"k {k}, efs {ef}")
        parity.counters_parity(cnt.cpu().numpy(), want["counters"], 0, what=f"k {k}, efs {ef}")
    assert P.search(G, codes, Xt, Qt[:0], 10, 32, routing=2)[0].shape == (0, 10)


def test_frame_q_and_permutation_ragged(P, ragged):
    X, Q, nbrs, entry, Xt, Qt, G = ragged
    perm = oracle.dim_permutation(X, nbrs, 8)
    cases = [(None, oracle.Index(X, nbrs, entry, 8, 16, 9)),
             (perm, oracle.Index(X, nbrs, entry, 8, 16, 9, perm=perm))]
    for p, ix in cases:
        codes = P.build_codes(G, Xt, 8, 16, 9, perm=None if p is None else torch.from_numpy(p).cuda())
        for frame in (0, 1):
            for k, ef in LISTS:
                ids, dists, cnt = P.search(G, codes, Xt, Qt, k, ef, routing=1, eps=0.1, frame=frame, counters=True)
                want = ix.search(Q, k, ef, routing=1, eps=0.1, frame=frame)
                what = f"permuted {p is not None}, frame {frame}, k {k}, efs {ef}"
                parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, what=what)
                parity.counters_parity(cnt.cpu().numpy(), want["counters"], 0, what=what)
        assert P.search(G, codes, Xt, Qt[:0], 10, 32, routing=1, frame=1)[0].shape == (0, 10)


def test_entries_ragged_and_empty(P, ragged):
    X, Q, nbrs, entry, Xt, Qt, G = ragged
    layers, top = build_hierarchy(X, 16, seed=4, M=8, min_nodes=16)
    H = P.Hierarchy(layers, top)
    ent = P.hier_entry(H, Xt, Qt)
    want, _ = oracle.hier_entries(X, Q, layers, top)
    assert np.array_equal(ent.cpu().numpy(), want)
    assert P.hier_entry(H, Xt, Qt[:0]).shape == (0,)
    ix = oracle.Index(X, nbrs, entry, 8, 16, 9)
    codes = P.build_codes(G, Xt, 8, 16, 9)
    for routing in (0, 1):
        for k, ef in LISTS:
            ids, dists, _ = P.search(G, codes, Xt, Qt, k, ef, routing=routing, eps=0.1, entries=ent)
            w = ix.search(Q, k, ef, routing=routing, eps=0.1, entries=want)
            parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), w, exact=routing == 0,
                                 what=f"routing {routing}, k {k}, efs {ef}")


def test_two_edges_per_lane_float_data(P):
    """R = 48, d = 100, L = 10 (GloVe-shaped unit vectors): >= 99% identical rows."""
    cfg = workloads.scaled(workloads.CONFIGS["glove"], 6000, 150)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 48)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    perm = oracle.dim_permutation(X, nbrs, 10)
    ix = oracle.Index(X, nbrs, entry, 10, 16, 5, perm=perm)
    codes = P.build_codes(G, Xt, 10, 16, 5, perm=torch.from_numpy(perm).cuda())
    gt, _ = oracle.knn_f64(X, Q, 10)
    for frame in (0, 1):
        ids, dists, _ = P.search(G, codes, Xt, Qt, 10, 64, routing=1, eps=0.2, frame=frame)
        want = ix.search(Q, 10, 64, routing=1, eps=0.2, frame=frame)
        parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=gt, what=f"frame {frame}")
    sh = oracle.SimHash(X, nbrs, 128, 6)
    sc = P.build_simhash(G, Xt, 128, 6)
    ids, dists, _ = P.search(G, sc, Xt, Qt, 10, 64, routing=2, eps=0.2)
    want = oracle.search(X, nbrs, entry, Q, 10, 64, routing=2, simhash=sh, eps=0.2)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=gt, what="SimHash")


@pytest.mark.parametrize("R", [1, 64])
def test_extreme_out_degrees(P, R):
    """The smallest and largest out-degree the library takes (R = 1: a ring through the
    points in id order, the longest walks; R = 64: the pruned graph in 64 slots, two
    edges per lane), plain routing bit for bit and PEOs at the parity bars, against the
    oracle on integer-valued rows."""
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 2000, 60)
    X, Q = workloads.generate(cfg)
    if R == 1:
        nbrs, entry = ((np.arange(len(X)) + 1) % len(X)).astype(np.int32)[:, None], 0
    else:
        nbrs, entry = build_graph(X, R)
    assert nbrs.shape[1] == R
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xt, 8, 16, 5)
    ix = oracle.Index(X, nbrs, entry, 8, 16, 5)
    gt, _ = oracle.knn_f64(X, Q, 10)
    for routing in (0, 1):
        for ef in (10, 64):
            ids, dists, cnt = P.search(G, codes, Xt, Qt, 10, ef, routing=routing, eps=0.2, eta_mode=1, counters=True)
            want = ix.search(Q, 10, ef, routing=routing, eps=0.2, eta_mode=1)
            what = f"R {R}, routing {routing}, efs {ef}"
            parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=gt, exact=routing == 0, what=what)
            parity.counters_parity(cnt.cpu().numpy(), want["counters"], 0, exact=routing == 0, what=what)
