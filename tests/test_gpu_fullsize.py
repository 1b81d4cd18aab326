"""Parity at the full SIFT-shaped size (1,000,000 x 128 integer-valued rows, 10,000
queries, R=32, L=8, m=16) in the launch configuration the benchmark times: the whole
batch in one call with the default launch shape.  The oracle recomputes a seeded sample
of the queries one by one (its index builds only the nodes they touch): plain routing
matches bit for bit on this integer data, PEOs within the bars of tests/parity.py."""
import numpy as np
import pytest
import torch

import oracle
import parity
import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def full():
    import paper_2402_11354_gb300 as P
    cfg = workloads.CONFIGS["sift"]
    X, Q = workloads.dataset(cfg)
    nbrs, entry = workloads.load_graph(cfg, X, device="cuda")
    Xd, Qd = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xd, cfg.L, cfg.m, cfg.proj_seed)
    ix = oracle.Index(X, nbrs, entry, cfg.L, cfg.m, cfg.proj_seed, lazy=True)
    sample = np.sort(np.random.default_rng(7).choice(len(Q), 200, replace=False))
    return P, cfg, X, Q, Xd, Qd, G, codes, ix, sample


@pytest.mark.parametrize("routing,ef,eps,eta", [(0, 16, 0.2, 0), (1, 18, 0.2, 1), (1, 64, 0.1, 0)])
def test_full_size_sampled(full, routing, ef, eps, eta):
    P, cfg, X, Q, Xd, Qd, G, codes, ix, sample = full
    ids, dists, cnt = P.search(G, codes, Xd, Qd, cfg.k, ef, eps=eps, routing=routing, eta_mode=eta, counters=True)
    orc = ix.search(Q[sample], cfg.k, ef, routing=routing, eps=eps, eta_mode=eta)
    ids, dists, cnt = ids.cpu().numpy(), dists.cpu().numpy(), cnt.cpu().numpy()
    exact = routing == 0
    parity.search_parity(ids[sample], dists[sample], orc, exact=exact)
    parity.counters_parity(cnt[sample], orc["counters"], 0, exact=exact)   # same expansions
    same = cnt[sample, 0] == orc["counters"][:, 0]
    # along the same trajectory the lossy visited table can only add re-evaluations of
    # forgotten nodes
    assert np.all(cnt[sample, 7][same] >= orc["counters"][same, 7])
    assert np.all(cnt[:, 9] == 0)


def test_full_size_stored_rows_sampled(full):
    """E4M3 storage with the FP32 re-rank at full size: sampled queries follow the oracle
    on the dequantised rows; re-ranked distances are exact (integer data)."""
    P, cfg, X, Q, Xd, Qd, G, codes, ix, sample = full
    st = P.quantize(Xd, "e4m3")
    _, _, deq = oracle.quantize(X, "e4m3")
    ids, dists, _ = P.search(G, codes, st, Qd, cfg.k, 24, eps=0.2, routing=1, eta_mode=1, rerank=Xd)
    orc = ix.search(Q[sample], cfg.k, 24, routing=1, eps=0.2, eta_mode=1, base=deq, rerank=X)
    ids, dists = ids.cpu().numpy()[sample], dists.cpu().numpy()[sample]
    parity.search_parity(ids, dists, orc)
    same = np.all(ids == orc["ids"], axis=1)
    assert np.array_equal(dists[same].view(np.uint32), orc["dists"][same].view(np.uint32))  # exact re-rank
