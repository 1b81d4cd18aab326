"""GPU parity of the hierarchical entry (greedy descent through HNSW-style upper layers)
and of searches with per-query entries, against the oracle on the same seeded inputs.

On integer-valued rows every distance is exact on both sides, so the descent and the
plain search that starts from its result match bit for bit (PEOs: the bars of
tests/parity.py); on float rows the warp's reduction order may break a near-tie
differently, so >= 99% of entries must agree."""
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
def env(P, sift20k):
    case = sift20k
    layers, top = build_hierarchy(case.X, 32, seed=11, M=8, min_nodes=32)
    X = torch.from_numpy(case.X).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    codes = P.build_codes(G, X, case.cfg.L, case.cfg.m, case.cfg.proj_seed)
    H = P.Hierarchy(layers, top)
    return case, layers, top, X, G, codes, H


def test_descent_bitwise_integer_data(P, env):
    case, layers, top, X, G, codes, H = env
    assert len(layers) >= 3
    got = P.hier_entry(H, X, torch.from_numpy(case.Q).cuda()).cpu().numpy()
    want, hops = oracle.hier_entries(case.X, case.Q, layers, top)
    assert np.array_equal(got, want)
    assert hops.mean() > 1  # the walks do move


def test_descent_on_stored_rows(P, env):
    case, layers, top, X, G, codes, H = env
    st = P.quantize(X, "bf16")  # integers 0..255 are exact in BF16
    got = P.hier_entry(H, st, torch.from_numpy(case.Q).cuda()).cpu().numpy()
    want, _ = oracle.hier_entries(case.X, case.Q, layers, top)
    assert np.array_equal(got, want)


def test_descent_float_data(P):
    cfg = workloads.scaled(workloads.CONFIGS["glove"], 12000, 300)
    X, Q = workloads.generate(cfg)
    layers, top = build_hierarchy(X, 24, seed=2, M=8, min_nodes=32)
    got = P.hier_entry(P.Hierarchy(layers, top), torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()).cpu().numpy()
    want, _ = oracle.hier_entries(X, Q, layers, top)
    assert (got == want).mean() >= 0.99


@pytest.mark.parametrize("routing", [0, 1])
@pytest.mark.parametrize("ef", [10, 64])
def test_search_from_hierarchical_entries(P, env, routing, ef):
    case, layers, top, X, G, codes, H = env
    Q = torch.from_numpy(case.Q).cuda()
    ent = P.hier_entry(H, X, Q)
    ids, dists, cnt = P.search(G, codes, X, Q, 10, ef, eps=0.2, routing=routing, counters=True, entries=ent)
    want = case.index.search(case.Q, 10, ef, routing=routing, eps=0.2, entries=ent.cpu().numpy())
    exact = routing == 0
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids, exact=exact)
    parity.counters_parity(cnt.cpu().numpy(), want["counters"], 0, exact=exact)


def test_entries_through_batch_and_host_calls(P, env):
    case, layers, top, X, G, codes, H = env
    Q = torch.from_numpy(case.Q).cuda()
    ent = P.hier_entry(H, X, Q)
    a, _, _ = P.search(G, codes, X, Q, 10, 48, eps=0.2, routing=1, entries=ent)
    nq = len(case.Q)
    b, _, _ = P.search_batch(G, codes, X, Q, 10, 48, torch.full((nq,), 10, dtype=torch.int32, device="cuda"),
                             torch.full((nq,), 48, dtype=torch.int32, device="cuda"), routing=1, eps=0.2, entries=ent)
    c, _, _ = P.search_host(G, codes, X, case.Q, 10, 48, eps=0.2, routing=1, entries=ent.cpu().numpy())
    d, _, _ = P.search_noalloc(G, codes, X, Q, 10, 48, eps=0.2, routing=1, entries=ent)
    a = a.cpu().numpy()
    assert np.array_equal(a, b.cpu().numpy()) and np.array_equal(a, c) and np.array_equal(a, d.cpu().numpy())
    # all entries equal to the graph's entry: the plain single-entry search
    same = torch.full((nq,), case.entry, dtype=torch.int32, device="cuda")
    e, _, _ = P.search(G, codes, X, Q, 10, 48, eps=0.2, routing=1, entries=same)
    f, _, _ = P.search(G, codes, X, Q, 10, 48, eps=0.2, routing=1)
    assert np.array_equal(e.cpu().numpy(), f.cpu().numpy())


def test_invalid_entries_give_empty_rows(P, env):
    case, layers, top, X, G, codes, H = env
    nq = len(case.Q)
    ent = torch.full((nq,), case.entry, dtype=torch.int32, device="cuda")
    ent[3] = -1
    ent[7] = len(case.X)
    ids, dists, cnt = P.search(G, codes, X, torch.from_numpy(case.Q).cuda(), 10, 32, routing=1, counters=True,
                               entries=ent)
    ids, dists, cnt = ids.cpu().numpy(), dists.cpu().numpy(), cnt.cpu().numpy()
    assert np.all(ids[[3, 7]] == -1) and np.all(np.isinf(dists[[3, 7]]))
    assert np.all(cnt[[3, 7], 9] == 1) and np.all(np.delete(cnt[:, 9], [3, 7]) == 0)


def test_hierarchy_checks(P, env):
    case, layers, top, X, G, codes, H = env
    Q = torch.from_numpy(case.Q[:4]).cuda()
    with pytest.raises(P.PeosError, match="top_entry"):
        P.hier_entry(P.Hierarchy(layers, len(layers[0]["ids"])), X, Q)
    wide = [dict(l) for l in layers]
    wide[-1]["nbrs"] = np.full((len(wide[-1]["ids"]), 33), -1, dtype=np.int32)
    with pytest.raises(P.PeosError, match="R <= 32"):
        P.hier_entry(P.Hierarchy(wide, top), X, Q)
    # a layer naming rows outside the base ends the walk with entry -1 (no read outside X)
    bad = [dict(l) for l in layers]
    bad[-1]["ids"] = bad[-1]["ids"].copy()
    bad[-1]["ids"][:] = len(case.X) + 5
    got = P.hier_entry(P.Hierarchy(bad, top), X, Q).cpu().numpy()
    assert np.all(got == -1)
    with pytest.raises(TypeError):  # one entry per query
        P.search(G, codes, X, Q, 10, 32, entries=torch.zeros(3, dtype=torch.int32, device="cuda"))
