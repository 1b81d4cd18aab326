"""GPU tests of uneven batches (per-query k and efs in one persistent launch, caller
workspace, CUDA-graph capture) and of the launch-shape autotuner.

Every query of an uneven batch must return what the oracle returns for that query
searched alone with its own k and efs (the bars of tests/parity.py; plain routing on
integer-valued data: bit-exact); every launch shape must give the same results, and so
must the launch captured and replayed."""
import numpy as np
import pytest
import torch

import oracle
import parity
from conftest import get_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module")
def env(P):
    case = get_case("sift", 20_000, 200)
    X, Q = torch.from_numpy(case.X).cuda(), torch.from_numpy(case.Q).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    codes = P.build_codes(G, X, case.cfg.L, case.cfg.m, case.cfg.proj_seed)
    rng = np.random.default_rng(11)
    nq = len(case.Q)
    k = rng.choice([1, 10, 100], size=nq).astype(np.int32)
    ef = np.maximum(rng.integers(32, 257, size=nq), k).astype(np.int32)
    return case, X, Q, G, codes, k, ef


def oracle_uneven(case, k, ef, k_max, routing, eps=0.2, base=None, rerank=None):
    ids = np.full((len(case.Q), k_max), -1, np.int32)
    dists = np.full((len(case.Q), k_max), np.inf, np.float32)
    for kk, ee in sorted(set(zip(k.tolist(), ef.tolist()))):
        sel = np.nonzero((k == kk) & (ef == ee))[0]
        r = case.index.search(case.Q[sel], kk, ee, routing=routing, eps=eps, base=base, rerank=rerank)
        ids[sel, :kk] = r["ids"]
        dists[sel, :kk] = r["dists"]
    return ids, dists


@pytest.mark.parametrize("routing", [0, 1])
def test_uneven_batch_equals_oracle_per_query(P, env, routing):
    case, X, Q, G, codes, k, ef = env
    kq, efq = torch.from_numpy(k).cuda(), torch.from_numpy(ef).cuda()
    ids, dists, cnt = P.search_batch(G, codes, X, Q, 100, 256, kq, efq, routing=routing, counters=True)
    oi, od = oracle_uneven(case, k, ef, 100, routing)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), dict(ids=oi, dists=od), exact=routing == 0)
    assert np.all(cnt.cpu().numpy()[:, 9] == 0)


def test_every_launch_shape_gives_the_same_results(P, env):
    from paper_2402_11354_gb300.batch import candidate_shapes
    case, X, Q, G, codes, k, ef = env
    kq, efq = torch.from_numpy(k).cuda(), torch.from_numpy(ef).cuda()
    ref = None
    for sh in candidate_shapes(256):
        for routing in (0, 1):
            try:
                ids, dists, _ = P.search_batch(G, codes, X, Q, 100, 256, kq, efq, routing=routing, **sh.kw())
            except P.PeosError as e:
                assert e.status == 6  # shared memory beyond the per-CTA limit
                continue
            got = (ids.cpu().numpy(), dists.cpu().numpy())
            if ref is None:
                ref = {}
            if routing not in ref:
                ref[routing] = got
            assert np.array_equal(got[0], ref[routing][0]), sh
            assert np.array_equal(got[1].view(np.uint32), ref[routing][1].view(np.uint32)), sh


def test_autotune_and_graph_replay(P, env):
    from paper_2402_11354_gb300.batch import BatchPlan, autotune
    case, X, Q, G, codes, k, ef = env
    kq, efq = torch.from_numpy(k).cuda(), torch.from_numpy(ef).cuda()
    tr = autotune(G, codes, X, Q, 100, 256, kq, efq, routing=1, eps=0.2, reps=1)
    assert tr.table and tr.ms == min(t for _, t in tr.table)
    plan = BatchPlan(G, codes, X, X.shape[1], len(case.Q), 100, 256, shape=tr.best, routing=1, eps=0.2)
    plan.load(Q, kq, efq)
    plan.capture()
    # new contents after capture: the replay reads the plan's buffers
    perm = torch.randperm(len(case.Q), generator=torch.Generator().manual_seed(3)).cuda()
    plan.load(Q[perm], kq[perm], efq[perm])
    ids, dists = plan.run()
    torch.cuda.synchronize()
    oi, od = oracle_uneven(case, k, ef, 100, 1)
    p = perm.cpu().numpy()
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), dict(ids=oi[p], dists=od[p]))
    ids2, dists2 = plan.run()  # a second replay gives the same
    assert torch.equal(ids2, ids) and torch.equal(dists2, dists)
    # and the captured launch returns what a plain call with the same shape returns
    direct = P.search_batch(G, codes, X, Q[perm], 100, 256, kq[perm], efq[perm], routing=1, eps=0.2,
                            **tr.best.kw())
    assert torch.equal(direct[0], ids) and torch.equal(direct[1], dists)


def test_invalid_per_query_values_give_empty_rows(P, env):
    case, X, Q, G, codes, k, ef = env
    k2, ef2 = k.copy(), ef.copy()
    bad = [0, 5, 17, 42]
    k2[0] = 0          # k < 1
    k2[5] = 101        # k > k_max
    ef2[17] = 300      # efs > ef_max
    k2[42], ef2[42] = 100, 64  # k > efs
    ids, dists, cnt = P.search_batch(G, codes, X, Q, 100, 256, torch.from_numpy(k2).cuda(),
                                     torch.from_numpy(ef2).cuda(), routing=1, counters=True)
    ids, dists, cnt = ids.cpu().numpy(), dists.cpu().numpy(), cnt.cpu().numpy()
    assert np.all(ids[bad] == -1) and np.all(np.isinf(dists[bad]))
    assert np.all(cnt[bad, 9] == 1) and np.all(np.delete(cnt[:, 9], bad) == 0)
    good = np.setdiff1d(np.arange(len(k)), bad)
    oi, od = oracle_uneven(case, k, ef, 100, 1)
    parity.search_parity(ids[good], dists[good], dict(ids=oi[good], dists=od[good]))


def test_uneven_batch_with_stored_rows_and_rerank(P, env):
    case, X, Q, G, codes, k, ef = env
    st = P.quantize(X, "e4m3")
    _, _, deq = oracle.quantize(case.X, "e4m3")
    ids, dists, _ = P.search_batch(G, codes, st, Q, 100, 256, torch.from_numpy(k).cuda(), torch.from_numpy(ef).cuda(),
                                   routing=1, rerank=X)
    oi, od = oracle_uneven(case, k, ef, 100, 1, base=deq, rerank=case.X)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), dict(ids=oi, dists=od))
    same = np.all(ids.cpu().numpy() == oi, axis=1)
    d = dists.cpu().numpy()
    assert np.array_equal(d[same].view(np.uint32), od[same].view(np.uint32))   # exact re-rank


def test_workspace_checks(P, env):
    case, X, Q, G, codes, k, ef = env
    need = P.batch_workspace_size(G, codes, X, len(case.Q), 100, 256)
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PeosError, match="workspace"):
        P.search_batch(G, codes, X, Q, 100, 256, workspace=small)
    big = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    with pytest.raises(P.PeosError, match="aligned"):
        P.search_batch(G, codes, X, Q, 100, 256, workspace=big[16:])
