"""GPU parity of the beam width W (W nodes expanded per iteration; Algorithm 1 with
the reading of the oracle: the W unexpanded entries of R with the smallest (dist, id),
the list bound frozen for the iteration, nodes tested in list order with earlier passes
of the iteration counting as visited, all passes inserted in ascending (dist, id)).

Plain routing on integer-valued rows matches the oracle bit for bit (trajectory, ids,
distances); PEOs meets the bars of tests/parity.py.  Uneven batches, R = 48 (two edges per
lane), ragged graphs with duplicate vectors, a visited table small enough to forget nodes
within an iteration, the smallest and largest lists, and every launch shape are covered;
variants without a W > 1 kernel are refused."""
import numpy as np
import pytest
import torch

import oracle
import parity
import workloads
from workloads.graph import build_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module")
def env(P, sift20k):
    case = sift20k
    X, Q = torch.from_numpy(case.X).cuda(), torch.from_numpy(case.Q).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    codes = P.build_codes(G, X, case.cfg.L, case.cfg.m, case.cfg.proj_seed)
    return case, X, Q, G, codes


@pytest.mark.parametrize("beam", [2, 4])
@pytest.mark.parametrize("ef", [16, 64, 200])
def test_plain_beam_bitwise_integer_data(P, env, beam, ef):
    case, X, Q, G, codes = env
    ids, dists, cnt = P.search(G, None, X, Q, 10, ef, routing=0, beam=beam, counters=True)
    want = oracle.search(case.X, case.nbrs, case.entry, case.Q, 10, ef, routing=0, beam=beam)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids, exact=True)
    c = cnt.cpu().numpy()
    parity.counters_parity(c, want["counters"], 0, exact=True)
    assert np.all(c[:, 9] == 0)


@pytest.mark.parametrize("beam", [2, 4])
@pytest.mark.parametrize("ef,eps", [(16, 0.2), (64, 0.1), (200, 0.2)])
def test_peos_beam(P, env, beam, ef, eps):
    case, X, Q, G, codes = env
    ids, dists, cnt = P.search(G, codes, X, Q, 10, ef, eps=eps, routing=1, beam=beam, counters=True)
    want = case.index.search(case.Q, 10, ef, routing=1, eps=eps, beam=beam)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids)
    c = cnt.cpu().numpy()
    parity.counters_parity(c, want["counters"], 0)
    assert np.all(c[:, 9] == 0)


def test_beam_one_is_the_default(P, env):
    case, X, Q, G, codes = env
    for routing in (0, 1):
        a = P.search(G, codes, X, Q, 10, 48, routing=routing)
        b = P.search(G, codes, X, Q, 10, 48, routing=routing, beam=1)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


@pytest.mark.parametrize("beam", [2, 4])
def test_beam_launch_shapes_do_not_change_results(P, env, beam):
    case, X, Q, G, codes = env
    for routing in (0, 1):
        ref = P.search(G, codes, X, Q, 10, 64, routing=routing, beam=beam)
        for slots, warps, g in ((256, 1, 4), (1024, 4, 8), (16384, 2, 4), (0, 8, 8)):
            got = P.search(G, codes, X, Q, 10, 64, routing=routing, beam=beam, visited_slots=slots,
                           warps_per_cta=warps, gather_rows=g)
            assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1]), (routing, slots, warps, g)


@pytest.mark.parametrize("beam", [2, 4])
def test_beam_uneven_batch(P, env, beam):
    case, X, Q, G, codes = env
    rng = np.random.default_rng(13)
    nq = len(case.Q)
    k = rng.choice([1, 10, 100], size=nq).astype(np.int32)
    ef = np.maximum(rng.integers(32, 257, size=nq), k).astype(np.int32)
    for routing in (0, 1):
        ids, dists, _ = P.search_batch(G, codes, X, Q, 100, 256, torch.from_numpy(k).cuda(),
                                       torch.from_numpy(ef).cuda(), routing=routing, eps=0.2, beam=beam)
        oi = np.full((nq, 100), -1, np.int32)
        od = np.full((nq, 100), np.inf, np.float32)
        for kk, ee in sorted(set(zip(k.tolist(), ef.tolist()))):
            sel = np.nonzero((k == kk) & (ef == ee))[0]
            r = case.index.search(case.Q[sel], kk, ee, routing=routing, eps=0.2, beam=beam)
            oi[sel, :kk] = r["ids"]
            od[sel, :kk] = r["dists"]
        parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), dict(ids=oi, dists=od), exact=routing == 0)


@pytest.mark.parametrize("beam", [2, 4])
def test_beam_ragged_graph_and_list_sizes(P, beam):
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 3000, 37)
    X, Q = workloads.generate(cfg)
    X[100:110] = X[200]
    Q[:5] = X[[0, 200, 1234, 2999, 105]]
    nbrs, entry = build_graph(X, 32)
    rng = np.random.default_rng(5)
    drop = rng.random(nbrs.shape) < 0.3
    drop[:, 0] = False
    nbrs = np.where(drop, -1, nbrs).astype(np.int32)
    ix = oracle.Index(X, nbrs, entry, 8, 16, 9)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xt, 8, 16, 9)
    for routing in (0, 1):
        for k, ef in ((1, 1), (1, 8), (10, 10), (10, 512), (100, 1024)):
            for slots in (0, 256):   # 256 slots: nodes forgotten within an iteration
                ids, dists, cnt = P.search(G, codes, Xt, Qt, k, ef, routing=routing, eps=0.1, beam=beam,
                                           visited_slots=slots, counters=True)
                want = ix.search(Q, k, ef, routing=routing, eps=0.1, beam=beam)
                what = f"routing {routing}, k {k}, efs {ef}, slots {slots}"
                parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, exact=routing == 0, what=what)
                parity.counters_parity(cnt.cpu().numpy(), want["counters"], 0, exact=routing == 0, what=what)


@pytest.mark.parametrize("beam", [2, 4])
def test_beam_two_edges_per_lane(P, beam):
    """R = 48 (two edges per lane, more candidates per iteration), GloVe-shaped float data."""
    cfg = workloads.scaled(workloads.CONFIGS["glove"], 6000, 150)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 48)
    ix = oracle.Index(X, nbrs, entry, 10, 16, 5)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xt, 10, 16, 5)
    gt, _ = oracle.knn_f64(X, Q, 10)
    for routing in (0, 1):
        ids, dists, _ = P.search(G, codes, Xt, Qt, 10, 64, routing=routing, eps=0.2, beam=beam)
        want = ix.search(Q, 10, 64, routing=routing, eps=0.2, beam=beam)
        parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=gt, what=f"routing {routing}")


def test_beam_argument_checks(P, env):
    case, X, Q, G, codes = env
    with pytest.raises(P.PeosError, match="beam"):
        P.search(G, codes, X, Q, 10, 32, routing=1, beam=3)
    with pytest.raises(P.PeosError, match="beam 2 / 4"):
        P.search(G, codes, X, Q, 10, 32, routing=1, frame=1, beam=2)
    sh = P.build_simhash(G, X, 64, 3)
    with pytest.raises(P.PeosError, match="beam 2 / 4"):
        P.search(G, sh, X, Q, 10, 32, routing=2, beam=2)
    cc = P.build_codes(G, X, 8, 16, 9, scalar_bits=8)
    with pytest.raises(P.PeosError, match="beam 2 / 4"):
        P.search(G, cc, X, Q, 10, 32, routing=1, beam=4)
    # reduced-precision rows are searched with W > 1 too
    st = P.quantize(X, "bf16")   # integers 0..255 are exact in BF16
    a = P.search(G, codes, X, Q, 10, 48, routing=1, beam=2)
    b = P.search(G, codes, st, Q, 10, 48, routing=1, beam=2)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))
