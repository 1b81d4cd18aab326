"""GPU parity: the CUDA path (through the C ABI) against the oracle on the same
seeded inputs.

Bars (tests/parity.py): integer/byte/index outputs bit-exact (codes, ids of the
records, random vectors); FP32 weights, tables, node terms, test statistics and
distances within 1e-5 relative, decisions equal outside the tolerance band; searches
with top-k ids identical on >= 99% of queries and recall@k within 0.3 points (plain
routing on integer-valued rows, where every distance is exact: bit for bit).  Sizes
span several CTAs/warps and a ragged tail of queries."""
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


class Dev:
    def __init__(self, P, case, build=True):
        self.case = case
        self.X = torch.from_numpy(case.X).cuda()
        self.Q = torch.from_numpy(case.Q).cuda()
        self.G = P.Graph.from_numpy(case.nbrs, case.entry)
        cfg = case.cfg
        self.codes = P.build_codes(self.G, self.X, cfg.L, cfg.m, cfg.proj_seed) if build else None


_devs = {}


def dev_of(P, case):
    key = id(case)
    if key not in _devs:
        _devs[key] = Dev(P, case)
    return _devs[key]


@pytest.mark.parametrize("seed,d,L,m", [(3000, 128, 8, 16), (3002, 100, 10, 16), (3004, 960, 24, 16), (7, 30, 3, 127)])
def test_projection_vectors_bitwise(P, seed, d, L, m):
    A1, B1 = P.projections(seed, d, L, m)
    A2, B2 = oracle.projections(seed, d, L, m)
    assert np.array_equal(A1.view(np.uint32), A2.view(np.uint32))
    assert np.array_equal(B1.view(np.uint32), B2.view(np.uint32))


@pytest.mark.parametrize("which", ["tiny", "sift20k"])
def test_build_codes_bitwise(P, tiny, sift20k, which):
    case = tiny if which == "tiny" else sift20k
    D = dev_of(P, case)
    arr = D.codes.arrays()
    ix = case.index
    assert np.array_equal(arr["ids"], case.nbrs)
    assert np.array_equal(arr["A"], ix.A) and np.array_equal(arr["B"], ix.B)
    assert np.array_equal(arr["codes"], ix.codes)
    assert np.array_equal(arr["enorm"].view(np.uint32), ix.enorm.view(np.uint32))
    assert np.array_equal(arr["wreg"].view(np.uint32), ix.wreg.view(np.uint32))
    assert np.array_equal(arr["cres"].view(np.uint32), ix.cres.view(np.uint32))
    # node tables (index time, the library's own summation order) and the node term of
    # every edge, S(t(v)), against FP64 restatements from the oracle's codes and weights
    X64 = case.X.astype(np.float64)
    L, m, d = case.cfg.L, case.cfg.m, case.X.shape[1]
    t0 = X64 @ ix.B.astype(np.float64).T
    tb = np.einsum("nlk,ljk->nlj", X64.reshape(len(X64), L, d // L), ix.A.astype(np.float64))
    tv_ref = np.concatenate([t0[:, None, :], tb], axis=1)
    tscale = np.linalg.norm(X64, axis=1)[:, None, None] * np.abs(np.concatenate(
        [np.linalg.norm(ix.B, axis=1)[None, :], np.linalg.norm(ix.A, axis=2)], axis=0))[None]
    assert np.all(parity.close(arr["tv"], tv_ref, tscale))
    assert np.all(parity.close(arr["tv"], ix.tv, tscale))
    sv_ref, sv_scale = parity.node_terms(tv_ref, ix.codes, ix.wreg, ix.cres)
    assert np.all(parity.close(arr["sv"], sv_ref, sv_scale))


@pytest.mark.parametrize("routing", [0, 1])
@pytest.mark.parametrize("ef", [16, 64, 200])
def test_search_parity_integer_data(P, sift20k, routing, ef):
    """SIFT-shaped integer data: exact distances, so plain routing matches bit for bit; the
    PEOs test's statistics differ from the oracle's by rounding only."""
    case = sift20k
    D = dev_of(P, case)
    k = case.cfg.k
    ids, dists, cnt = P.search(D.G, D.codes, D.X, D.Q, k, ef, eps=0.2, routing=routing, counters=True)
    torch.cuda.synchronize()
    orc = case.index.search(case.Q, k, ef, routing=routing, eps=0.2)
    exact = routing == 0
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), orc, gt=case.gt_ids, exact=exact)
    c = cnt.cpu().numpy()
    parity.counters_parity(c, orc["counters"], 0, exact=exact)   # same number of expansions
    assert np.all(c[:, 9] == 0)


@pytest.mark.parametrize("routing", [0, 1])
def test_search_parity_tiny(P, tiny, routing):
    case = tiny
    D = dev_of(P, case)
    cfg = case.cfg
    ids, dists, _ = P.search(D.G, D.codes, D.X, D.Q, cfg.k, cfg.ef, eps=cfg.eps, routing=routing)
    orc = case.index.search(case.Q, cfg.k, cfg.ef, routing=routing, eps=cfg.eps)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), orc, gt=case.gt_ids)


def test_edge_statistics(P, sift20k):
    """A, H, T and the decision of every edge of sampled expansions, by the search's own
    device code, against the oracle's plain evaluation (tests/parity.py's bars)."""
    case = sift20k
    D = dev_of(P, case)
    orc = case.index.search(case.Q[:20], 10, 64, routing=1, eps=0.2, trace_cap=512)
    z, c_eta = oracle.test_constants(case.cfg.L, case.cfg.m, 0.2)
    rng = np.random.default_rng(0)
    checked = flips = 0
    for qi in range(20):
        n_exp = int(min(orc["counters"][qi, 0], 512))
        d2 = orc["trace_d2"][qi, :n_exp]
        full = np.nonzero(np.isfinite(d2))[0]
        for t in rng.choice(full, size=min(4, len(full)), replace=False):
            v, dv, delta2 = int(orc["trace_v"][qi, t]), float(orc["trace_dv"][qi, t]), float(d2[t])
            g = P.edge_stats(D.codes, D.Q[qi], v, dv, delta2, eps=0.2)
            o = case.index.edge_stats(case.Q[qi], v, dv, delta2, eps=0.2)
            valid = case.nbrs[v] >= 0
            n, f = parity.stats_parity(g, o, valid, c_eta, parity.a_scale(dv, case.index.enorm[v], delta2))
            checked += n
            flips += f
    assert checked > 500
    assert flips <= 0.001 * checked, f"{flips} decisions differ inside the band of {checked}"


def test_edge_statistics_a_rules_and_degenerate_edges(P):
    """The search's device code on the edges where Algorithm 2's rules decide, against the
    oracle: a star of mixed edge lengths (one edge to a duplicate of v), a tight list bound
    under which the A >= 1 rule rejects the edges much longer or shorter than ||x||, a
    loose one under which the A <= 0 rule accepts the short edges, and q = v, where every
    edge passes as degenerate."""
    rng = np.random.default_rng(12)
    d, R, L, m = 64, 32, 8, 16
    v = rng.standard_normal(d)
    lengths = np.geomspace(0.05, 8.0, R)
    E = rng.standard_normal((R, d))
    E *= (lengths / np.linalg.norm(E, axis=1))[:, None]
    E[7] = 0.0
    X = np.vstack([v, v + E]).astype(np.float32)
    nbrs = np.full((R + 1, R), -1, dtype=np.int32)
    nbrs[0] = np.arange(1, R + 1)
    ix = oracle.Index(X, nbrs, 0, L, m, seed=4)
    G = P.Graph.from_numpy(nbrs, 0)
    Xd = torch.from_numpy(X).cuda()
    codes = P.build_codes(G, Xd, L, m, 4)
    q = (v + rng.standard_normal(d) / np.sqrt(d)).astype(np.float32)
    qd = torch.from_numpy(q).cuda()
    dv = oracle.dist2_f32(q, X[0])
    _, c_eta = oracle.test_constants(L, m, 0.2)
    valid = nbrs[0] >= 0
    for delta2, rule in ((0.25, 0), (float(dv) + 4.0, 1)):
        g = P.edge_stats(codes, qd, 0, float(dv), delta2, eps=0.2)
        o = ix.edge_stats(q, 0, float(dv), delta2, eps=0.2)
        parity.stats_parity(g, o, valid, c_eta, parity.a_scale(dv, ix.enorm[0], delta2))
        assert np.sum(g["kind"] == rule) >= 3
        assert np.all(g["passed"][g["kind"] == 0] == 0) and np.all(g["passed"][g["kind"] == 1] == 1)
        assert g["kind"][7] == 3 and g["passed"][7] == 1
    g = P.edge_stats(codes, torch.from_numpy(X[0]).cuda(), 0, 0.0, 0.25, eps=0.2)
    assert np.all(g["kind"] == 3) and np.all(g["passed"] == 1)
    codes.free()


def test_knn_bruteforce(P, sift20k, tiny):
    for case, exact in ((sift20k, True), (tiny, False)):
        D = dev_of(P, case)
        ids, dists = P.knn_bruteforce(D.X, D.Q, 10)
        ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
        if exact:
            assert np.array_equal(ids, case.gt_ids)
            assert np.array_equal(dists.astype(np.float64), case.gt_d)
        else:
            assert np.allclose(dists, case.gt_d, rtol=1e-5)
            assert np.mean(np.all(ids == case.gt_ids, axis=1)) >= 0.99


def test_host_api_equals_device_api(P, sift20k):
    case = sift20k
    D = dev_of(P, case)
    a_ids, a_d, a_c = P.search(D.G, D.codes, D.X, D.Q, 10, 48, routing=1, counters=True)
    b_ids, b_d, b_c = P.search_host(D.G, D.codes, D.X, case.Q, 10, 48, routing=1, counters=True)
    assert np.array_equal(a_ids.cpu().numpy(), b_ids)
    assert np.array_equal(a_d.cpu().numpy(), b_d)
    assert np.array_equal(a_c.cpu().numpy(), b_c)


@pytest.mark.parametrize("slots,warps", [(256, 1), (1024, 4), (16384, 2), (0, 8)])
def test_launch_shapes_do_not_change_results(P, sift20k, slots, warps):
    case = sift20k
    D = dev_of(P, case)
    ref = P.search(D.G, D.codes, D.X, D.Q, 10, 64, routing=1)
    got = P.search(D.G, D.codes, D.X, D.Q, 10, 64, routing=1, visited_slots=slots, warps_per_cta=warps)
    assert torch.equal(ref[0], got[0]) and torch.equal(ref[1], got[1])


def test_automatic_visited_table_long_lists(P, sift20k):
    """At efs 144 the automatic visited table (16 efs -> 4,096 slots, 16 KB per query)
    would leave one CTA of 8 warps per SM; the launcher lowers it to the largest size
    that keeps the launch shape's register-bound CTAs resident (512 slots at 4 rows per
    gather batch).  The table is lossy, so the results equal those of the full-size
    table bit for bit, and they meet the oracle's at the parity bars."""
    case = sift20k
    D = dev_of(P, case)
    ix = oracle.Index(case.X, case.nbrs, case.entry, case.cfg.L, case.cfg.m, case.cfg.proj_seed, lazy=True)
    for routing, g in ((1, 4), (1, 8), (0, 8)):
        auto = P.search(D.G, D.codes, D.X, D.Q, 10, 144, routing=routing, eps=0.3, eta_mode=1, gather_rows=g,
                        counters=True)
        full = P.search(D.G, D.codes, D.X, D.Q, 10, 144, routing=routing, eps=0.3, eta_mode=1, gather_rows=g,
                        visited_slots=4096)
        assert torch.equal(auto[0], full[0]) and torch.equal(auto[1], full[1])
        want = ix.search(case.Q, 10, 144, routing=routing, eps=0.3, eta_mode=1)
        what = f"routing {routing}, G {g}"
        parity.search_parity(auto[0].cpu().numpy(), auto[1].cpu().numpy(), want, gt=case.gt_ids,
                             exact=routing == 0, what=what)
        parity.counters_parity(auto[2].cpu().numpy(), want["counters"], 0, what=what)


def test_edge_cases(P):
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 3000, 37)
    X, Q = workloads.generate(cfg)
    # duplicated vectors (degenerate edges), queries equal to base points, ragged degrees
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
    arr = codes.arrays()
    assert np.array_equal(arr["codes"], ix.codes) and np.array_equal(arr["enorm"], ix.enorm)
    for routing in (0, 1):
        for k, ef in ((1, 1), (1, 8), (10, 10), (10, 512), (100, 1024)):
            ids, dists, cnt = P.search(G, codes, Xt, Qt, k, ef, routing=routing, eps=0.1, counters=True)
            orc = ix.search(Q, k, ef, routing=routing, eps=0.1)
            what = f"routing {routing}, k {k}, efs {ef}"
            parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), orc, exact=routing == 0, what=what)
            parity.counters_parity(cnt.cpu().numpy(), orc["counters"], 0, exact=routing == 0, what=what)
    # empty query batch
    ids, dists, _ = P.search(G, codes, Xt, Qt[:0], 10, 32)
    assert ids.shape == (0, 10)
    # expansion cap reports overflow per query
    _, _, cnt = P.search(G, codes, Xt, Qt, 10, 64, max_expansions=3, counters=True)
    assert np.all(cnt.cpu().numpy()[:, 9] == 4)


def test_wide_degree_and_other_dims(P):
    """R = 48 (two edges per lane), d = 100, L = 10 (GloVe-shaped, unit vectors)."""
    cfg = workloads.scaled(workloads.CONFIGS["glove"], 4000, 45)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 48)
    ix = oracle.Index(X, nbrs, entry, 10, 16, 4)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xt, 10, 16, 4)
    arr = codes.arrays()
    assert np.array_equal(arr["codes"], ix.codes)
    gt, _ = oracle.knn_f64(X, Q, 10)
    for routing in (0, 1):
        ids, dists, _ = P.search(G, codes, Xt, Qt, 10, 64, routing=routing, eps=0.2)
        orc = ix.search(Q, 10, 64, routing=routing, eps=0.2)
        parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), orc, gt=gt, what=f"routing {routing}")


@pytest.mark.parametrize("R", [7, 37])
def test_odd_degree_records(P, R):
    """Odd out-degrees (the record's arrays start at offsets that are not multiples of 8
    unless padded) on integer-valued data: codes, scalars and results bit for bit."""
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 3000, 40)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, R)
    ix = oracle.Index(X, nbrs, entry, 8, 16, 9)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xt, 8, 16, 9)
    arr = codes.arrays()
    assert np.array_equal(arr["ids"], nbrs) and np.array_equal(arr["codes"], ix.codes)
    for f in ("enorm", "wreg", "cres"):
        assert np.array_equal(arr[f].view(np.uint32), getattr(ix, f).view(np.uint32)), f
    sv_ref, sv_scale = parity.node_terms(ix.tv, ix.codes, ix.wreg, ix.cres)
    assert np.all(parity.close(arr["sv"], sv_ref, sv_scale))
    for routing in (0, 1):
        ids, dists, _ = P.search(G, codes, Xt, Qt, 10, 40, routing=routing, eps=0.2)
        orc = ix.search(Q, 10, 40, routing=routing, eps=0.2)
        parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), orc, exact=routing == 0)


def test_invalid_arguments(P, sift20k):
    case = sift20k
    D = dev_of(P, case)
    with pytest.raises(P.PeosError, match="INVAL"):
        P.search(D.G, D.codes, D.X, D.Q, 20, 10)                      # k > ef
    with pytest.raises(P.PeosError, match="INVAL"):
        P.search(D.G, D.codes, D.X, D.Q, 10, 32, eps=0.0)             # eps outside (0, 0.5]
    with pytest.raises(P.PeosError, match="INVAL"):
        P.search(D.G, D.codes, D.X, D.Q, 10, 32, eps=0.7)
    with pytest.raises(P.PeosError, match="INVAL"):
        P.search(D.G, None, D.X, D.Q, 10, 32, routing=1)              # PEOs without codes
    with pytest.raises(P.PeosError, match="INVAL"):
        P.build_codes(D.G, D.X, 7, 16, 1)                            # L does not divide d
    with pytest.raises(P.PeosError, match="INVAL"):
        P.build_codes(D.G, D.X, 8, 200, 1)                           # m > 127
    bad = case.nbrs.copy()
    bad[5, 3] = len(case.X) + 10
    with pytest.raises(P.PeosError, match="INVAL"):
        P.build_codes(P.Graph.from_numpy(bad, case.entry), D.X, 8, 16, 1)
    # a plain search over an unvalidated graph never reads outside the base
    ids, _, _ = P.search(P.Graph.from_numpy(bad, case.entry), None, D.X, D.Q, 10, 32, routing=0)
    assert int(ids.max()) < len(case.X)


def test_long_rows(P):
    """GIST-shaped rows (d = 960, L = 24, three code words per edge): the kernels read such
    a query from global memory instead of shared memory; results meet the same bars, also
    over BF16 rows with the FP32 re-rank and with a beam width of 2 (query in shared
    memory again)."""
    cfg = workloads.scaled(workloads.CONFIGS["gist"], 3000, 60)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 32)
    ix = oracle.Index(X, nbrs, entry, 24, 16, 11)
    gt, _ = oracle.knn_f64(X, Q, 10)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xt, 24, 16, 11)
    for routing in (0, 1):
        for ef, g in ((16, 4), (64, 8), (200, 8)):
            ids, dists, cnt = P.search(G, codes, Xt, Qt, 10, ef, routing=routing, eps=0.2, gather_rows=g,
                                       counters=True)
            want = ix.search(Q, 10, ef, routing=routing, eps=0.2)
            what = f"routing {routing}, efs {ef}"
            parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=gt, what=what)
            parity.counters_parity(cnt.cpu().numpy(), want["counters"], 0, what=what)
        b = P.search(G, codes, Xt, Qt, 10, 48, routing=routing, eps=0.2, beam=2)
        want = ix.search(Q, 10, 48, routing=routing, eps=0.2, beam=2)
        parity.search_parity(b[0].cpu().numpy(), b[1].cpu().numpy(), want, gt=gt, what=f"beam 2, routing {routing}")
    st = P.quantize(Xt, "bf16")
    _, _, deq = oracle.quantize(X, "bf16")
    ids, dists, _ = P.search(G, codes, st, Qt, 10, 48, routing=1, eps=0.2, rerank=Xt)
    want = ix.search(Q, 10, 48, routing=1, eps=0.2, base=deq, rerank=X)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=gt, what="bf16 rows, re-ranked")
