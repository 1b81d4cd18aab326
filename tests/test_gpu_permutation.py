"""GPU parity of the dimension permutation (Appendix D.1) and of indexes built in
permuted coordinates, against the oracle on the same seeded inputs.

The permutation itself is bit-exact on integer-valued rows (every FP64 sum of squared
differences is exact there, so the summation order cannot matter); on float rows it must
agree wherever the per-coordinate means are not within rounding of each other.  Codes and
weights of a permuted index are bit-exact on integer data, as for the unpermuted index;
node tables, node terms, test statistics and searches meet the bars of tests/parity.py."""
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


def _avg(X, nbrs):
    v, s = np.nonzero(nbrs >= 0)
    acc = np.zeros(X.shape[1])
    for c in range(0, len(v), 200_000):
        E = X[nbrs[v[c:c + 200_000], s[c:c + 200_000]]].astype(np.float64) - X[v[c:c + 200_000]].astype(np.float64)
        acc += (E * E).sum(axis=0)
    return acc / len(v)


@pytest.mark.parametrize("L", [8, 4, 16, 128])
def test_permutation_integer_data_bit_exact(P, sift20k, L):
    case = sift20k
    X = torch.from_numpy(case.X).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    got = P.dim_permutation(G, X, L).cpu().numpy()
    want = oracle.dim_permutation(case.X, case.nbrs, L)
    assert np.array_equal(got, want)


def test_permutation_float_data(P):
    cfg = workloads.scaled(workloads.CONFIGS["glove"], 8000, 10)
    X, _ = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 24)
    G = P.Graph.from_numpy(nbrs, entry)
    got = P.dim_permutation(G, torch.from_numpy(X).cuda(), cfg.L).cpu().numpy()
    want = oracle.dim_permutation(X, nbrs, cfg.L)
    assert sorted(got.tolist()) == list(range(X.shape[1]))
    if not np.array_equal(got, want):
        # only a rounding-level near-tie of two means may reorder coordinates
        avg = _avg(X, nbrs)
        srt = np.sort(avg)
        gaps = np.diff(srt) / np.maximum(srt[1:], 1e-300)
        assert gaps.min() < 1e-12, "permutations differ without a near-tie of means"


def test_permutation_degenerate_cases(P):
    X = np.arange(2 * 12, dtype=np.float32).reshape(2, 12)
    # no edges: every mean is 0, subspaces take coordinates in order
    nbrs = np.full((2, 4), -1, dtype=np.int32)
    G = P.Graph.from_numpy(nbrs, 0)
    got = P.dim_permutation(G, torch.from_numpy(X).cuda(), 3).cpu().numpy()
    assert np.array_equal(got, oracle.dim_permutation(X, nbrs, 3))
    # L = d (one coordinate per subspace) and L = 1 (identity order by mean)
    nbrs = np.array([[1, -1, -1, -1], [0, -1, -1, -1]], dtype=np.int32)
    G = P.Graph.from_numpy(nbrs, 0)
    for L in (1, 12):
        got = P.dim_permutation(G, torch.from_numpy(X).cuda(), L).cpu().numpy()
        assert np.array_equal(got, oracle.dim_permutation(X, nbrs, L)), L
    with pytest.raises(P.PeosError):
        P.dim_permutation(G, torch.from_numpy(X).cuda(), 5)  # L must divide d


@pytest.fixture(scope="module")
def permuted(P, sift20k):
    case = sift20k
    cfg = case.cfg
    perm = oracle.dim_permutation(case.X, case.nbrs, cfg.L)
    ix = oracle.Index(case.X, case.nbrs, case.entry, cfg.L, cfg.m, cfg.proj_seed, perm=perm)
    X = torch.from_numpy(case.X).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    codes = P.build_codes(G, X, cfg.L, cfg.m, cfg.proj_seed, perm=torch.from_numpy(perm).cuda())
    return case, perm, ix, X, G, codes


def test_permuted_codes_bitwise(P, permuted):
    case, perm, ix, X, G, codes = permuted
    arr = codes.arrays()
    assert np.array_equal(arr["codes"], ix.codes)
    for f in ("enorm", "wreg", "cres"):
        assert np.array_equal(arr[f].view(np.uint32), getattr(ix, f).view(np.uint32)), f
    Xp = case.X[:, perm].astype(np.float64)
    tscale = np.linalg.norm(Xp, axis=1)[:, None, None] * 8.0
    assert np.all(parity.close(arr["tv"], ix.tv, tscale))
    sv_ref, sv_scale = parity.node_terms(ix.tv, ix.codes, ix.wreg, ix.cres)
    assert np.all(parity.close(arr["sv"], sv_ref, sv_scale))
    # the handle holds its own copy (the fixture's device tensor is gone by now)
    assert codes.info()["perm"]
    # and the codes differ from the unpermuted ones (the permutation is not the identity)
    plain = P.build_codes(G, X, case.cfg.L, case.cfg.m, case.cfg.proj_seed).arrays()
    assert not np.array_equal(plain["codes"], arr["codes"])


@pytest.mark.parametrize("ef", [10, 64, 200])
def test_permuted_search(P, permuted, ef):
    case, perm, ix, X, G, codes = permuted
    Q = torch.from_numpy(case.Q).cuda()
    ids, dists, cnt = P.search(G, codes, X, Q, 10, ef, eps=0.2, routing=1, counters=True)
    want = ix.search(case.Q, 10, ef, routing=1, eps=0.2)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids)
    c = cnt.cpu().numpy()
    parity.counters_parity(c, want["counters"], 0)  # same number of expansions
    # along the same trajectory the GPU's visited table (lossy: a forgotten node is tested
    # again) can only add to the test counters
    same = c[:, 0] == want["counters"][:, 0]
    for name in ("a_reject", "a_accept", "n_dist"):
        i = P.COUNTER_NAMES.index(name)
        assert np.all(c[same, i] >= want["counters"][same, i]), name


def test_permuted_uneven_batch(P, permuted):
    case, perm, ix, X, G, codes = permuted
    rng = np.random.default_rng(4)
    nq = len(case.Q)
    k = rng.choice([1, 10, 50], size=nq).astype(np.int32)
    ef = np.maximum(rng.integers(32, 129, size=nq), k).astype(np.int32)
    ids, dists, _ = P.search_batch(G, codes, X, torch.from_numpy(case.Q).cuda(), 50, 128,
                                   torch.from_numpy(k).cuda(), torch.from_numpy(ef).cuda(), routing=1, eps=0.2)
    oi = np.full((nq, 50), -1, np.int32)
    od = np.full((nq, 50), np.inf, np.float32)
    for kk, ee in sorted(set(zip(k.tolist(), ef.tolist()))):
        sel = np.nonzero((k == kk) & (ef == ee))[0]
        r = ix.search(case.Q[sel], kk, ee, routing=1, eps=0.2)
        oi[sel, :kk] = r["ids"]
        od[sel, :kk] = r["dists"]
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), dict(ids=oi, dists=od))


def test_permuted_edge_statistics(P, permuted):
    case, perm, ix, X, G, codes = permuted
    _, c_eta = oracle.test_constants(case.cfg.L, case.cfg.m, 0.2)
    rng = np.random.default_rng(9)
    checked = 0
    for qi in rng.choice(len(case.Q), 12, replace=False):
        v = int(rng.integers(0, len(case.X)))
        dv = float(np.float32(np.sum((case.Q[qi].astype(np.float64) - case.X[v]) ** 2)))
        got = P.edge_stats(codes, torch.from_numpy(case.Q[qi]).cuda(), v, dv, dv * 1.5, eps=0.2)
        want = ix.edge_stats(case.Q[qi], v, dv, dv * 1.5, eps=0.2)
        ok = case.nbrs[v] >= 0  # empty slots carry no statistics
        n, _ = parity.stats_parity(got, want, ok, c_eta, parity.a_scale(dv, ix.enorm[v], dv * 1.5))
        checked += n
    assert checked > 50


def test_permuted_generic_table_path(P):
    """m > 16 builds the query table with the generic (not k-major) builder."""
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 4000, 37)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 20)
    L, m = 8, 32
    perm = oracle.dim_permutation(X, nbrs, L)
    ix = oracle.Index(X, nbrs, entry, L, m, 77, perm=perm)
    G = P.Graph.from_numpy(nbrs, entry)
    Xd = torch.from_numpy(X).cuda()
    codes = P.build_codes(G, Xd, L, m, 77, perm=P.dim_permutation(G, Xd, L))
    ids, dists, _ = P.search(G, codes, Xd, torch.from_numpy(Q).cuda(), 10, 48, eps=0.2, routing=1)
    want = ix.search(Q, 10, 48, routing=1, eps=0.2)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want)


def test_bad_permutations_rejected(P, sift20k):
    case = sift20k
    X = torch.from_numpy(case.X).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    d = X.shape[1]
    dup = torch.arange(d, dtype=torch.int32, device="cuda")
    dup[5] = 6
    with pytest.raises(P.PeosError, match="permutation"):
        P.build_codes(G, X, 8, 16, 1, perm=dup)
    out = torch.arange(d, dtype=torch.int32, device="cuda")
    out[0] = d
    with pytest.raises(P.PeosError, match="permutation"):
        P.build_codes(G, X, 8, 16, 1, perm=out)
    big = torch.zeros((4, 2052), dtype=torch.float32, device="cuda")
    Gb = P.Graph.from_numpy(np.full((4, 2), -1, dtype=np.int32), 0)
    with pytest.raises(P.PeosError):
        P.dim_permutation(Gb, big, 4)
