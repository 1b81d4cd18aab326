"""Pins of the oracle's paper-literal frame Q (the projection table of q' = q / ||q|| built
once per query, A_r of Eq. (A_r) with r = ||p||^2 / 2 - p.q, plain FP32 dot products).

Fixed by: the threshold deciding cos(e, q) > A_r exactly when u is closer than delta
(the comparison Eq. A_r restates); H equal to the FP64 statistic of step 5 on
the table of q'; the special case where every neighbour passes; and searches in the two
frames agreeing on almost every result."""
import numpy as np
import pytest

import oracle
import workloads
from workloads.graph import build_graph


@pytest.fixture(scope="module", params=["glove", "sift"])
def small(request):
    """Unit-normalised glove-shaped rows (‖q‖ = 1, where frame Q is the angular form) and
    sift-shaped rows with norms in the thousands (where every ‖q‖ in the formulas counts)."""
    n = 4000 if request.param == "glove" else 3000
    cfg = workloads.scaled(workloads.CONFIGS[request.param], n, 40)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 16)
    ix = oracle.Index(X, nbrs, entry, cfg.L, cfg.m, cfg.proj_seed)
    return cfg, X, Q, nbrs, entry, ix


def test_frame_q_threshold_decides_the_distance_comparison(small):
    """cos(e, q) > A_r exactly when u is closer to q than delta (Eq. A_r; the frame-Q
    angle is between e and q itself, not the translated x = q - v)."""
    cfg, X, Q, nbrs, entry, ix = small
    rng = np.random.default_rng(2)
    checked = 0
    for qi in range(len(Q)):
        q = Q[qi].astype(np.float64)
        v, p = rng.integers(0, len(X), size=2)
        dv = float(np.sum((q - X[v]) ** 2))
        d2 = float(np.sum((q - X[p]) ** 2))
        f = ix.edge_stats(Q[qi], int(v), dv, d2, eps=0.2, frame=1, p=int(p))
        for s in np.nonzero(nbrs[v] >= 0)[0]:
            u = nbrs[v, s]
            e = X[u].astype(np.float64) - X[v]
            if np.linalg.norm(e) == 0:
                continue
            cos = e @ q / (np.linalg.norm(e) * np.linalg.norm(q))
            closer = np.sum((q - X[u]) ** 2) < d2
            if abs(cos - f["A"][s]) > 1e-5:
                assert (cos > f["A"][s]) == closer
                checked += 1
    assert checked > 300


def test_frame_q_H_is_the_statistic_of_the_normalised_query(small):
    """H of every edge that reaches the H >= T stage against the FP64 statistic of
    q' = q / ||q|| (step 5), for random expanded nodes v with p = the query's 10th nearest
    row (a list bound as a search would hold it), so that many edges have 0 < A < 1."""
    cfg, X, Q, nbrs, entry, ix = small
    L, m = cfg.L, cfg.m
    dp = X.shape[1] // L
    rng = np.random.default_rng(4)
    D = ((Q[:, None, :].astype(np.float64) - X[None].astype(np.float64)) ** 2).sum(-1)
    checked = 0
    for qi in range(len(Q)):
        q = Q[qi].astype(np.float64)
        qn = q / np.linalg.norm(q)
        p = int(np.argsort(D[qi])[9])
        for v in rng.integers(0, len(X), size=4):
            v = int(v)
            f = ix.edge_stats(Q[qi], v, float(D[qi, v]), float(D[qi, p]), eps=0.2, frame=1, p=p)
            for s in np.nonzero((nbrs[v] >= 0) & (f["kind"] == 2))[0]:
                cd = ix.codes[v, s].astype(int)
                h1 = sum(np.sign(cd[i]) * (qn[(i - 1) * dp:i * dp] @ ix.A[i - 1, abs(cd[i]) - 1].astype(np.float64))
                         for i in range(1, L + 1))
                h2 = np.sign(cd[0]) * (qn @ ix.B[abs(cd[0]) - 1].astype(np.float64))
                H = ix.wreg[v, s] * h1 + ix.cres[v, s] * h2
                assert abs(f["H"][s] - H) <= 1e-5 * max(abs(H), np.sqrt(L) * np.sqrt(2 * np.log(m)))
                checked += 1
    assert checked >= 20


def test_frame_q_searches(small):
    cfg, X, Q, nbrs, entry, ix = small
    plain = ix.search(Q, 10, 48, routing=0)
    always = ix.search(Q, 10, 48, routing=1, frame=1, test_mode=2)
    assert np.array_equal(plain["ids"], always["ids"])
    a = ix.search(Q, 10, 48, routing=1, eps=0.2, frame=0)
    b = ix.search(Q, 10, 48, routing=1, eps=0.2, frame=1)
    assert (np.all(a["ids"] == b["ids"], axis=1)).mean() >= 0.9
    assert b["counters"][:, 7].sum() < plain["counters"][:, 7].sum()


def test_frame_q_search_follows_the_test_definition():
    """The frame-Q search against the second implementation of Algorithm 1
    (tests/lossy_search.py) whose test is the frame-Q statistics of v's edges computed
    outside the search (pinned above against Eq. (A_r) and the FP64 statistic of q'),
    given p = the list's efs-th entry: the same trajectory, results and distance count.
    On sift-shaped rows (on the unit-normalised glove-shaped rows nearly every edge is
    accepted by A <= 0, so the H >= T stage would go untested)."""
    import lossy_search
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 3000, 10)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 16)
    ix = oracle.Index(X, nbrs, entry, cfg.L, cfg.m, cfg.proj_seed)
    orc = ix.search(Q[:10], 10, 32, routing=1, eps=0.2, frame=1, trace_cap=4096)
    tested = 0
    for qi in range(10):
        def test(v, dv, d2, p, q=Q[qi]):
            return ix.edge_stats(q, v, dv, d2, eps=0.2, frame=1, p=p)["passed"].astype(bool)
        ids, dists, trace, nd = lossy_search.search(X, nbrs, entry, Q[qi], 10, 32, test=test, bound_node=True)
        n_exp = int(orc["counters"][qi, 0])
        assert trace == orc["trace_v"][qi, :n_exp].tolist()
        assert np.array_equal(ids, orc["ids"][qi]) and np.array_equal(dists, orc["dists"][qi])
        assert nd == orc["counters"][qi, 7]
        tested += int(orc["counters"][qi, 5])
    assert tested > 100                      # the H >= T stage decided many edges


def test_quantile_table_is_slightly_conservative(small):
    """test_mode 3 (the quantile table of Sec. 4.3: variance on 256 L bins, the bin's upper
    edge) never rejects an edge the exact quantile passes, and lowers T by at most
    |z| (sqrt(var + 1/256) - sqrt(var))."""
    cfg, X, Q, nbrs, entry, ix = small
    z, c = oracle.test_constants(cfg.L, cfg.m, 0.2, 0)
    rng = np.random.default_rng(6)
    for qi in range(len(Q)):
        v, p = (int(t) for t in rng.integers(0, len(X), size=2))
        q = Q[qi].astype(np.float64)
        dv = float(np.sum((q - X[v]) ** 2))
        d2 = float(np.sum((q - X[p]) ** 2))
        a = ix.edge_stats(Q[qi], v, dv, d2, eps=0.2, frame=1, p=p)
        b = ix.edge_stats(Q[qi], v, dv, d2, eps=0.2, frame=1, p=p, test_mode=3)
        h = (a["kind"] == 2) & (nbrs[v] >= 0)
        assert np.all(b["passed"][h] >= a["passed"][h])
        assert np.all(b["T"][h] <= a["T"][h] + 1e-6)
        w, cr = ix.wreg[v][h].astype(np.float64), ix.cres[v][h].astype(np.float64)
        A = a["A"][h].astype(np.float64)
        var = np.maximum(w * w + cr * cr - cfg.L / (cfg.L + 1) * A * A, 0)
        assert np.all(a["T"][h] - b["T"][h] <= abs(z) * (np.sqrt(var + 1 / 256) - np.sqrt(var)) + 1e-5)


def test_quantile_table_search(small):
    cfg, X, Q, nbrs, entry, ix = small
    a = ix.search(Q, 10, 48, routing=1, eps=0.2, frame=1)
    b = ix.search(Q, 10, 48, routing=1, eps=0.2, frame=1, test_mode=3)
    # slightly more neighbours pass, so at least as many exact distances overall
    assert b["counters"][:, 6].sum() >= a["counters"][:, 6].sum() * 0.99
    assert (np.all(a["ids"] == b["ids"], axis=1)).mean() >= 0.8
