"""The comparison helpers the GPU parity tests rely on (tests/parity.py) have teeth.

Each is fed the oracle's own output twice (which must pass) and then the oracle's output
against a copy with a planted difference: ids changed on more than 1% of the queries,
distances moved by twice the relative tolerance, one distance one ulp off where bit
equality is asked for, recall moved by more than 0.3 points, a counter differing on more
than 1% of the queries, a test statistic moved beyond its tolerance, a decision flipped
away from the tolerance band.  Each planted difference must fail the helper, while a
decision flipped inside the band passes and is counted."""
import math

import numpy as np
import pytest

import oracle
import parity
import workloads
from workloads.graph import build_graph


@pytest.fixture(scope="module")
def search_case():
    cfg = workloads.scaled(workloads.CONFIGS["glove"], 3000, 200)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 16)
    ix = oracle.Index(X, nbrs, entry, cfg.L, cfg.m, cfg.proj_seed)
    r = ix.search(Q, 10, 32, routing=1, eps=0.2)
    gt, _ = oracle.knn_f64(X, Q, 10)
    return r, gt


def test_search_parity_accepts_itself_and_rejects_planted_differences(search_case):
    r, gt = search_case
    ids, d = r["ids"].copy(), r["dists"].copy()
    assert parity.search_parity(ids, d, r, gt=gt) == 1.0
    assert parity.search_parity(ids, d, r, gt=gt, exact=True) == 1.0
    nq = len(ids)
    # ids changed on 2% of the queries (a result replaced by another row of the base)
    bad = ids.copy()
    bad[: math.ceil(0.02 * nq), -1] = (bad[: math.ceil(0.02 * nq), -1] + 1) % 3000
    with pytest.raises(AssertionError):
        parity.search_parity(bad, d, r)
    # one query in a hundred may differ
    ok = ids.copy()
    ok[0, -1] = (ok[0, -1] + 1) % 3000
    assert parity.search_parity(ok, d, r) >= 0.99
    # distances 2e-5 relative off
    with pytest.raises(AssertionError):
        parity.search_parity(ids, (d.astype(np.float64) * (1 + 2e-5)).astype(np.float32), r)
    # bit equality asked for: one ulp on one distance fails
    ulp = d.copy()
    ulp[5, 3] = np.nextafter(ulp[5, 3], np.float32(np.inf))
    parity.search_parity(ids, ulp, r)  # within the tolerance
    with pytest.raises(AssertionError):
        parity.search_parity(ids, ulp, r, exact=True)
    # recall moved by more than 0.3 points (with top-k ids still identical on 99%)
    worse = ids.copy()
    worse[:2, :] = np.arange(3000 - 10, 3000)[None]  # two queries' lists replaced by far rows
    assert abs(parity.recall(worse, gt) - parity.recall(ids, gt)) > parity.RECALL_PTS
    with pytest.raises(AssertionError, match="recall"):
        parity.search_parity(worse, d, r, gt=gt, min_same=0.0)


def test_counters_parity(search_case):
    r, _ = search_case
    c = r["counters"].copy()
    assert parity.counters_parity(c, r["counters"], 0, exact=True) == 1.0
    bad = c.copy()
    bad[: math.ceil(0.02 * len(c)), 0] += 1
    with pytest.raises(AssertionError):
        parity.counters_parity(bad, r["counters"], 0)
    one = c.copy()
    one[0, 0] += 1
    assert parity.counters_parity(one, r["counters"], 0) >= 0.99
    with pytest.raises(AssertionError):
        parity.counters_parity(one, r["counters"], 0, exact=True)


@pytest.fixture(scope="module")
def stats_case():
    """Test statistics of one node's edges from the oracle, with the list bound placed so
    that the edges spread over 0 < A < 1 (most of them reach the H >= T stage)."""
    rng = np.random.default_rng(5)
    d, R, L, m = 128, 32, 8, 16
    v = rng.standard_normal(d)
    E = rng.standard_normal((R, d)) * 0.3
    X = np.vstack([v, v + E]).astype(np.float32)
    nbrs = np.full((R + 1, R), -1, dtype=np.int32)
    nbrs[0] = np.arange(1, R + 1)
    q = (v + 0.3 * rng.standard_normal(d)).astype(np.float32)
    ix = oracle.Index(X, nbrs, 0, L, m, seed=9)
    dv = oracle.dist2_f32(q, X[0])
    en2 = float(np.median((E.astype(np.float64) ** 2).sum(1)))
    delta2 = float(dv + en2 - 0.3 * math.sqrt(dv * en2))
    st = ix.edge_stats(q, 0, dv, delta2, eps=0.2)
    c_eta = math.sqrt(L) * oracle.eta(m, 0)
    s_A = parity.a_scale(dv, ix.enorm[0], delta2)
    valid = nbrs[0] >= 0
    assert np.sum(st["kind"] == 2) >= 10
    return st, valid, c_eta, s_A


def _copy(st):
    return {k: np.array(v, copy=True) for k, v in st.items()}


def test_stats_parity_accepts_itself_and_rejects_planted_differences(stats_case):
    st, valid, c_eta, s_A = stats_case
    n, flips = parity.stats_parity(_copy(st), st, valid, c_eta, s_A)
    assert n == valid.sum() and flips == 0
    tested = np.nonzero(st["kind"] == 2)[0]
    far = tested[np.argmax(np.abs(st["H"][tested] - st["T"][tested]))]
    # H moved by 1e-4 of its scale on one edge
    g = _copy(st)
    g["H"][far] += 1e-4 * c_eta
    with pytest.raises(AssertionError):
        parity.stats_parity(g, st, valid, c_eta, s_A)
    # T moved likewise
    g = _copy(st)
    g["T"][far] -= 1e-4 * c_eta
    with pytest.raises(AssertionError):
        parity.stats_parity(g, st, valid, c_eta, s_A)
    # A moved beyond its tolerance
    g = _copy(st)
    i = tested[0]
    g["A"][i] += 1e-4 * max(abs(float(st["A"][i])), float(s_A[i]))
    with pytest.raises(AssertionError):
        parity.stats_parity(g, st, valid, c_eta, s_A)
    # a decision flipped far from the band
    g = _copy(st)
    g["passed"][far] = 1 - g["passed"][far]
    with pytest.raises(AssertionError):
        parity.stats_parity(g, st, valid, c_eta, s_A)
    # a decision flipped where H and T agree to within the band: passes, counted
    g = _copy(st)
    o = _copy(st)
    near = tested[np.argmin(np.abs(st["H"][tested] - st["T"][tested]))]
    o["T"][near] = o["H"][near]                      # the oracle's statistic sits on the threshold
    o["passed"][near] = 1
    g["H"][near] = o["H"][near]
    g["T"][near] = np.float32(o["H"][near] + 1e-6 * c_eta)
    g["passed"][near] = 0
    n, flips = parity.stats_parity(g, o, valid, c_eta, s_A)
    assert flips == 1


def test_close_is_relative_to_the_largest_magnitude():
    assert parity.close([1.0], [1.0 + 0.9e-5], 0.0).all()
    assert not parity.close([1.0], [1.0 + 1.1e-5], 0.0).any()
    # a small value compared on the scale of the terms it came from
    assert parity.close([1e-9], [5e-6], 1.0).all()
    assert not parity.close([1e-9], [5e-6], 0.1).any()
    # infinities (empty result slots) are never "close": search_parity checks them apart
    with np.errstate(invalid="ignore"):
        assert not parity.close([np.inf], [np.inf], 0.0).any()
