"""Pins of the oracle's SimHash test (Sec. 3.1, Lemma 4.1), the baseline routing test
with the residual remedy: per-edge sign bits of S_i . e, the query's bits in the frame
translated by -v, and a Hoeffding threshold on the collision count.

Fixed by: the bits against FP64 signs; Lemma 4.1 (the fraction of differing bits
estimates theta / pi) on random pairs; the translated bits against the signs of
S_i . (q - v); the threshold's coverage guarantee (Definition 3.1) by Monte Carlo over
the binomial collision count, and its power; and the special cases that reduce the
search to plain routing."""
import numpy as np
import pytest

import oracle
import workloads
from workloads.graph import build_graph


def _pairs(E):
    n, d = E.shape
    X = np.zeros((2 * n, d), dtype=np.float32)
    X[1::2] = E
    nbrs = np.full((2 * n, 1), -1, dtype=np.int32)
    nbrs[0::2, 0] = np.arange(1, 2 * n, 2)
    return X, nbrs


def _unpack(bits, K):
    w = np.arange(K) // 64
    b = np.arange(K) % 64
    return ((bits[..., w] >> b.astype(np.uint64)) & np.uint64(1)).astype(bool)


@pytest.mark.parametrize("K", [64, 128, 192])
def test_bits_and_norms_match_definitions(K):
    rng = np.random.default_rng(K)
    E = rng.standard_normal((300, 48)).astype(np.float32)
    X, nbrs = _pairs(E)
    sh = oracle.SimHash(X, nbrs, K, seed=9)
    dots = E.astype(np.float64) @ sh.S.astype(np.float64).T
    got = _unpack(sh.bits[0::2, 0], K)
    clear = np.abs(dots) > 1e-4
    assert np.array_equal(got[clear], (dots >= 0)[clear])
    assert np.allclose(sh.en[0::2, 0], np.linalg.norm(E.astype(np.float64), axis=1), rtol=1e-6)
    assert np.all(sh.bits[1::2] == 0) and np.all(sh.en[1::2] == 0)  # empty slots


def test_lemma41_hamming_fraction_estimates_angle():
    rng = np.random.default_rng(3)
    d, n, K = 32, 4000, 192
    # pairs at angles spread over (0.1, 3.0): V = cos t U' + sin t W' with W' orthogonal to U
    U = rng.standard_normal((n, d))
    W = rng.standard_normal((n, d))
    W -= (np.sum(W * U, 1) / np.sum(U * U, 1))[:, None] * U
    t = rng.uniform(0.1, 3.0, size=n)
    Vv = np.cos(t)[:, None] * U / np.linalg.norm(U, axis=1)[:, None] + \
        np.sin(t)[:, None] * W / np.linalg.norm(W, axis=1)[:, None]
    theta = np.arccos(np.clip(np.sum(U * Vv, 1) / np.linalg.norm(U, axis=1) / np.linalg.norm(Vv, axis=1), -1, 1))
    X1, nb1 = _pairs(U.astype(np.float32))
    X2, nb2 = _pairs(Vv.astype(np.float32))
    a = _unpack(oracle.SimHash(X1, nb1, K, seed=4).bits[0::2, 0], K)
    b = _unpack(oracle.SimHash(X2, nb2, K, seed=4).bits[0::2, 0], K)
    frac = (a != b).mean(1)
    # E[frac] = theta / pi; average over pairs binned by angle
    for lo in (0.3, 0.8, 1.3, 1.8, 2.3):
        sel = (theta >= lo) & (theta < lo + 0.5)
        assert abs(frac[sel].mean() - (theta[sel] / np.pi).mean()) < 0.01


@pytest.mark.parametrize("K,eps", [(64, 0.1), (128, 0.2), (192, 0.05)])
def test_threshold_coverage_and_power(K, eps):
    ac = oracle.simhash_acrit(K, eps)
    assert ac[K] == 1.0 and np.all(np.diff(ac) >= 0)
    rng = np.random.default_rng(K)
    # an edge exactly at the bound (theta = arccos A): passes with probability >= 1 - eps
    for A in (0.1, 0.3, 0.6, 0.9):
        p = 1 - np.arccos(A) / np.pi
        col = rng.binomial(K, p, size=200_000)
        assert (A <= ac[col]).mean() >= 1 - eps
    # and an edge far beyond it (angle near pi/2 when A = 0.9) is mostly rejected
    col = rng.binomial(K, 1 - (np.pi / 2) / np.pi, size=100_000)
    assert (np.float32(0.9) <= ac[col]).mean() < 0.5


@pytest.fixture(scope="module")
def small():
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 5000, 50)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 16)
    sh = oracle.SimHash(X, nbrs, 64, seed=21)
    return X, Q, nbrs, entry, sh


def test_search_follows_the_test_definition(small):
    """The oracle's SimHash search against a second implementation of Algorithm 1
    (tests/lossy_search.py) whose test is restated here: the bits of x = q - v from FP64
    signs of S_i . x, #Col = K - popcount(bits(e) xor bits(x)), A in the translated frame,
    pass iff A <= acrit[#Col] (A >= 1 rejects, A <= 0 accepts)."""
    import lossy_search
    X, Q, nbrs, entry, sh = small
    K, eps = 64, 0.1
    acrit = oracle.simhash_acrit(K, eps)
    S = sh.S.astype(np.float64)
    ebits = _unpack(sh.bits.reshape(-1, 1), K).reshape(len(X), nbrs.shape[1], K)

    def make_test(q):
        def test(v, dv, delta2):
            xb = (S @ (q.astype(np.float64) - X[v].astype(np.float64))) >= 0
            en = sh.en[v]
            f = np.float32
            with np.errstate(divide="ignore", invalid="ignore"):
                A = ((f(dv) + en * en) - f(delta2)) / (f(2.0) * (np.sqrt(f(dv)) * en))
            col = K - (ebits[v] != xb[None, :]).sum(1)
            out = np.where(A >= 1, False, np.where(A <= 0, True, A <= acrit[col]))
            return np.where((en == 0) | (dv == 0), True, out)
        return test

    r = oracle.search(X, nbrs, entry, Q[:10], 10, 32, routing=2, simhash=sh, eps=eps, trace_cap=4096)
    same = 0
    for qi in range(10):
        ids, dists, trace, nd = lossy_search.search(X, nbrs, entry, Q[qi], 10, 32, test=make_test(Q[qi]))
        n_exp = int(r["counters"][qi, 0])
        same += trace == r["trace_v"][qi, :n_exp].tolist() and np.array_equal(ids, r["ids"][qi]) \
            and nd == r["counters"][qi, 7]
    assert same >= 9            # a sign at rounding level may differ between FP32 and FP64


def test_search_special_cases(small):
    X, Q, nbrs, entry, sh = small
    plain = oracle.search(X, nbrs, entry, Q, 10, 32, routing=0)
    always = oracle.search(X, nbrs, entry, Q, 10, 32, routing=2, simhash=sh, eps=0.1, test_mode=2)
    assert np.array_equal(plain["ids"], always["ids"]) and np.array_equal(plain["counters"], always["counters"])
    cut = oracle.search(X, nbrs, entry, Q, 10, 32, routing=2, simhash=sh, eps=0.1, test_mode=1)
    assert np.array_equal(plain["ids"], cut["ids"])
    r = oracle.search(X, nbrs, entry, Q, 10, 32, routing=2, simhash=sh, eps=0.1)
    c, p = r["counters"], plain["counters"]
    assert c[:, 7].sum() < p[:, 7].sum()                  # the test saves distances
    assert c[:, 5].sum() > 0 and c[:, 6].sum() < c[:, 5].sum()
    full = oracle.search(X, nbrs, entry, Q, 10, len(X), routing=2, simhash=sh, eps=0.1)
    gt, _ = oracle.knn_f64(X, Q, 10)
    assert np.array_equal(full["ids"], gt)                # efs = N: exact
