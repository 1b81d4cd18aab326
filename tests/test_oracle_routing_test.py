"""Pins of the oracle's PEOs routing test (Sec. 4.2 steps (4)-(6), Algorithm 2).

- A, H, T of every edge against FP64 evaluations of the definitions: H from the
  normalised query direction (step 5), T as scipy's eps-quantile of N^{e,A}_min
  (Eq. N_ex_min), A in the frame translated by -v.
- The translated A equals the paper's A_r (Eq. A_r) evaluated literally in the
  translated coordinates; dist(u, q) < delta exactly when cos(e, q - v) > A, so
  A >= 1 rejects only neighbours at distance >= delta (proof of Theorem 5.3 (1)).
- Monte Carlo over fresh projection vectors: mean and variance of H against
  Eq. (combination) with the finite-m moments of max_j |g_j|; equal block norms give
  mean sqrt(L) mu_m cos(theta) (Lemma 5.2).
- Coverage (Definition 3.1 / Theorem 5.3 (1)): a neighbour closer than delta passes
  with probability >= 1 - eps when eta is the finite-m mean.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle


def _star(d, R, seed, equal_blocks=False, L=8):
    """Node 0 = v; nodes 1..R = u_s; returns X, nbrs, query."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(d)
    E = rng.standard_normal((R, d))
    if equal_blocks:
        b = E.reshape(R, L, d // L)
        b /= np.linalg.norm(b, axis=2, keepdims=True)
        E = b.reshape(R, d)
    E /= np.linalg.norm(E, axis=1, keepdims=True)
    X = np.vstack([v, v + E]).astype(np.float32)
    nbrs = np.full((R + 1, R), -1, dtype=np.int32)
    nbrs[0] = np.arange(1, R + 1)
    q = (v + 0.8 * rng.standard_normal(d) / math.sqrt(d)).astype(np.float32)
    return X, nbrs, q


def _definitions(ix, q, v, dv, delta2, eps):
    """FP64 A, H, T of every out-edge of v from the definitions."""
    L, m = ix.L, ix.m
    d = ix.d
    dp = d // L
    x = q.astype(np.float64) - ix.X[v].astype(np.float64)
    qn = x / np.linalg.norm(x)
    A_, H_, T_ = [], [], []
    eta = math.sqrt(2 * math.log(m))
    for s in range(ix.R):
        u = ix.nbrs[v, s]
        if u < 0:
            A_.append(np.nan); H_.append(np.nan); T_.append(np.nan)
            continue
        e = ix.X[u].astype(np.float64) - ix.X[v].astype(np.float64)
        en = np.linalg.norm(e)
        A = (dv + en * en - delta2) / (2.0 * math.sqrt(dv) * en)
        c = ix.codes[v, s].astype(int)
        wr = float(ix.wreg[v, s])
        wres = math.sqrt(max(0.0, 1 - wr * wr))
        h1 = sum(np.sign(c[i]) * qn[(i - 1) * dp:i * dp] @ ix.A[i - 1, abs(c[i]) - 1].astype(np.float64)
                 for i in range(1, L + 1))
        h2 = np.sign(c[0]) * qn @ ix.B[abs(c[0]) - 1].astype(np.float64)
        H = wr * h1 + math.sqrt(L) * wres * h2
        var = wr * wr + L * wres * wres - L * A * A / (L + 1)
        T = stats.norm.ppf(eps, loc=A * math.sqrt(2 * L * math.log(m)), scale=math.sqrt(var)) if 0 < A < 1 else np.nan
        A_.append(A); H_.append(H); T_.append(T)
    return np.array(A_), np.array(H_), np.array(T_)


@pytest.mark.parametrize("eps", [0.1, 0.2])
def test_edge_statistics_match_definitions(eps):
    X, nbrs, q = _star(128, 32, 7)
    ix = oracle.Index(X, nbrs, 0, 8, 16, seed=21)
    dv = oracle.dist2_f32(q, X[0])
    delta2 = np.float32(dv + 0.5)
    st = ix.edge_stats(q, 0, dv, float(delta2), eps=eps)
    A, H, T = _definitions(ix, q, 0, float(dv), float(delta2), eps)
    L = 8
    scaleA = (dv + 1.0 + delta2) / (2 * math.sqrt(dv))
    assert np.all(np.abs(st["A"] - A) <= 1e-5 * np.maximum(np.abs(A), scaleA))
    mid = (A > 1e-6) & (A < 1 - 1e-6)
    assert mid.sum() >= 10
    s = math.sqrt(L) * math.sqrt(2 * math.log(16))
    assert np.all(np.abs(st["H"][mid] - H[mid]) <= 1e-5 * np.maximum(np.abs(H[mid]), s))
    assert np.all(np.abs(st["T"][mid] - T[mid]) <= 1e-5 * np.maximum(np.abs(T[mid]), s))
    band = np.abs(H[mid] - T[mid]) > 1e-4 * s
    assert np.array_equal(st["passed"][mid][band], (H[mid] >= T[mid])[band])
    assert np.all(st["passed"][A >= 1] == 0) and np.all(st["passed"][A <= 0] == 1)


@pytest.mark.parametrize("eps", [0.1, 0.2])
def test_edge_statistics_match_definitions_sift_scale(eps):
    """The same definitions at the norms of SIFT-shaped data: integer-valued rows in
    0..255 (||v|| ~ 1.7e3), neighbours and the query close to v (||q|| / ||x|| >= 5), so
    that any evaluation that cancels large terms (a table of q minus a table of v, or
    norms expanded into inner products) would show its rounding here."""
    rng = np.random.default_rng(31)
    d, R, L = 128, 32, 8
    v = rng.integers(0, 256, d).astype(np.float64)
    E = np.rint(rng.normal(0.0, 14.0, (R, d)))
    X = np.clip(np.vstack([v, v + E]), 0, 255).astype(np.float32)
    nbrs = np.full((R + 1, R), -1, dtype=np.int32)
    nbrs[0] = np.arange(1, R + 1)
    q = np.clip(v + np.rint(rng.normal(0.0, 9.0, d)), 0, 255).astype(np.float32)
    ix = oracle.Index(X, nbrs, 0, L, 16, seed=23)
    dv = oracle.dist2_f32(q, X[0])
    assert np.linalg.norm(q) / math.sqrt(dv) >= 5.0
    en2 = ((X[1:].astype(np.float64) - X[0]) ** 2).sum(1)
    # delta chosen so that the edges spread over 0 < A < 1
    delta2 = np.float32(dv + np.median(en2) - 0.2 * math.sqrt(dv) * math.sqrt(np.median(en2)))
    st = ix.edge_stats(q, 0, dv, float(delta2), eps=eps)
    A, H, T = _definitions(ix, q, 0, float(dv), float(delta2), eps)
    s = math.sqrt(L) * math.sqrt(2 * math.log(16))
    scaleA = (dv + en2 + delta2) / (2 * math.sqrt(dv) * np.sqrt(en2))
    assert np.all(np.abs(st["A"] - A) <= 1e-5 * np.maximum(np.abs(A), scaleA))
    mid = (A > 1e-5) & (A < 1 - 1e-5)
    assert mid.sum() >= 10
    assert np.all(np.abs(st["H"][mid] - H[mid]) <= 1e-5 * np.maximum(np.abs(H[mid]), s))
    assert np.all(np.abs(st["T"][mid] - T[mid]) <= 1e-5 * np.maximum(np.abs(T[mid]), s))
    band = np.abs(H[mid] - T[mid]) > 1e-4 * s
    assert np.array_equal(st["passed"][mid][band], (H[mid] >= T[mid])[band])
    assert 0 < st["passed"][mid].sum() < mid.sum()        # both outcomes occur


def test_translated_A_is_paper_A_r():
    """Eq. (A_r) with v' = 0, u' = e, q' = x, p' any point at distance delta from x."""
    rng = np.random.default_rng(8)
    for _ in range(200):
        d = 64
        x, e, w = rng.standard_normal((3, d))
        w /= np.linalg.norm(w)
        delta = abs(rng.normal(np.linalg.norm(x), 1.0))
        p = x + delta * w
        r = p @ p / 2 - p @ x
        A_r = (e @ e / 2 - r - 0.0) / (np.linalg.norm(x) * np.linalg.norm(e))
        A_T = (x @ x + e @ e - delta ** 2) / (2 * np.linalg.norm(x) * np.linalg.norm(e))
        assert A_r == pytest.approx(A_T, rel=1e-9, abs=1e-9)
        # dist(u, q) = ||e - x|| < delta exactly when cos(e, x) > A; hence A >= 1 implies dist >= delta
        cos = e @ x / (np.linalg.norm(x) * np.linalg.norm(e))
        dist = np.linalg.norm(e - x)
        if abs(cos - A_T) > 1e-9:
            assert (cos > A_T) == (dist < delta)
        if A_T >= 1:
            assert dist >= delta - 1e-9


def test_a_rules_decide_by_distance_and_degenerate_cases_pass():
    """Algorithm 2's two rules on a star whose edges have mixed lengths, with the bound δ
    chosen so that both fire: every edge with A >= 1 is rejected and every edge with
    A <= 0 accepted, and the A >= 1 rule only rejects neighbours at distance >= δ
    (A >= 1 means |‖x‖ - ‖e‖| >= δ, so ‖e - x‖ >= δ; proof of Theorem 5.3 (1)).  The
    degenerate cases (R10): an edge to a duplicate of v (‖e‖ = 0) passes, and with q = v
    (‖x‖ = 0) every edge passes."""
    rng = np.random.default_rng(12)
    d, R, L = 64, 32, 8
    v = rng.standard_normal(d)
    lengths = np.geomspace(0.05, 8.0, R)
    E = rng.standard_normal((R, d))
    E *= (lengths / np.linalg.norm(E, axis=1))[:, None]
    E[7] = 0.0                                        # u_7 duplicates v
    X = np.vstack([v, v + E]).astype(np.float32)
    nbrs = np.full((R + 1, R), -1, dtype=np.int32)
    nbrs[0] = np.arange(1, R + 1)
    ix = oracle.Index(X, nbrs, 0, L, 16, seed=4)
    q = (v + rng.standard_normal(d) / math.sqrt(d)).astype(np.float32)   # ||x|| ~ 1
    dv = oracle.dist2_f32(q, X[0])
    dist2 = ((X[1:].astype(np.float64) - q.astype(np.float64)) ** 2).sum(1)
    # a tight bound: A >= 1 for the edges much longer or much shorter than ||x||
    delta2 = 0.25
    st = ix.edge_stats(q, 0, dv, delta2, eps=0.2)
    A, kinds = st["A"].astype(np.float64), st["kind"]
    assert np.sum(kinds == 0) >= 3
    assert np.all(st["passed"][kinds == 0] == 0) and np.all(A[kinds == 0] >= 1)
    assert np.all(dist2[kinds == 0] >= delta2 * (1 - 1e-6))
    assert kinds[7] == 3 and st["passed"][7] == 1
    # a loose bound: A <= 0 wherever ||x||^2 + ||e||^2 <= delta^2
    delta2 = float(dv) + 4.0
    st = ix.edge_stats(q, 0, dv, delta2, eps=0.2)
    A, kinds = st["A"].astype(np.float64), st["kind"]
    assert np.sum(kinds == 1) >= 3
    assert np.all(st["passed"][kinds == 1] == 1) and np.all(A[kinds == 1] <= 0)
    assert np.all(np.isin(kinds[lengths ** 2 < 4.0 - 1e-3], (1, 3)))   # accepted by A <= 0 (or degenerate)
    assert kinds[7] == 3 and st["passed"][7] == 1
    # q = v: x = 0, every edge passes as degenerate
    st0 = ix.edge_stats(X[0], 0, 0.0, delta2, eps=0.2)
    assert np.all(st0["passed"] == 1) and np.all(st0["kind"] == 3)


def _mc_H(d, L, R, seeds, eps=0.2, eta_mode=0, equal_blocks=False, delta_for=None):
    X, nbrs, q = _star(d, R, 11, equal_blocks=equal_blocks, L=L)
    dv = oracle.dist2_f32(q, X[0])
    H = np.zeros((len(seeds), R))
    P = np.zeros((len(seeds), R), dtype=bool)
    for t, sd in enumerate(seeds):
        ix = oracle.Index(X, nbrs, 0, L, 16, seed=int(sd))
        if delta_for is None:
            st = ix.edge_stats(q, 0, dv, dv + 0.5, eps=eps, eta_mode=eta_mode)
            H[t] = st["H"]
        else:
            for s in range(R):
                st = ix.edge_stats(q, 0, dv, float(delta_for[s]), eps=eps, eta_mode=eta_mode)
                P[t, s] = st["passed"][s]
    return X, q, dv, H, P


def _finite_m_moments(m, n=400_000):
    g = np.abs(np.random.default_rng(1).standard_normal((n, m))).max(1)
    return g.mean(), g.var()


def test_estimator_moments_monte_carlo():
    d, L, R, S = 128, 8, 8, 800
    X, q, dv, H, _ = _mc_H(d, L, R, np.arange(100, 100 + S))
    mu, s2 = _finite_m_moments(16)
    dp = d // L
    x = q.astype(np.float64) - X[0]
    qn = x / np.linalg.norm(x)
    for s in range(R):
        e = X[s + 1].astype(np.float64) - X[0]
        blocks = e.reshape(L, dp)
        bn = np.linalg.norm(blocks, axis=1)
        qb = qn.reshape(L, dp)
        qnorm = np.linalg.norm(qb, axis=1)
        cos_i = np.sum(qb * blocks, axis=1) / (qnorm * bn)
        u = (blocks / (math.sqrt(L) * bn[:, None])).ravel()
        e_reg = (e @ u) * u
        e_res = e - e_reg
        wr = np.linalg.norm(e_reg) / np.linalg.norm(e)
        wres = np.linalg.norm(e_res) / np.linalg.norm(e)
        cos_res = qn @ e_res / np.linalg.norm(e_res)
        mean = wr * mu * np.sum(qnorm * cos_i) + math.sqrt(L) * wres * mu * cos_res
        var = wr ** 2 * (1 - (1 - s2) * np.sum(qnorm ** 2 * cos_i ** 2)) + L * wres ** 2 * (1 - (1 - s2) * cos_res ** 2)
        h = H[:, s]
        assert abs(h.mean() - mean) < 5 * math.sqrt(var / S)
        assert abs(h.var() - var) < 6 * var * math.sqrt(2.0 / S)


def test_equal_block_norms_mean_lemma52():
    d, L, R, S = 128, 8, 6, 600
    X, q, dv, H, _ = _mc_H(d, L, R, np.arange(5000, 5000 + S), equal_blocks=True)
    mu, _ = _finite_m_moments(16)
    x = q.astype(np.float64) - X[0]
    for s in range(R):
        e = X[s + 1].astype(np.float64) - X[0]
        cos = x @ e / (np.linalg.norm(x) * np.linalg.norm(e))
        sd = H[:, s].std() / math.sqrt(S)
        assert abs(H[:, s].mean() - math.sqrt(L) * mu * cos) < 5 * sd


@pytest.mark.parametrize("eps", [0.1, 0.2])
def test_coverage_finite_m(eps):
    """Neighbours just inside delta (cos theta = A + 0.02) pass with probability >= 1 - eps."""
    d, L, R, S = 128, 8, 6, 500
    X, nbrs, q = _star(d, R, 11, L=L)
    dv = float(oracle.dist2_f32(q, X[0]))
    x = q.astype(np.float64) - X[0]
    deltas = []
    for s in range(R):
        e = X[s + 1].astype(np.float64) - X[0]
        cos = x @ e / (np.linalg.norm(x) * np.linalg.norm(e))
        A = cos - 0.02
        deltas.append(dv + e @ e - 2 * A * math.sqrt(dv) * np.linalg.norm(e))
    _, _, _, _, P = _mc_H(d, L, R, np.arange(900, 900 + S), eps=eps, eta_mode=1, delta_for=deltas)
    rate = P.mean(0)
    sigma = math.sqrt(eps * (1 - eps) / S)
    assert np.all(rate >= 1 - eps - 3 * sigma), rate
