"""Pins of the constants the routing test uses and of w_reg (Lemma 5.4).

- Phi^{-1}(eps), the quantile in F^{-1} of Eq. (N_ex_min): textbook values and scipy.
- eta: sqrt(2 ln m) (Lemma 4.2) and the finite-m mean of max_j |g_j| (quadrature by
  scipy, and Monte Carlo).
- w_reg: the oracle's code builder on isotropic edges against the Gamma closed form
  of E[w_reg] in the proof of Lemma 5.4, and the paper's printed bound (>= 0.978 at
  d = 128, L = 8; tests/golden/lemma54.txt).
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, special, stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_norm_ppf_textbook_values():
    assert oracle.norm_ppf(0.1) == pytest.approx(-1.2815515655446004, abs=1e-12)
    assert oracle.norm_ppf(0.2) == pytest.approx(-0.8416212335729142, abs=1e-12)
    assert oracle.norm_ppf(0.5) == pytest.approx(0.0, abs=1e-15)
    for p in np.linspace(0.001, 0.5, 57):
        assert oracle.norm_ppf(p) == pytest.approx(stats.norm.ppf(p), abs=1e-11)


@pytest.mark.parametrize("m", [2, 16, 128])
def test_eta_modes(m):
    assert oracle.eta(m, 0) == pytest.approx(math.sqrt(2.0 * math.log(m)), rel=1e-15)
    ref, _ = integrate.quad(lambda x: 1.0 - special.erf(x / math.sqrt(2.0)) ** m, 0.0, np.inf, limit=200)
    assert oracle.eta(m, 1) == pytest.approx(ref, rel=1e-9)
    g = np.abs(np.random.default_rng(m).standard_normal((200_000, m))).max(1)
    assert oracle.eta(m, 1) == pytest.approx(g.mean(), abs=5 * g.std() / math.sqrt(g.size))


def wreg_closed_form(L, d):
    """E[w_reg] for isotropic e (proof of Lemma 5.4, Beta/Gamma form)."""
    dp = d // L
    lg = (special.gammaln((dp - 1) / 2) + special.gammaln(d / 2) - special.gammaln(dp / 2)
          - special.gammaln((d - 1) / 2))
    return math.sqrt(L) * math.exp(lg) * (dp - 1) / (d - 1)


def wreg_bound(L, d):
    """Lemma 5.4's lower bound (via Gautschi's inequality)."""
    dp = d // L
    return (dp - 1) * math.sqrt(2 * L * d - 3 * L) / ((d - 1) * math.sqrt(2 * dp + 2 * math.sqrt(3) - 6))


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split("=")
                vals[k.strip()] = v.strip()
    return vals


def test_lemma54_printed_bound():
    g = _golden("lemma54.txt")
    d, L, printed = int(g["d"]), int(g["L"]), float(g["bound_at_least"])
    b = wreg_bound(L, d)
    assert b >= printed
    assert round(b, 3) == printed or b - printed < 1e-3
    assert wreg_closed_form(L, d) >= b


def _isotropic_edges(d, n, seed):
    rng = np.random.default_rng(seed)
    E = rng.standard_normal((n, d)).astype(np.float32)
    # pairs (v_i = 0, u_i = E_i): node 2i has one edge to 2i+1
    X = np.zeros((2 * n, d), dtype=np.float32)
    X[1::2] = E
    nbrs = np.full((2 * n, 1), -1, dtype=np.int32)
    nbrs[0::2, 0] = np.arange(1, 2 * n, 2)
    return X, nbrs


@pytest.mark.parametrize("L,d", [(8, 128), (10, 100), (8, 96), (24, 960)])
def test_oracle_wreg_matches_lemma54_expectation(L, d):
    n = 4000 if d <= 128 else 1500
    X, nbrs = _isotropic_edges(d, n, 99 + L)
    A, B = oracle.projections(5, d, L, 16)
    _, enorm, wreg = oracle.build_codes(X, nbrs, L, 16, A, B)
    w = wreg[0::2, 0].astype(np.float64)
    cf = wreg_closed_form(L, d)
    assert abs(w.mean() - cf) < 5 * w.std() / math.sqrt(n) + 1e-6
    assert w.mean() >= wreg_bound(L, d) - 5 * w.std() / math.sqrt(n)
    assert np.allclose(enorm[0::2, 0], np.linalg.norm(X[1::2].astype(np.float64), axis=1), rtol=1e-5)
