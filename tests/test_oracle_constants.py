"""Pins of the constants the routing test uses and of w_reg (Lemma 5.4).

- Phi^{-1}(eps), the quantile in F^{-1} of Eq. (N_ex_min): textbook values and scipy.
- eta: sqrt(2 ln m) (Lemma 4.2) and the finite-m mean of max_j |g_j| (quadrature by
  scipy, and Monte Carlo).
- w_reg: the oracle's code builder on isotropic edges against the Gamma closed form
  of E[w_reg] in the proof of Lemma 5.4, and the paper's printed bound (>= 0.978 at
  d = 128, L = 8; tests/golden/lemma54.txt).
- w_res and J_rel (Sec. 5.2, "Impact of L"): the oracle's E[w_res^2] on isotropic edges
  against its closed form from the Dirichlet law of the block norms (the Beta law in the
  proof of Lemma 5.4), J_rel(8, 128) against J_opt = 1/8, and w_res growing with L
  (tests/golden/jrel.txt).
- Table 6 (Appendix C): the printed 428957 projected vectors for RCEOs and L > 2.67 /
  L > 2.69 for PEOs (opt) / PEOs against 64-bit SimHash at d = 384, theta = pi/2, from
  Lemma C.1's condition m > exp(n / (2 theta (pi - theta))) and its PEOs forms, the PEOs
  one with the oracle's own weights (tests/golden/table6_test_comparison.txt).
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


def ewreg2_closed_form(L, d):
    """E[w_reg^2] for isotropic e: w_reg^2 = (sum_i ||e_i||)^2 / (L ||e||^2) and the block
    shares X_i = ||e_i||^2 / ||e||^2 are Dirichlet(d'/2, ..., d'/2), so
    E[w_reg^2] = 1/L + (L - 1) E[sqrt(X_1 X_2)] with E[sqrt(X_1 X_2)] = G(a + 1/2)^2 / (G(a)^2 d/2),
    a = d'/2."""
    a = d / L / 2.0
    return 1.0 / L + (L - 1) * math.exp(2 * (special.gammaln(a + 0.5) - special.gammaln(a))) / (d / 2.0)


def _oracle_w(L, d, n, seed):
    X, nbrs = _isotropic_edges(d, n, seed)
    A, B = oracle.projections(7, d, L, 16)
    _, _, wreg, cres = oracle.build_codes(X, nbrs, L, 16, A, B, with_cres=True)
    w = wreg[0::2, 0].astype(np.float64)
    wres = cres[0::2, 0].astype(np.float64) / math.sqrt(L)
    return w, wres


def test_jrel_impact_of_L():
    g = _golden("jrel.txt")
    d, L, j_opt = int(g["d"]), int(g["L"]), float(g["J_opt"])
    assert j_opt == 1.0 / L
    n = 6000
    w, wres = _oracle_w(L, d, n, 314)
    ewres2 = 1.0 - ewreg2_closed_form(L, d)
    assert abs((wres ** 2).mean() - ewres2) < 5 * (wres ** 2).std() / math.sqrt(n)
    j_rel = (1 + (L - 1) * (wres ** 2).mean()) / L
    j_cf = (1 + (L - 1) * ewres2) / L
    assert abs(j_rel - j_cf) < 5 * (L - 1) / L * (wres ** 2).std() / math.sqrt(n)
    assert j_opt < j_rel < 1.25 * j_opt                  # close to J_opt at L = 8
    # w_res grows with L (isotropic edges, d = 128)
    means = [(_oracle_w(l, d, 2000, 400 + l)[1] ** 2).mean() for l in (2, 4, 8, 16)]
    assert all(a < b for a, b in zip(means, means[1:])), means


def test_table6_routing_test_comparison():
    g = _golden("table6_test_comparison.txt")
    d, n, m = int(g["d"]), int(g["n"]), int(g["m"])
    theta = math.pi / 2
    c = n / (2 * theta * (math.pi - theta))
    # RCEOs outperforms SimHash iff m > exp(n / (2 theta (pi - theta))) (Lemma C.1)
    assert math.floor(math.exp(c)) + 1 == int(g["rceos_m_greater_than"])
    # PEOs (opt): L ln m > n / (2 theta (pi - theta))
    assert round(c / math.log(m), 2) == float(g["peos_opt_L_greater_than"])
    # PEOs: L ln m > (w_reg^2 + L w_res^2) n / (2 theta (pi - theta)), the squared weights at
    # their expected values under the isotropic distribution, taken at the smallest L
    # (dividing d) above the PEOs (opt) bound, L = 3; the oracle's weights on isotropic edges
    L = 3
    w, wres = _oracle_w(L, d, 3000, 27)
    bound = c * ((w ** 2).mean() + L * (wres ** 2).mean()) / math.log(m)
    assert round(bound, 2) == float(g["peos_L_greater_than"])
