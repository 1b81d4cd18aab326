"""Pins of the oracle's code builder (Sec. 4.2 steps (1) and (3)) and projection table.

Each edge record is recomputed from the definitions in FP64 with numpy:
  e_reg = projection of e on the unit direction [e_i / (sqrt(L) ||e_i||)]_i,
  e_res = e - e_reg, w_reg = ||e_reg||/||e||, w_res = ||e_res||/||e||,
  e[i] = sgn(e_i . a^i_j) j with j = argmax_j |e_i . a^i_j|, e[0] likewise over b_j with e_res.
Codes must agree wherever the top two |projections| are not a rounding-level tie.
Special cases: L = 1 is RCEOs (Sec. 4.1): w_reg = 1, w_res = 0; equal block norms give
w_res = 0 (Lemma 5.2's equal-norm case); zero blocks and duplicate vectors are degenerate."""
import numpy as np
import pytest

import oracle


def _pairs(E):
    n, d = E.shape
    X = np.zeros((2 * n, d), dtype=np.float32)
    X[1::2] = E
    nbrs = np.full((2 * n, 2), -1, dtype=np.int32)
    nbrs[0::2, 0] = np.arange(1, 2 * n, 2)
    return X, nbrs


def _reference(E, L, A, B):
    """FP64 definitions of step (1) and step (3)."""
    E = E.astype(np.float64)
    n, d = E.shape
    dp = d // L
    blocks = E.reshape(n, L, dp)
    bn = np.linalg.norm(blocks, axis=2)
    with np.errstate(invalid="ignore", divide="ignore"):
        u = np.where(bn[:, :, None] > 0, blocks / (np.sqrt(L) * bn[:, :, None]), 0.0).reshape(n, d)
    e_reg = (np.sum(E * u, axis=1, keepdims=True) / np.maximum(np.sum(u * u, axis=1, keepdims=True), 1e-300)) * u
    e_res = E - e_reg
    en = np.linalg.norm(E, axis=1)
    wreg = np.linalg.norm(e_reg, axis=1) / en
    wres = np.linalg.norm(e_res, axis=1) / en
    P_blk = np.einsum("nlk,ljk->nlj", blocks, A.astype(np.float64))          # [n, L, m]
    P_res = e_res @ B.astype(np.float64).T                                    # [n, m]
    return dict(bn=bn, wreg=wreg, wres=wres, en=en, P_blk=P_blk, P_res=P_res)


def _check_codes(code_col, P, tol=1e-5):
    """code = sgn(P_j*) (j*+1), j* = argmax |P|; returns the number of rounding-level ties skipped."""
    a = np.abs(P)
    order = np.argsort(-a, axis=1, kind="stable")
    top, second = a[np.arange(len(a)), order[:, 0]], a[np.arange(len(a)), order[:, 1]]
    clear = (top - second) > tol * np.maximum(top, 1e-30)
    j = order[:, 0]
    expect = np.where(P[np.arange(len(P)), j] >= 0, j + 1, -(j + 1))
    assert np.array_equal(code_col[clear], expect[clear])
    return int((~clear).sum())


@pytest.mark.parametrize("L,d,m", [(8, 128, 16), (10, 100, 16), (24, 960, 16), (4, 32, 127), (1, 64, 16)])
def test_codes_match_definitions(L, d, m):
    rng = np.random.default_rng(L * 1000 + d)
    E = (rng.standard_normal((600, d)) * rng.gamma(2.0, 1.0, size=(1, d))).astype(np.float32)
    X, nbrs = _pairs(E)
    A, B = oracle.projections(42, d, L, m)
    codes, enorm, wreg, cres = oracle.build_codes(X, nbrs, L, m, A, B, with_cres=True)
    ref = _reference(X[1::2] - X[0::2], L, A, B)
    c = codes[0::2, 0, :]
    assert np.all(cres[0::2, 1] == 0) and np.all(cres[1::2] == 0)    # empty slots
    assert np.allclose(enorm[0::2, 0], ref["en"], rtol=1e-6)
    assert np.allclose(wreg[0::2, 0], ref["wreg"], rtol=2e-6, atol=1e-7)
    # cres = sqrt(L) w_res = sqrt(L) ||e_res|| / ||e||
    assert np.allclose(cres[0::2, 0].astype(np.float64) ** 2, L * ref["wres"] ** 2, atol=2e-5 * L)
    wres = np.sqrt(np.maximum(0.0, 1.0 - wreg[0::2, 0].astype(np.float64) ** 2))
    assert np.allclose(wres ** 2, ref["wres"] ** 2, atol=2e-5)      # e_reg is orthogonal to e_res
    ties = 0
    for i in range(L):
        ties += _check_codes(c[:, i + 1], ref["P_blk"][:, i, :])
    assert ties <= 2
    if L > 1:
        # e_res = e - e_reg cancels in FP32: its relative error grows as w_res shrinks
        assert _check_codes(c[:, 0], ref["P_res"], tol=1e-3) <= 0.02 * len(c)
    # empty slots carry zero codes
    assert np.all(codes[0::2, 1, :] == 0) and np.all(codes[1::2] == 0)


def test_rceos_special_case_L1():
    """L = 1 (RCEOs): e_reg = e, so w_reg = 1, w_res = 0, and e[0] is over a zero vector (+1)."""
    E = np.random.default_rng(3).standard_normal((200, 64)).astype(np.float32)
    X, nbrs = _pairs(E)
    A, B = oracle.projections(1, 64, 1, 16)
    codes, enorm, wreg = oracle.build_codes(X, nbrs, 1, 16, A, B)
    assert np.allclose(wreg[0::2, 0], 1.0, atol=1e-6)
    assert np.all(codes[0::2, 0, 0] == 1)


def test_equal_block_norms_give_zero_residual():
    rng = np.random.default_rng(4)
    L, dp = 8, 16
    blocks = rng.standard_normal((300, L, dp))
    blocks /= np.linalg.norm(blocks, axis=2, keepdims=True)
    E = (3.0 * blocks.reshape(300, L * dp)).astype(np.float32)
    X, nbrs = _pairs(E)
    A, B = oracle.projections(2, L * dp, L, 16)
    _, _, wreg = oracle.build_codes(X, nbrs, L, 16, A, B)
    assert np.allclose(wreg[0::2, 0], 1.0, atol=2e-6)


def test_degenerate_edges():
    L, d = 4, 32
    E = np.random.default_rng(5).standard_normal((4, d)).astype(np.float32)
    E[1, 8:16] = 0.0          # zero block 2
    E[2, :] = 0.0             # duplicate vectors
    X, nbrs = _pairs(E)
    A, B = oracle.projections(3, d, L, 16)
    codes, enorm, wreg = oracle.build_codes(X, nbrs, L, 16, A, B)
    assert codes[2, 0, 2] == 1                           # zero block -> +1
    assert enorm[4, 0] == 0.0 and np.all(codes[4, 0] == 1)
    assert 0.0 < wreg[2, 0] <= 1.0


@pytest.mark.parametrize("L,d", [(8, 128), (24, 960)])
def test_node_projection_table(L, d):
    rng = np.random.default_rng(d)
    Xs = rng.standard_normal((50, d)).astype(np.float32)
    A, B = oracle.projections(11, d, L, 16)
    T = oracle.node_proj(Xs, L, 16, A, B)
    X64 = Xs.astype(np.float64)
    ref0 = X64 @ B.astype(np.float64).T
    refb = np.einsum("nlk,ljk->nlj", X64.reshape(50, L, d // L), A.astype(np.float64))
    scale = np.linalg.norm(X64, axis=1)[:, None] * 4
    assert np.all(np.abs(T[:, 0, :] - ref0) <= 1e-5 * scale)
    assert np.all(np.abs(T[:, 1:, :] - refb) <= 1e-5 * scale[:, :, None])
