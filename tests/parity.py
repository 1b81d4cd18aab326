"""The bars the CUDA path is held to against the oracle, in one place.

Both sides evaluate the same definitions in FP32, in different operation orders (the
oracle in the plain order of Sec. 4.2, the kernels in whatever order suits the GPU), so
floating-point results are compared within a tolerance and the decisions they feed are
compared outside the band that tolerance leaves:

- the statistics A, H, T of the PEOs test: |a - b| <= 1e-5 * max(|a|, |b|, s), where s is
  the magnitude of the terms combined: (||x||^2 + ||e||^2 + delta^2) / (2 ||x|| ||e||) for
  A in the translated frame, and c = sqrt(2 L ln m) (the scale of the threshold) for H
  and T;
- decisions: equal wherever |H - T| > 1e-5 * max(|H|, |T|, c); inside that band a
  decision may differ (counted and reported, never failed); likewise the A >= 1 and
  A <= 0 rules within the tolerance of A around 1 and 0;
- exact distances: within 1e-5 relative;
- searches: the top-k ids of a query identical on >= 99% of the queries, distances within
  1e-5 relative wherever the ids agree, recall@k within 0.3 points.

Where both sides are exact (integer-valued rows: every distance, norm and inner product
of plain routing is an exactly representable integer), searches with plain routing are
also held bit for bit.
"""
from __future__ import annotations

import numpy as np

RTOL = 1e-5
MIN_SAME = 0.99
RECALL_PTS = 0.003


def close(a, b, scale, rtol: float = RTOL) -> np.ndarray:
    """Elementwise |a - b| <= rtol * max(|a|, |b|, scale)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    bound = rtol * np.maximum(np.maximum(np.abs(a), np.abs(b)), np.asarray(scale, dtype=np.float64))
    return (np.abs(a - b) <= bound) | ((a == b) & np.isfinite(a))


def recall(found, truth) -> float:
    found = np.asarray(found)
    truth = np.asarray(truth)
    k = truth.shape[1]
    hits = sum(len(set(f[:k].tolist()) & set(t.tolist())) for f, t in zip(found, truth))
    return hits / float(truth.shape[0] * k)


def search_parity(gpu_ids, gpu_d, ref: dict, gt=None, exact: bool = False, min_same: float = MIN_SAME,
                  what: str = "") -> float:
    """Compare one batch of search results with the oracle's (`ref` = its dict with ids and
    dists).  Returns the fraction of queries whose top-k ids are identical."""
    gpu_ids = np.asarray(gpu_ids)
    gpu_d = np.asarray(gpu_d, dtype=np.float32)
    ids_o, d_o = ref["ids"], np.asarray(ref["dists"], dtype=np.float32)
    assert gpu_ids.shape == ids_o.shape, (what, gpu_ids.shape, ids_o.shape)
    same = np.all(gpu_ids == ids_o, axis=1)
    frac = float(same.mean()) if len(same) else 1.0
    if exact:
        assert same.all(), f"{what}: {(~same).sum()} of {len(same)} queries differ"
        assert np.array_equal(gpu_d.view(np.uint32), d_o.view(np.uint32)), f"{what}: distances differ"
    else:
        assert frac >= min_same, f"{what}: only {frac:.4f} of queries have identical top-k ids"
        agree = gpu_ids == ids_o
        fin = agree & np.isfinite(d_o)
        assert np.all(close(gpu_d[fin], d_o[fin], 0.0)), f"{what}: distances beyond 1e-5 relative"
        assert np.all(np.isinf(gpu_d[agree & ~np.isfinite(d_o)])), f"{what}: empty slots differ"
    if gt is not None:
        r_g, r_o = recall(gpu_ids, gt), recall(ids_o, gt)
        assert abs(r_g - r_o) <= RECALL_PTS, f"{what}: recall {r_g:.4f} vs oracle {r_o:.4f}"
    return frac


def counters_parity(gpu_c, ref_c, col: int, exact: bool = False, min_same: float = MIN_SAME, what: str = "") -> float:
    """A per-query counter (e.g. expansions): identical on >= min_same of the queries
    (all, when exact)."""
    g = np.asarray(gpu_c)[:, col]
    o = np.asarray(ref_c)[:, col]
    same = g == o
    frac = float(same.mean()) if len(same) else 1.0
    if exact:
        assert same.all(), f"{what}: counter {col} differs on {(~same).sum()} queries"
    else:
        assert frac >= min_same, f"{what}: counter {col} identical on only {frac:.4f} of queries"
    return frac


def a_scale(dv, en, delta2):
    """Magnitude of the terms of A in the translated frame: (||x||^2 + ||e||^2 + delta^2) / (2 ||x|| ||e||)."""
    dv = np.float64(dv)
    en = np.asarray(en, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(en > 0, (dv + en * en + np.float64(delta2)) / (2.0 * np.sqrt(dv) * en), 0.0)


def stats_parity(g: dict, o: dict, valid, c_eta: float, s_A, what: str = ""):
    """Element-wise comparison of the test statistics of one node's edges (dicts with A, H,
    T, passed, kind).  Returns (edges checked, decisions that differ inside the band)."""
    valid = np.asarray(valid, dtype=bool)
    s_A = np.broadcast_to(np.asarray(s_A, dtype=np.float64), valid.shape)
    A_g, A_o = g["A"][valid], o["A"][valid]
    assert np.all(close(A_g, A_o, s_A[valid])), f"{what}: A beyond tolerance"
    kg, ko = g["kind"][valid], o["kind"][valid]
    pg, po = g["passed"][valid].astype(bool), o["passed"][valid].astype(bool)
    tolA = RTOL * np.maximum(np.maximum(np.abs(A_g), np.abs(A_o)), s_A[valid])
    near_rule = (np.abs(A_o - 1.0) <= tolA) | (np.abs(A_o) <= tolA)
    # the outcome kinds (A rule or H test) agree except where A sits within tolerance of 0 or 1
    assert np.all((kg == ko) | near_rule), f"{what}: outcome kinds differ away from the A rules' band"
    both = (kg == 2) & (ko == 2)
    H_g, H_o, T_g, T_o = g["H"][valid][both], o["H"][valid][both], g["T"][valid][both], o["T"][valid][both]
    assert np.all(close(H_g, H_o, c_eta)), f"{what}: H beyond tolerance"
    assert np.all(close(T_g, T_o, c_eta)), f"{what}: T beyond tolerance"
    band = np.abs(H_o - T_o) <= RTOL * np.maximum(np.maximum(np.abs(H_o), np.abs(T_o)), c_eta)
    differ = pg[both] != po[both]
    assert not np.any(differ & ~band), f"{what}: decisions differ outside the tolerance band"
    other = ~both
    assert np.all((pg[other] == po[other]) | near_rule[other]), f"{what}: A-rule decisions differ"
    return int(valid.sum()), int(np.sum(differ) + np.sum((pg[other] != po[other])))


def node_terms(tv, codes, wreg, cres):
    """The node term of every edge, sv = S(t(v)) = w_reg sum_{i=1..L} sgn(e[i]) t(v)[i][|e[i]|-1]
    + sqrt(L) w_res sgn(e[0]) t(v)[0][|e[0]|-1], in FP64 from a node table t(v) [n, L+1, m],
    the codes [n, R, L+1] and the weights [n, R] (cres = sqrt(L) w_res).  Returns (sv, scale)
    where scale is the sum of the magnitudes of its terms.  Empty slots (codes 0) give 0."""
    tv = np.asarray(tv, dtype=np.float64)
    codes = np.asarray(codes).astype(np.int64)
    n, R, L1 = codes.shape
    j = np.abs(codes) - 1
    valid = codes[:, :, 0] != 0
    jj = np.where(j < 0, 0, j)
    sel = np.take_along_axis(tv[:, None, :, :].repeat(R, 1), jj[:, :, :, None], axis=3)[..., 0]  # [n, R, L+1]
    sgn = np.where(codes > 0, 1.0, -1.0)
    h1 = (sgn[:, :, 1:] * sel[:, :, 1:]).sum(2)
    h2 = sgn[:, :, 0] * sel[:, :, 0]
    w = np.asarray(wreg, dtype=np.float64)
    c = np.asarray(cres, dtype=np.float64)
    sv = np.where(valid, w * h1 + c * h2, 0.0)
    scale = np.where(valid, np.abs(w) * np.abs(sel[:, :, 1:]).sum(2) + np.abs(c) * np.abs(sel[:, :, 0]), 0.0)
    return sv, scale
