"""Pins of the oracle's reduced-precision storage and its exact re-rank (the precision
form of the search: BF16 or FP8-E4M3 rows with a per-row scale, FP32 accumulation, the
final list re-ranked in FP32).

- BF16 and E4M3 rounding equal torch's own conversions (independent code) on random
  rows and on constructed halfway cases; format facts of E4M3 (largest 448, smallest
  subnormal 2^-9, 127 increasing non-negative values) and round trips of representable
  values; rounding error within half a unit in the last place.
- Re-rank: with efs = N every node ends in R, so the re-ranked top k of a search on E4M3
  rows equals the FP64 brute-force K-NN of the FP32 rows, and without the re-rank it
  equals the brute force of the dequantised rows; re-ranking with the base the search
  read changes nothing.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads


def _rows(seed=0, n=64, d=96):
    rng = np.random.default_rng(seed)
    mag = np.array([1e-6, 1e-3, 1.0, 37.0, 1e4, 3e5])[rng.integers(0, 6, size=(n, 1))]
    X = (rng.standard_normal((n, d)) * mag * np.exp(rng.standard_normal((n, d)))).astype(np.float32)
    X[3] = 0.0
    X[4, :] = 0.0
    X[4, 7] = -2.5e-3
    return X


def test_bf16_equals_torch_rounding():
    X = _rows()
    # halfway cases between two bfloat16 neighbours: ties go to the even one
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), 2 ** -130 * 1.5, 65504.0 + 128.0, 3.0e38],
                    dtype=np.float32)
    X[5, :ties.size] = ties
    codes, scales, deq = oracle.quantize(X, "bf16")
    ref = torch.from_numpy(X).to(torch.bfloat16)
    assert np.array_equal(codes, ref.view(torch.int16).numpy().view(np.uint16))
    assert np.array_equal(deq, ref.to(torch.float32).numpy())
    assert np.all(scales == 1.0)
    assert deq[5, 0] == 1.0 and deq[5, 1] == np.float32(1 + 4 * 2 ** -8)


def test_e4m3_equals_torch_rounding():
    X = _rows(1)
    # a row whose largest magnitude is 448 (scale 1) holding values halfway between two
    # E4M3 neighbours, where ties go to the even code: 1.0625 -> 1, 1.1875 -> 1.25,
    # -1.0625 -> -1, 17 -> 16, 19 -> 20, 1.5 * 2^-9 -> 2^-8, 2.5 * 2^-9 -> 2^-8, 432 -> 448
    X[5, :] = 0.0
    X[5, :9] = [448.0, 1.0625, 1.1875, -1.0625, 17.0, 19.0, 1.5 * 2 ** -9, 2.5 * 2 ** -9, 432.0]
    codes, scales, deq = oracle.quantize(X, "e4m3")
    amax = np.abs(X).max(1)
    inv = np.ones_like(amax)
    inv[amax > 0] = np.float32(448.0) / amax[amax > 0]
    Y = (X * inv[:, None]).astype(np.float32)
    Y = np.clip(Y, -448.0, 448.0)  # torch maps values beyond the range to NaN; the format saturates
    ref = torch.from_numpy(Y).to(torch.float8_e4m3fn)
    ours = codes.copy()
    # +0 and -0 both stand for zero
    ours[ours == 0x80] = 0
    theirs = ref.view(torch.uint8).numpy().copy()
    theirs[theirs == 0x80] = 0
    assert np.array_equal(ours, theirs)
    assert np.array_equal(scales, np.where(amax > 0, amax / np.float32(448.0), 1.0).astype(np.float32))
    assert np.array_equal(deq, (scales[:, None] * ref.to(torch.float32).numpy()).astype(np.float32))
    assert deq[5, :9].tolist() == [448.0, 1.0, 1.25, -1.0, 16.0, 20.0, 2.0 ** -8, 2.0 ** -8, 448.0]


def test_e4m3_format_facts_and_round_trip():
    # all 127 non-negative finite codes, in code order, through a row whose max is 448 (scale 1)
    vals = np.array([oracle.quantize(np.array([[448.0, 0, 0, 0]], np.float32), "e4m3")[2][0, 0]], np.float32)
    assert vals[0] == 448.0
    grid = []
    for ex in range(16):
        for man in range(8):
            if ex == 15 and man == 7:
                continue  # NaN
            grid.append((man / 8) * 2.0 ** -6 if ex == 0 else (1 + man / 8) * 2.0 ** (ex - 7))
    grid = np.array(grid, np.float32)
    assert grid.size == 127 and np.all(np.diff(grid) > 0) and grid[-1] == 448.0 and grid[1] == 2.0 ** -9
    d = 128
    row = np.zeros((1, d), np.float32)
    row[0, :d - 1] = grid[:d - 1] * np.where(np.arange(d - 1) % 2, -1, 1)
    row[0, -1] = 448.0
    codes, scales, deq = oracle.quantize(row, "e4m3")
    assert scales[0] == 1.0
    assert np.array_equal(deq, row)
    # code of +v is its index in the grid; the sign is bit 7
    assert codes[0, 0] == 0 and codes[0, 2] == 2 and codes[0, 1] == 0x80 | 1


def test_rounding_error_bounds():
    X = _rows(2, n=200, d=64)
    _, _, deq = oracle.quantize(X, "bf16")
    nz = X != 0
    assert np.all(np.abs(deq[nz] - X[nz]) <= np.abs(X[nz]) * 2.0 ** -8 * (1 + 1e-6))
    _, scales, deq = oracle.quantize(X, "e4m3")
    # half a unit: 2^-4 relative in the normal range, 2^-10 * scale in the subnormal range
    bound = np.maximum(np.abs(X) * 2.0 ** -4, scales[:, None] * 2.0 ** -10) * (1 + 1e-5)
    assert np.all(np.abs(deq - X) <= bound)


@pytest.fixture(scope="module")
def tiny_glove():
    cfg = workloads.scaled(workloads.CONFIGS["glove"], 600, 20)
    X, Q = workloads.generate(cfg)
    nbrs, entry = oracle.build_graph(X, 16)
    ix = oracle.Index(X, nbrs, entry, cfg.L, cfg.m, cfg.proj_seed)
    return cfg, X, Q, nbrs, entry, ix


@pytest.mark.parametrize("routing", [0, 1])
def test_rerank_with_full_list_is_exact_knn(tiny_glove, routing):
    cfg, X, Q, nbrs, entry, ix = tiny_glove
    _, _, deq = oracle.quantize(X, "e4m3")
    gt, gd = oracle.knn_f64(X, Q, 10)
    gq, _ = oracle.knn_f64(deq, Q, 10)
    kw = dict(routing=routing, eps=0.2)
    r = ix.search(Q, 10, X.shape[0], base=deq, rerank=X, **kw)
    assert np.array_equal(r["ids"], gt)
    assert np.allclose(r["dists"], gd, rtol=1e-5, atol=0)
    plain = ix.search(Q, 10, X.shape[0], base=deq, **kw)
    assert np.array_equal(plain["ids"], gq)
    assert not np.array_equal(gq, gt)  # the storage error is visible without the re-rank


def test_rerank_with_search_base_changes_nothing(tiny_glove):
    cfg, X, Q, nbrs, entry, ix = tiny_glove
    a = ix.search(Q, 10, 40, routing=1, eps=0.2)
    b = ix.search(Q, 10, 40, routing=1, eps=0.2, rerank=X)
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["dists"], b["dists"])


def test_lazy_index_reads_fp32_rows_when_searching_stored_rows(tiny_glove):
    """The lazily built codes come from the index's FP32 rows, not from the rows the search
    reads: lazy and eager indexes agree on a search over dequantised rows."""
    cfg, X, Q, nbrs, entry, ix = tiny_glove
    _, _, deq = oracle.quantize(X, "e4m3")
    lazy = oracle.Index(X, nbrs, entry, cfg.L, cfg.m, cfg.proj_seed, lazy=True)
    a = ix.search(Q, 10, 32, routing=1, eps=0.2, base=deq)
    b = lazy.search(Q, 10, 32, routing=1, eps=0.2, base=deq)
    assert np.array_equal(a["ids"], b["ids"]) and np.array_equal(a["dists"], b["dists"])
    touched = lazy.ready.astype(bool)
    assert np.array_equal(lazy.codes[touched], ix.codes[touched])
