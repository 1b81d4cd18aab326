"""Pins of the compact index's scalar quantisation (oracle.quantize_scalars; the 8/16-bit
edge scalars of the paper's space analysis, Sec. 4.3, and of PEOs (Compact), Sec. 6.4).
The paper fixes no scheme; the reading (per-node linear steps, round half to even) is
pinned by properties any correct implementation of it has: the node's largest magnitude
maps to the end of the code range, every value is within half a step, exact half steps
round to even, zeros and empty slots stay zero; and by the search: a compact index keeps
the recall of the FP32 one within a small margin."""
import numpy as np
import pytest

import oracle
import workloads
from workloads.graph import build_graph


def _random_scalars(rng, n, R):
    nbrs = rng.integers(0, n, (n, R)).astype(np.int32)
    nbrs[rng.random((n, R)) < 0.15] = -1
    arrs = [rng.gamma(2.0, 50.0, (n, R)).astype(np.float32), rng.random((n, R)).astype(np.float32),
            (rng.random((n, R)) * 2.8).astype(np.float32)]
    return nbrs, arrs


@pytest.mark.parametrize("bits", [8, 16])
def test_extremes_and_error_bound(bits):
    rng = np.random.default_rng(11)
    n, R = 300, 32
    nbrs, arrs = _random_scalars(rng, n, R)
    *deq, steps, q = oracle.quantize_scalars(nbrs, bits, *arrs)
    Qb = (1 << (bits - 1)) - 1
    valid = nbrs >= 0
    assert np.all(np.abs(q) <= Qb)
    for k in range(3):
        x = arrs[k].astype(np.float64)
        s = np.where(valid, np.abs(x), 0).max(axis=1)
        st = steps[:, k].astype(np.float64)
        assert np.allclose(st, s / Qb, rtol=2e-7)  # the step is the node's largest magnitude / Qb
        for v in range(n):
            if s[v] > 0:
                at_max = valid[v] & (np.abs(x[v]) == s[v])
                assert np.all(np.abs(q[v, at_max, k]) == Qb)
        err = np.abs(deq[k].astype(np.float64) - x)
        bound = 0.5 * st[:, None] * (1 + 1e-6) + 1e-6 * np.abs(x)
        assert np.all(err[valid] <= bound[valid])
        assert np.all(deq[k][~valid] == 0) and np.all(q[~valid][:, k] == 0)
        # the stored value is the integer times the step, in FP32
        assert np.array_equal(deq[k], (q[:, :, k].astype(np.float32) * steps[:, k:k + 1]).astype(np.float32))


@pytest.mark.parametrize("bits", [8, 16])
def test_half_steps_round_to_even_and_zero_nodes(bits):
    Qb = (1 << (bits - 1)) - 1
    # one node whose largest magnitude is Qb: the step is exactly 1
    x = np.array([[Qb, 2.5, 3.5, -2.5, -3.5, 0.5, 1.5, 0.0]], dtype=np.float32)
    nbrs = np.zeros(x.shape, dtype=np.int32)
    zeros = np.zeros_like(x)
    *deq, steps, q = oracle.quantize_scalars(nbrs, bits, x, zeros, zeros)
    assert steps[0, 0] == 1.0
    assert q[0, :, 0].tolist() == [Qb, 2, 4, -2, -4, 0, 2, 0]
    # a node with only zero scalars (duplicate vectors) has step 0 and codes 0
    assert np.all(steps[0, 1:] == 0) and np.all(q[0, :, 1:] == 0) and np.all(deq[1] == 0)


def test_compact_index_keeps_recall():
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 3000, 60)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 32)
    gt, _ = oracle.knn_f64(X, Q, 10)
    rec = {}
    for bits in (32, 16, 8):
        ix = oracle.Index(X, nbrs, entry, 8, 16, 9, scalar_bits=bits)
        ids = ix.search(Q, 10, 32, routing=1, eps=0.2)["ids"]
        rec[bits] = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids, gt)])
    assert rec[16] >= rec[32] - 0.01 and rec[8] >= rec[32] - 0.03, rec
    with pytest.raises(ValueError):
        oracle.Index(X, nbrs, entry, 8, 16, 9, lazy=True, scalar_bits=8)
