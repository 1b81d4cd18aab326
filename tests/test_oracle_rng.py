"""Pins of the oracle's random projection vectors (Sec. 4.2 step (2)).

The generator is Philox4x64-10 restated from Salmon et al. (SC'11); numpy ships an
independent implementation of the same generator, so the block function is pinned
word for word against it.  The Gaussian vectors are then pinned by their
distribution (Kolmogorov-Smirnov against N(0,1), moments, independence)."""
import numpy as np
import pytest
from scipy import stats

import oracle


@pytest.mark.parametrize("key,ctr", [
    ([0, 0], [0, 0, 0, 0]),
    ([5, 7], [1, 2, 3, 4]),
    ([0xFFFFFFFFFFFFFFFF, 0x0123456789ABCDEF], [0xFFFFFFFFFFFFFFFE, 9, 0xDEADBEEF, 1 << 63]),
    ([3000, 0x50454F5350524F4A], [17, 3, 1, 0]),
])
def test_philox_block_matches_numpy(key, ctr):
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(ctr, dtype=np.uint64))
    raw = bg.random_raw(4)
    # numpy advances the 256-bit counter by one before producing a block
    c = list(ctr)
    c[0] = (c[0] + 1) & 0xFFFFFFFFFFFFFFFF
    if c[0] == 0:
        c[1] = (c[1] + 1) & 0xFFFFFFFFFFFFFFFF
    ours = oracle.philox4x64_10(np.array(c, dtype=np.uint64), np.array(key, dtype=np.uint64))
    assert np.array_equal(ours, raw)


def test_projections_are_standard_normal():
    A, B = oracle.projections(777, 960, 24, 64)
    for z in (A.ravel(), B.ravel()):
        assert abs(z.mean()) < 4.0 / np.sqrt(z.size)
        assert abs(z.var() - 1.0) < 4.0 * np.sqrt(2.0 / z.size)
        assert stats.kstest(z.astype(np.float64), "norm").pvalue > 1e-3
    # A and B are independent draws
    n = min(A.size, B.size)
    r = np.corrcoef(A.ravel()[:n], B.ravel()[:n])[0, 1]
    assert abs(r) < 4.0 / np.sqrt(n)


def test_projections_deterministic_and_seeded():
    A1, B1 = oracle.projections(3000, 128, 8, 16)
    A2, B2 = oracle.projections(3000, 128, 8, 16)
    A3, B3 = oracle.projections(3001, 128, 8, 16)
    assert np.array_equal(A1, A2) and np.array_equal(B1, B2)
    assert not np.any(A1 == A3) or np.mean(A1 == A3) < 1e-3
    assert A1.shape == (8, 16, 16) and B1.shape == (16, 128)
    # consecutive columns are not correlated (pairs come from one Box-Muller draw)
    x = B1.reshape(-1, 2)
    assert abs(np.corrcoef(x[:, 0], x[:, 1])[0, 1]) < 4.0 / np.sqrt(x.shape[0])


def _numpy_block(ctr, key):
    """Philox4x64-10 block of counter `ctr` from numpy's generator (which advances its
    256-bit counter by one before producing a block, so it is started one below)."""
    c = sum(int(w) << (64 * i) for i, w in enumerate(ctr))
    c = (c - 1) % (1 << 256)
    start = np.array([(c >> (64 * i)) & 0xFFFFFFFFFFFFFFFF for i in range(4)], dtype=np.uint64)
    return np.random.Philox(key=np.array(key, dtype=np.uint64), counter=start).random_raw(4)


def _normals(seed, mat, row, g):
    """The four normals of block (g, row, mat, 0) under key (seed, tag): two Box-Muller
    pairs in FP64 from 53-bit uniforms, u1 in (0, 1] and u2 in [0, 1)."""
    import math
    w = [int(x) for x in _numpy_block([g, row, mat, 0], [seed, 0x50454F5350524F4A])]
    z = []
    for h in range(2):
        u1 = ((w[2 * h] >> 11) + 1) * 2.0 ** -53
        u2 = (w[2 * h + 1] >> 11) * 2.0 ** -53
        r = math.sqrt(-2.0 * math.log(u1))
        th = 2.0 * math.pi * u2
        z += [r * math.cos(th), r * math.sin(th)]
    return np.array(z, dtype=np.float64).astype(np.float32)


@pytest.mark.parametrize("seed,d,L,m", [(3000, 128, 8, 16), (3004, 960, 24, 16)])
def test_projection_layout_follows_the_counter_reading(seed, d, L, m):
    """Where each normal goes: a^i_j[k] is normal k % 4 of the block with counter
    (k / 4, row i m + j, matrix 0, 0), b_j[k] normal k % 4 of (k / 4, j, 1, 0), the key
    (seed, tag); recomputed at sampled positions from numpy's own Philox4x64-10 and the
    Box-Muller pairs, so that a transposed row, matrix or column index fails."""
    A, B = oracle.projections(seed, d, L, m)
    dp = d // L
    rng = np.random.default_rng(seed)
    for i, j, k in zip(rng.integers(0, L, 40), rng.integers(0, m, 40), rng.integers(0, dp, 40)):
        want = _normals(seed, 0, int(i) * m + int(j), int(k) // 4)[int(k) % 4]
        assert A[i, j, k].view(np.uint32) == want.view(np.uint32), (i, j, k)
    for j, k in zip(rng.integers(0, m, 40), rng.integers(0, d, 40)):
        want = _normals(seed, 1, int(j), int(k) // 4)[int(k) % 4]
        assert B[j, k].view(np.uint32) == want.view(np.uint32), (j, k)
