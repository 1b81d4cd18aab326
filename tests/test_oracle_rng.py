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
