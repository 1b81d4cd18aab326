"""The benchmark's byte accounting and its committed DRAM-traffic table, on the CPU.

- The algorithmic bytes follow the per-unit figures: per query its row (4d) and k results
  (8k); per expansion the edge record R (4 + (L + 1) + 12) plus the expanded node's row
  under PEOs, or 4R ids under plain routing; per exact distance one row.  Checked on
  hand-made counters against the same sums written out for the sift-shaped shape.
- The kernel-read bytes take the record only on expansions under the test.
- Every line of the traffic table parses (kernel-sources hash, config, operating point,
  bytes), and the lookup finds an entry only under its own key."""
import os

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _counters(exps, dists, full):
    c = np.zeros((len(exps), 16), dtype=np.int32)
    c[:, 0] = exps
    c[:, 7] = dists
    c[:, 10] = full
    return c


def test_algorithmic_bytes_per_unit():
    d, R, L, k = 128, 32, 8, 10
    c = _counters([25, 26], [250, 260], [20, 21])
    nq, exp, nd = 2, 51, 510
    peos = nq * 4 * d + nq * 8 * k + exp * (R * (4 + L + 1 + 12) + 4 * d) + nd * 4 * d
    plain = nq * 4 * d + nq * 8 * k + exp * 4 * R + nd * 4 * d
    assert bench.algorithmic_bytes(c, d, R, L, k, 1) == peos
    assert bench.algorithmic_bytes(c, d, R, L, k, 0) == plain
    # BF16 rows: 2d bytes per row
    assert bench.algorithmic_bytes(c, d, R, L, k, 0, row_bytes=2 * d) == nq * 4 * d + nq * 8 * k + exp * 4 * R + nd * 2 * d
    # the sift-shaped launch of the benchmark: 10,000 queries, 25.5447 expansions and
    # 257.6769 distances per query -> 1.66 GB
    big = np.zeros((10_000, 16))
    big[:, 0], big[:, 7] = 25.5447, 257.6769
    got = bench.algorithmic_bytes(big, d, R, L, k, 1)
    assert abs(got - 1.6604e9) / 1.6604e9 < 2e-3


def test_kernel_read_bytes_record_only_under_the_test():
    d, R, k, stride = 128, 32, 10, 896
    c = _counters([25, 26], [250, 260], [20, 21])
    base = 2 * 4 * d + 2 * 8 * k + 51 * 4 * R + 510 * 4 * d
    assert bench.kernel_read_bytes(c, d, R, k, stride, 0) == base
    assert bench.kernel_read_bytes(c, d, R, k, stride, 1) == base + 41 * (stride - 4 * R)


def test_traffic_table_parses_and_keys():
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    rows = []
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        assert len(f) == 9, line
        h, cfg, routing, ef, eps, eta, gather, beam, b = f
        assert len(h) == 16 and int(h, 16) >= 0
        assert routing in ("0", "1") and eta in ("0", "1") and gather in ("4", "8") and beam in ("1", "2", "4")
        assert int(ef) > 0 and 0 < float(eps) <= 0.5 and int(b) > 0
        rows.append(f)
    assert rows
    # a key that is not in the table finds nothing
    assert bench.measured_traffic("no-such-config", 1, 18, 0.2, 1, 4, 1) is None
