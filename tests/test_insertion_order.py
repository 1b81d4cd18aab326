"""The insertion rule of Algorithm 1 as the search kernel applies it to an out-degree above
32: the passes of one expansion come in two groups (edges 0..31, then 32..R-1), tested
against the same list bound δ, and the second group is inserted after the first.  The
rule - a candidate enters iff the list holds fewer than efs entries or its (dist, id) is
below the list's last entry, the last entry dropping out when the list is full - keeps
the efs smallest of everything inserted, so inserting the groups one after the other
leaves the same list as inserting all passes in one ascending pass.  Checked here
on random lists, candidate sets and splits, with ties in distance broken by id."""
import numpy as np


def insert(lst, cands, ef):
    """Algorithm 1's rule on a sorted list of (dist, id), candidates taken in ascending order."""
    lst = list(lst)
    for c in sorted(cands):
        if len(lst) < ef:
            lst.append(c)
            lst.sort()
        elif c < lst[-1]:
            lst[-1] = c
            lst.sort()
    return lst


def test_two_groups_equal_one_sorted_insertion():
    rng = np.random.default_rng(7)
    for _ in range(3000):
        ef = int(rng.integers(1, 40))
        ids = rng.permutation(200)
        dist = rng.integers(0, 30, size=200).astype(float)  # many equal distances
        n0 = int(rng.integers(0, ef + 1))
        lst = sorted(zip(dist[:n0], ids[:n0]))
        m = int(rng.integers(0, 64))
        cands = list(zip(dist[n0:n0 + m], ids[n0:n0 + m]))
        split = int(rng.integers(0, m + 1))
        one = insert(lst, cands, ef)
        two = insert(insert(lst, cands[:split], ef), cands[split:], ef)
        assert one == two
        assert one == sorted(lst + cands)[:ef]
