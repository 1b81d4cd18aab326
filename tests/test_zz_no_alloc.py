"""The allocation-free entry point (peos_search_noalloc) against peos_search.

For callers that cannot allocate device memory while serving (engines that reserve
all memory up front, latency-critical loops): the search's scratch comes from a
fixed array in the library's device image.  Both calls run through the C ABI on the
same inputs; the results must agree exactly, on two calls in a row (the array keeps
the previous call's contents, which must not leak into the next).  This file is
collected last so that a failure here stops a -x run only after everything else ran;
it also passes on its own in a fresh process."""
import numpy as np
import pytest
import torch

import workloads
from workloads.graph import build_graph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import paper_2402_11354_gb300 as P
    P.load()
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 6000, 333)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, cfg.R)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xt, cfg.L, cfg.m, cfg.proj_seed)
    return P, G, codes, Xt, Qt


@pytest.mark.parametrize("routing,ef", [(1, 32), (0, 32), (1, 96)])
def test_noalloc_matches_search_twice(setup, routing, ef):
    P, G, codes, Xt, Qt = setup
    ref_ids, ref_d, ref_c = P.search(G, codes, Xt, Qt, 10, ef, routing=routing, eps=0.2, counters=True)
    for half in (Qt, Qt[:200]):      # two calls in a row, the second on a different batch
        ids, d, c = P.search_noalloc(G, codes, Xt, half, 10, ef, routing=routing, eps=0.2, counters=True)
        torch.cuda.synchronize()
        n = half.shape[0]
        assert torch.equal(ids, ref_ids[:n])
        assert torch.equal(d, ref_d[:n])
        assert torch.equal(c, ref_c[:n])


def test_noalloc_large_batch(setup):
    """The search needs no per-query scratch (each warp builds its query's table in shared
    memory), so a batch far beyond the fixed array's size runs and matches peos_search."""
    P, G, codes, Xt, Qt = setup
    many = Qt.repeat(60, 1).contiguous()
    a = P.search(G, codes, Xt, many, 10, 32, routing=1)
    b = P.search_noalloc(G, codes, Xt, many, 10, 32, routing=1)
    torch.cuda.synchronize()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
