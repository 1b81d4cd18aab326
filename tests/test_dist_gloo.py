"""Multi-rank host logic on CPU (gloo, world size 2): query sharding with results
gathered in order equals the single-process search; base sharding with the top-k
exchange equals the search over the whole base (exact with efs >= shard size).
The per-rank searcher is the oracle (CPU), the plumbing is paper_2402_11354_gb300.dist."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import workloads
from paper_2402_11354_gb300 import dist as pdist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = workloads.scaled(workloads.CONFIGS["sift"], 1200, 30)
        X, Q = workloads.generate(cfg)
        if mode == "queries":
            nbrs, entry = oracle.build_graph(X, 16)
            s, e = pdist.shard_range(len(Q), rank, world)
            r = oracle.search(X, nbrs, entry, Q[s:e], 10, 32, routing=0)
            ids = pdist.gather_rows(torch.from_numpy(r["ids"]), len(Q))
            dd = pdist.gather_rows(torch.from_numpy(r["dists"]), len(Q))
            if rank == 0:
                q.put((ids.numpy(), dd.numpy()))
        else:
            s, e = pdist.shard_range(len(X), rank, world)
            Xs = X[s:e]
            nbrs, entry = oracle.build_graph(Xs, 16)
            r = oracle.search(Xs, nbrs, entry, Q, 10, len(Xs), routing=0)
            ids, dd = pdist.merge_shards(torch.from_numpy(r["ids"]), torch.from_numpy(r["dists"]), s, 10)
            if rank == 0:
                q.put((ids.numpy(), dd.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = q.get(timeout=240)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


def test_shard_range_covers_exactly():
    for n in (0, 1, 7, 10, 1001):
        for w in (1, 2, 3, 8):
            parts = [pdist.shard_range(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            assert max(e - s for s, e in parts) - min(e - s for s, e in parts) <= 1


def test_merge_topk_orders_by_dist_then_id():
    ids = torch.tensor([[5, 3, -1, 9, 2]], dtype=torch.int32)
    d = torch.tensor([[1.0, 1.0, 0.0, 0.5, 2.0]])
    i2, d2 = pdist.merge_topk(ids, d, 3)
    assert i2.tolist() == [[9, 3, 5]] and d2.tolist() == [[0.5, 1.0, 1.0]]


def test_query_sharding_equals_single_process():
    ids, dd = _run("queries")
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 1200, 30)
    X, Q = workloads.generate(cfg)
    nbrs, entry = oracle.build_graph(X, 16)
    r = oracle.search(X, nbrs, entry, Q, 10, 32, routing=0)
    assert np.array_equal(ids, r["ids"]) and np.array_equal(dd, r["dists"])


def test_base_sharding_merge_is_exact():
    ids, dd = _run("base")
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 1200, 30)
    X, Q = workloads.generate(cfg)
    gt, gd = oracle.knn_f64(X, Q, 10)
    assert np.array_equal(ids, gt)
    assert np.allclose(dd, gd, rtol=0, atol=0)
