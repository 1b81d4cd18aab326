"""Multi-process use of the library: two gloo ranks (spawned processes) on the one GPU a
run has, each with its own CUDA context running its own kernels; only the host-side
exchange (torch.distributed over gloo, on CPU tensors) connects them.  No kernel waits on
another process's kernel.

- Query sharding (replicas): each rank builds the whole index and searches its slice of
  the queries with PEOs routing; the rows gathered in rank order equal the one-process
  search bit for bit (a query's result does not depend on the batch it is in).
- Base sharding: each rank builds a graph and PEOs codes over its id range of the base
  and searches every query with efs >= its shard size (every node of the shard is
  reached); merging the per-shard top-k by (dist, id) gives the exact k nearest
  neighbours of the whole base (FP64 brute force)."""
import datetime
import os
import socket

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

N, NQ, K = 2000, 90, 10     # base shards of N / 2 = 1000 rows: searched with efs = 1000 <= 1024


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, mode, q):
    import torch.distributed as dist

    import paper_2402_11354_gb300 as P
    from paper_2402_11354_gb300 import dist as pdist
    from workloads.graph import build_graph
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        torch.cuda.set_device(0)
        cfg = workloads.scaled(workloads.CONFIGS["sift"], N, NQ)
        X, Q = workloads.generate(cfg)
        if mode == "queries":
            nbrs, entry = build_graph(X, cfg.R)
            G = P.Graph.from_numpy(nbrs, entry)
            Xd = torch.from_numpy(X).cuda()
            codes = P.build_codes(G, Xd, cfg.L, cfg.m, cfg.proj_seed)
            s, e = pdist.shard_range(len(Q), rank, world)
            ids, dd, _ = P.search(G, codes, Xd, torch.from_numpy(Q[s:e]).cuda(), K, 48, eps=0.2, routing=1)
            ids = pdist.gather_rows(ids.cpu(), len(Q))
            dd = pdist.gather_rows(dd.cpu(), len(Q))
        else:
            s, e = pdist.shard_range(len(X), rank, world)
            Xs = np.ascontiguousarray(X[s:e])
            nbrs, entry = build_graph(Xs, cfg.R)
            G = P.Graph.from_numpy(nbrs, entry)
            Xd = torch.from_numpy(Xs).cuda()
            codes = P.build_codes(G, Xd, cfg.L, cfg.m, cfg.proj_seed)
            ids, dd, _ = P.search(G, codes, Xd, torch.from_numpy(Q).cuda(), K, len(Xs), eps=0.2, routing=1)
            ids, dd = pdist.merge_shards(ids.cpu(), dd.cpu(), s, K)
        torch.cuda.synchronize()
        if rank == 0:
            q.put((ids.numpy(), dd.numpy()))
        dist.barrier()
    except Exception as e:      # report it to the parent instead of leaving it waiting
        q.put(("error", f"rank {rank}: {e!r}"))
        raise
    finally:
        dist.destroy_process_group()


def _run(mode):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        out = q.get(timeout=600)
    finally:
        for p in procs:
            p.join(timeout=300)
    assert not (isinstance(out, tuple) and len(out) == 2 and isinstance(out[0], str)), out[1]
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    return out


def test_query_sharding_equals_one_process():
    import paper_2402_11354_gb300 as P
    from workloads.graph import build_graph
    ids, dd = _run("queries")
    cfg = workloads.scaled(workloads.CONFIGS["sift"], N, NQ)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, cfg.R)
    G = P.Graph.from_numpy(nbrs, entry)
    Xd = torch.from_numpy(X).cuda()
    codes = P.build_codes(G, Xd, cfg.L, cfg.m, cfg.proj_seed)
    a_ids, a_d, _ = P.search(G, codes, Xd, torch.from_numpy(Q).cuda(), K, 48, eps=0.2, routing=1)
    assert np.array_equal(ids, a_ids.cpu().numpy())
    assert np.array_equal(dd.view(np.uint32), a_d.cpu().numpy().view(np.uint32))


def test_base_sharding_merge_is_exact():
    ids, dd = _run("base")
    cfg = workloads.scaled(workloads.CONFIGS["sift"], N, NQ)
    X, Q = workloads.generate(cfg)
    gt, gd = oracle.knn_f64(X, Q, K)
    assert np.array_equal(ids, gt)
    assert np.array_equal(dd.astype(np.float64), gd)     # integer-valued rows: exact distances
