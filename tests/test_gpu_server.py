"""GPU tests of the serving loop (peos_server_*): continuous batching with admission by
device memory.

A request's result depends only on the request, so it must be the same when the
request runs alone and when it runs in a mix of concurrent batches (bit for bit), and
meet the bars of tests/parity.py against the oracle's search with its own k and efs."""
import time

import numpy as np
import pytest
import torch

import oracle
import parity
from conftest import get_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module")
def env(P):
    case = get_case("sift", 20_000, 200)
    X = torch.from_numpy(case.X).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    codes = P.build_codes(G, X, case.cfg.L, case.cfg.m, case.cfg.proj_seed)
    rng = np.random.default_rng(5)
    nq = len(case.Q)
    k = rng.choice([10, 100], size=nq).astype(np.int32)
    ef = np.maximum(rng.choice([64, 256], size=nq), k).astype(np.int32)
    return case, X, G, codes, k, ef


def collect(srv, n, timeout_s=60.0):
    got = {}
    t_end = time.time() + timeout_s
    while len(got) < n and time.time() < t_end:
        r = srv.poll(max_results=1024, wait_us=2000)
        for i, rid in enumerate(r["request_id"]):
            got[int(rid)] = (int(r["status"][i]), r["ids"][i].copy(), r["dists"][i].copy(), int(r["arrival_ns"][i]),
                             int(r["complete_ns"][i]))
    assert len(got) == n, f"only {len(got)} of {n} requests completed"
    return got


def oracle_rows(case, k, ef, k_max, routing=1, base=None, rerank=None):
    ids = np.full((len(k), k_max), -1, np.int32)
    dists = np.full((len(k), k_max), np.inf, np.float32)
    for kk, ee in sorted(set(zip(k.tolist(), ef.tolist()))):
        sel = np.nonzero((k == kk) & (ef == ee))[0]
        r = case.index.search(case.Q[sel], kk, ee, routing=routing, eps=0.2, base=base, rerank=rerank)
        ids[sel, :kk] = r["ids"]
        dists[sel, :kk] = r["dists"]
    return ids, dists


def test_same_result_alone_and_in_mix(P, env):
    case, X, G, codes, k, ef = env
    nq = len(case.Q)
    srv = P.Server(G, codes, X, k_max=100, ef_max=256, max_batch=48, streams=4, memory_budget=64 << 20, routing=1,
                   eps=0.2)
    try:
        alone = {}
        for i in range(0, nq, 9):
            srv.submit(i, case.Q[i], int(k[i]), int(ef[i]))
            alone[i] = collect(srv, 1)[i]
        # the whole set at ~200k requests/s (Poisson), so batches overlap on the GPU
        rng = np.random.default_rng(8)
        arrival = np.cumsum(rng.exponential(1e9 / 200_000, size=nq)).astype(np.int64)
        srv.replay(np.arange(nq) + 10_000, case.Q, k, ef, arrival)
        mix = collect(srv, nq)
        st = srv.stats()
    finally:
        srv.close()
    oi, od = oracle_rows(case, k, ef, 100)
    for i in range(nq):
        status, ids, dists, t_arr, t_done = mix[10_000 + i]
        assert status == 0 and t_done >= t_arr
        if i in alone:
            assert np.array_equal(ids, alone[i][1]) and np.array_equal(dists, alone[i][2])
    gi = np.stack([mix[10_000 + i][1] for i in range(nq)])
    gd = np.stack([mix[10_000 + i][2] for i in range(nq)])
    parity.search_parity(gi, gd, dict(ids=oi, dists=od))
    assert st["completed"] == st["submitted"] == nq + len(alone)
    assert st["failed"] == 0 and st["pending"] == 0
    assert st["batched_queries"] == st["completed"] and st["batches"] < st["completed"]  # requests were batched


def test_admission_by_device_memory(P, env):
    """A budget that holds only a few requests at a time: every request still completes
    (the scheduler waits for memory), and the arena never exceeds the budget."""
    case, X, G, codes, k, ef = env
    nq = len(case.Q)
    per_batch_of_4 = P.batch_workspace_size(G, codes, X, 4, 100, 256) + 4 * (X.shape[1] * 4 + 8 + 800) + 6 * 256
    budget = per_batch_of_4
    srv = P.Server(G, codes, X, k_max=100, ef_max=256, max_batch=64, streams=4, memory_budget=budget, routing=1,
                   eps=0.2)
    try:
        srv.replay(np.arange(nq), case.Q, k, ef, np.zeros(nq, dtype=np.int64))
        got = collect(srv, nq)
        st = srv.stats()
    finally:
        srv.close()
    assert st["arena_peak"] <= st["arena_bytes"] == budget
    assert st["admission_waits"] > 0 and st["batches"] >= nq // 4
    oi, od = oracle_rows(case, k, ef, 100)
    assert all(got[i][0] == 0 for i in range(nq))
    parity.search_parity(np.stack([got[i][1] for i in range(nq)]), np.stack([got[i][2] for i in range(nq)]),
                         dict(ids=oi, dists=od))


def test_server_with_stored_rows_and_rerank(P, env):
    case, X, G, codes, k, ef = env
    nq = len(case.Q)
    st = P.quantize(X, "e4m3")
    srv = P.Server(G, codes, st, k_max=100, ef_max=256, max_batch=32, streams=3, memory_budget=64 << 20, rerank=X,
                   routing=1, eps=0.2)
    try:
        srv.replay(np.arange(nq), case.Q, k, ef, np.arange(nq, dtype=np.int64) * 2000)
        got = collect(srv, nq)
    finally:
        srv.close()
    direct, dd, _ = P.search_batch(G, codes, st, torch.from_numpy(case.Q).cuda(), 100, 256,
                                   torch.from_numpy(k).cuda(), torch.from_numpy(ef).cuda(), routing=1, eps=0.2, rerank=X)
    direct, dd = direct.cpu().numpy(), dd.cpu().numpy()
    for i in range(nq):
        assert np.array_equal(got[i][1], direct[i]) and np.array_equal(got[i][2], dd[i])


def test_server_rejects_bad_requests(P, env):
    case, X, G, codes, k, ef = env
    srv = P.Server(G, codes, X, k_max=10, ef_max=64, max_batch=8, streams=1, memory_budget=16 << 20)
    try:
        with pytest.raises(P.PeosError):
            srv.submit(1, case.Q[0], 11, 64)     # k > k_max
        with pytest.raises(P.PeosError):
            srv.submit(2, case.Q[0], 10, 65)     # ef > ef_max
        with pytest.raises(P.PeosError):
            srv.submit(3, case.Q[0], 10, 9)      # ef < k
        with pytest.raises(P.PeosError):
            srv.replay([1, 2], case.Q[:2], [10, 10], [64, 64], [5, 1])  # arrivals must ascend
    finally:
        srv.close()
    with pytest.raises(P.PeosError):
        P.Server(G, codes, X, k_max=10, ef_max=64, memory_budget=1024)   # below one request
    with pytest.raises(P.PeosError):
        P.Server(G, codes, X, k_max=10, ef_max=64, streams=0)
