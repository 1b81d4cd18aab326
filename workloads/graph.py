"""Proximity-graph construction for the synthetic workloads.

The search method takes a graph index G = (V, E) as input (Algorithm 1 of the
paper runs over any proximity graph: kNN graph, HNSW, NSG, NSSG).  The
workloads here use an exact-kNN graph with relative-neighbourhood pruning:

1. candidates: the Kc = 2R exact nearest other points of every x, ordered by
   (distance, id) (for bases of 4M points and more, from the library's tensor-core
   brute force: BF16 scores, exact FP32 distances of each row's best Kc + 16);
2. prune: walk the candidates in that order and keep c unless a kept s has
   d(s, c) < d(x, c); stop at R kept;
3. reverse edges: every kept edge x -> y also offers y -> x; y's list becomes
   the union of its own and offered edges, ordered by (distance, id) and cut to
   its `ucap` nearest, re-pruned with rule 2 if longer than R;
4. entry: the point nearest the centroid;
5. repair: while a point is unreachable from the entry, the smallest-id
   unreachable z gets an in-edge from its nearest reachable point with a free
   slot (or, if none has one, from its nearest reachable point, whose furthest
   edge z replaces).

Lists are ordered by (distance from owner, id) and padded with -1.  The graph is
an input to both the CUDA path and the oracle; this module holds none of the
PEOs arithmetic.  Distances are FP64 on the CPU and FP32 on a GPU (exact for the
integer-valued SIFT-shaped data; within FP32 rounding otherwise).
"""
from __future__ import annotations

import numpy as np
import torch


def _dtype(device: torch.device) -> torch.dtype:
    return torch.float64 if device.type == "cpu" else torch.float32


def _pairwise_sq(a: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """Squared distances by direct differences: a [..., p, d], b [..., r, d] -> [..., p, r]."""
    diff = a.unsqueeze(-2) - b.unsqueeze(-3)
    return (diff * diff).sum(-1)


def _lexsort_rows(dist: torch.Tensor, ids: torch.Tensor):
    """Sort each row by (dist, id) ascending; invalid entries carry dist=+inf, id=big."""
    o1 = torch.argsort(ids, dim=1, stable=True)
    d1 = torch.gather(dist, 1, o1)
    i1 = torch.gather(ids, 1, o1)
    o2 = torch.argsort(d1, dim=1, stable=True)
    return torch.gather(d1, 1, o2), torch.gather(i1, 1, o2)


# Bases at least this large take their candidates from the library's tensor-core brute
# force (the GEMM-and-top-k below would take tens of minutes at 10M points).
TENSOR_KNN_MIN_N = 4_000_000


def _knn_candidates_tensor(X: torch.Tensor, Kc: int):
    """Kc nearest other points of every row from the tensor-core brute force (BF16 scores,
    exact FP32 distances of the candidates, ranked by (distance, id)); each row's own
    entry is dropped."""
    import paper_2402_11354_gb300 as P
    n = X.shape[0]
    Xf = X.float().contiguous()
    ids, dists = P.knn_tensor(Xf, Xf, Kc + 1)
    ids = ids.long()
    own = ids == torch.arange(n, device=X.device).unsqueeze(1)
    # keep the first Kc entries that are not the row itself
    keep = ~own
    keep &= torch.cumsum(keep.long(), 1) <= Kc
    out_i = ids[keep].view(n, Kc)
    out_d = dists[keep].view(n, Kc).to(X.dtype)
    return out_d, out_i


def knn_candidates(X: torch.Tensor, Kc: int, block: int, slack: int = 32):
    """Exact Kc nearest other points of every row (distances by direct differences)."""
    n, d = X.shape
    if X.is_cuda and n >= TENSOR_KNN_MIN_N and Kc + 1 <= 96:
        return _knn_candidates_tensor(X, Kc)
    kk = min(Kc + slack, n - 1)
    sq = (X * X).sum(1)
    out_d = torch.empty((n, Kc), dtype=X.dtype, device=X.device)
    out_i = torch.empty((n, Kc), dtype=torch.int64, device=X.device)
    for s in range(0, n, block):
        e = min(n, s + block)
        G = sq[s:e, None] + sq[None, :] - 2.0 * (X[s:e] @ X.T)
        G[torch.arange(e - s, device=X.device), torch.arange(s, e, device=X.device)] = float("inf")
        _, idx = torch.topk(G, kk, dim=1, largest=False, sorted=False)
        del G
        exact = ((X[s:e].unsqueeze(1) - X[idx]) ** 2).sum(-1)
        dd, ii = _lexsort_rows(exact, idx)
        out_d[s:e] = dd[:, :Kc]
        out_i[s:e] = ii[:, :Kc]
    return out_d, out_i


def rng_prune(X: torch.Tensor, cand_d: torch.Tensor, cand_i: torch.Tensor, R: int, block: int):
    """Relative-neighbourhood pruning of sorted candidate rows (rule 2), vectorised over rows.
    Invalid candidates are id < 0.  Returns kept ids [rows, R] (-1 padded) and counts."""
    rows, K = cand_i.shape
    kept = torch.full((rows, R), -1, dtype=torch.int64, device=X.device)
    nk = torch.zeros(rows, dtype=torch.int64, device=X.device)
    for s in range(0, rows, block):
        e = min(rows, s + block)
        ci = cand_i[s:e]
        cd = cand_d[s:e]
        valid = ci >= 0
        V = X[ci.clamp(min=0)]                      # [b, K, d]
        sq = (V * V).sum(-1)
        PD = (sq.unsqueeze(2) + sq.unsqueeze(1) - 2.0 * torch.bmm(V, V.transpose(1, 2))).clamp_min(0.0)  # [b, K, K]
        acc = torch.zeros((e - s, K), dtype=torch.bool, device=X.device)
        cnt = torch.zeros(e - s, dtype=torch.int64, device=X.device)
        for c in range(K):
            blocked = (acc[:, :c] & (PD[:, :c, c] < cd[:, c:c + 1])).any(1) if c > 0 else \
                torch.zeros(e - s, dtype=torch.bool, device=X.device)
            ok = valid[:, c] & ~blocked & (cnt < R)
            acc[:, c] = ok
            cnt += ok.long()
        # gather the kept ids in candidate order
        pos = torch.cumsum(acc.long(), 1) - 1
        rr, cc = torch.nonzero(acc, as_tuple=True)
        kept[s + rr, pos[rr, cc]] = ci[rr, cc]
        nk[s:e] = cnt
    return kept, nk


def _bfs_from(nbrs: np.ndarray, starts: np.ndarray, seen: np.ndarray) -> int:
    """Mark every node reachable from `starts` (not yet seen); returns how many were newly marked."""
    frontier = starts[~seen[starts]]
    seen[frontier] = True
    total = len(frontier)
    while len(frontier):
        nb = nbrs[frontier].ravel()
        nb = nb[nb >= 0]
        nb = np.unique(nb[~seen[nb]])
        seen[nb] = True
        total += len(nb)
        frontier = nb
    return total


def build_graph(X: np.ndarray, R: int, Kc: int | None = None, device: str | torch.device = "cpu",
                ucap: int | None = None, block: int | None = None, verbose: bool = False):
    """Build the graph described in the module docstring.  Returns (nbrs [n, R] int32, entry)."""
    device = torch.device(device)
    dt = _dtype(device)
    n, d = X.shape
    Kc = 2 * R if Kc is None else Kc
    Kc = min(Kc, n - 1)
    ucap = 4 * R if ucap is None else ucap
    Xt = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float32)).to(device=device, dtype=dt)
    big = device.type != "cpu"
    kblock = block or (2048 if big else 1024)
    cand_d, cand_i = knn_candidates(Xt, Kc, kblock)
    pblock = 4096 if big else 512
    fwd, fdeg = rng_prune(Xt, cand_d, cand_i, R, pblock)
    del cand_d, cand_i
    # reverse edges: union of own and offered edges
    src = torch.arange(n, device=device).unsqueeze(1).expand(n, R)
    m = fwd >= 0
    e_src = fwd[m]          # offered edge e_src -> src
    e_dst = src[m]
    all_owner = torch.cat([src[m], e_src])
    all_tgt = torch.cat([fwd[m], e_dst])
    key = all_owner * n + all_tgt
    key = torch.unique(key)
    owner = key // n
    tgt = key % n
    dist = ((Xt[owner] - Xt[tgt]) ** 2).sum(1)
    # sort by (owner, dist, tgt)
    o = torch.argsort(tgt, stable=True)
    owner, tgt, dist = owner[o], tgt[o], dist[o]
    o = torch.argsort(dist, stable=True)
    owner, tgt, dist = owner[o], tgt[o], dist[o]
    o = torch.argsort(owner, stable=True)
    owner, tgt, dist = owner[o], tgt[o], dist[o]
    counts = torch.bincount(owner, minlength=n)
    starts = torch.cumsum(counts, 0) - counts
    rank = torch.arange(len(owner), device=device) - starts[owner]
    keep = rank < ucap
    owner, tgt, dist, rank = owner[keep], tgt[keep], dist[keep], rank[keep]
    usize = counts.clamp(max=ucap)
    U_i = torch.full((n, ucap), -1, dtype=torch.int64, device=device)
    U_d = torch.full((n, ucap), float("inf"), dtype=dt, device=device)
    U_i[owner, rank] = tgt
    U_d[owner, rank] = dist
    nbrs = torch.full((n, R), -1, dtype=torch.int64, device=device)
    small = usize <= R
    nbrs[small] = U_i[small, :R]
    over = torch.nonzero(~small, as_tuple=True)[0]
    if len(over):
        kept, _ = rng_prune(Xt, U_d[over], U_i[over], R, max(1, pblock // 4))
        nbrs[over] = kept
    deg = (nbrs >= 0).sum(1)
    del U_i, U_d
    # entry: nearest to centroid (FP64 centroid)
    cen = torch.from_numpy(np.asarray(X, dtype=np.float64).mean(0)).to(device=device, dtype=dt)
    dc = ((Xt - cen) ** 2).sum(1)
    entry = int(torch.nonzero(dc == dc.min())[0, 0])
    nb = nbrs.cpu().numpy().astype(np.int32)
    deg = deg.cpu().numpy()
    seen = np.zeros(n, dtype=bool)
    _bfs_from(nb, np.array([entry]), seen)
    repairs = 0
    while not seen.all():
        z = int(np.argmin(seen))  # smallest unreached id
        dz = ((Xt - Xt[z]) ** 2).sum(1)
        reach = torch.from_numpy(seen).to(device)
        free = torch.from_numpy(deg < R).to(device)
        cand = reach & free
        if not bool(cand.any()):
            cand = reach
        dzm = torch.where(cand, dz, torch.full_like(dz, float("inf")))
        w = int(torch.nonzero(dzm == dzm.min())[0, 0])
        dwz = float(dz[w])
        lst = [int(t) for t in nb[w] if t >= 0]
        full = len(lst) >= R
        if full:
            lst = lst[:R - 1]
        dl = ((Xt[torch.tensor(lst, device=device, dtype=torch.long)] - Xt[w]) ** 2).sum(1).tolist() if lst else []
        pos = len(lst)
        while pos > 0 and (dwz < dl[pos - 1] or (dwz == dl[pos - 1] and z < lst[pos - 1])):
            pos -= 1
        lst.insert(pos, z)
        nb[w, :] = -1
        nb[w, :len(lst)] = lst
        deg[w] = len(lst)
        repairs += 1
        if full:
            seen[:] = False
            _bfs_from(nb, np.array([entry]), seen)
        else:
            _bfs_from(nb, np.array([z]), seen)
    if verbose:
        print(f"graph: n={n} R={R} mean_deg={deg.mean():.2f} repairs={repairs} entry={entry}")
    return nb, entry
