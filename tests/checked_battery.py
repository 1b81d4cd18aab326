"""A fixed battery of searches for the self-checked build of the library: every search
variant (plain, PEOs in frames T and Q, with and without the dimension permutation,
the compact index's 16/8-bit scalars, SimHash, hierarchical entries, uneven batches,
reduced-precision storage with the FP32 re-rank, R = 48, beam widths 2 and 4, the latter
also with a small visited table so that nodes are forgotten within an iteration) over
lists from 1 to 300 entries, on a graph with duplicate vectors and empty slots.  Run as `python -m tests.checked_battery OUT.npz` with PEOS_LIBRARY naming
the library: it saves every result and prints the violation counts as one JSON line
(null for a normal build)."""
import json
import sys

import numpy as np
import torch

import workloads
from workloads.graph import build_graph
from workloads.hier import build_hierarchy


def battery(P) -> dict:
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 4000, 64)
    X, Q = workloads.generate(cfg)
    X[100:110] = X[200]  # duplicated vectors: degenerate edges
    Q[:3] = X[[0, 200, 3999]]  # queries on base points
    nbrs, entry = build_graph(X, 32)
    rng = np.random.default_rng(7)
    drop = rng.random(nbrs.shape) < 0.2
    drop[:, 0] = False
    nbrs = np.where(drop, -1, nbrs).astype(np.int32)  # ragged degrees
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xt, 8, 16, 9)
    perm = P.dim_permutation(G, Xt, 8)
    pcodes = P.build_codes(G, Xt, 8, 16, 9, perm=perm)
    sh = P.build_simhash(G, Xt, 64, 3)
    out = {}
    for ef in (1, 10, 64, 300):
        k = min(10, ef)
        out[f"plain_{ef}"] = P.search(G, None, Xt, Qt, k, ef, routing=0)
        for frame in (0, 1):
            out[f"peos_{ef}_{frame}"] = P.search(G, codes, Xt, Qt, k, ef, routing=1, eps=0.2, frame=frame)
            out[f"perm_{ef}_{frame}"] = P.search(G, pcodes, Xt, Qt, k, ef, routing=1, eps=0.1, frame=frame)
        out[f"simhash_{ef}"] = P.search(G, sh, Xt, Qt, k, ef, routing=2, eps=0.2)
        for beam in (2, 4):
            out[f"beam{beam}_plain_{ef}"] = P.search(G, None, Xt, Qt, k, ef, routing=0, beam=beam)
            out[f"beam{beam}_peos_{ef}"] = P.search(G, codes, Xt, Qt, k, ef, routing=1, eps=0.2, beam=beam,
                                                    visited_slots=256)
    for sb in (16, 8):
        cc = P.build_codes(G, Xt, 8, 16, 9, scalar_bits=sb)
        for ef in (10, 64):
            out[f"compact{sb}_{ef}"] = P.search(G, cc, Xt, Qt, 10, ef, routing=1, eps=0.2)
    layers, top = build_hierarchy(X, 16, seed=4, M=8, min_nodes=16)
    ent = P.hier_entry(P.Hierarchy(layers, top), Xt, Qt)
    out["entries"] = P.search(G, codes, Xt, Qt, 10, 32, routing=1, entries=ent)
    kq = torch.from_numpy(rng.integers(1, 11, len(Q)).astype(np.int32)).cuda()
    efq = torch.from_numpy(rng.integers(10, 129, len(Q)).astype(np.int32)).cuda()
    out["batch"] = P.search_batch(G, codes, Xt, Qt, 10, 128, k_per_query=kq, ef_per_query=efq, routing=1)
    for dt in ("bf16", "e4m3"):
        out[f"rerank_{dt}"] = P.search(G, codes, P.quantize(Xt, dt), Qt, 10, 48, routing=1, rerank=Xt)
    cfg48 = workloads.scaled(workloads.CONFIGS["glove"], 3000, 48)
    X48, Q48 = workloads.generate(cfg48)
    n48, e48 = build_graph(X48, 48)
    G48 = P.Graph.from_numpy(n48, e48)
    X48t, Q48t = torch.from_numpy(X48).cuda(), torch.from_numpy(Q48).cuda()
    c48 = P.build_codes(G48, X48t, 10, 16, 5)
    for routing in (0, 1):
        out[f"r48_{routing}"] = P.search(G48, c48 if routing else None, X48t, Q48t, 10, 64, routing=routing)
        out[f"r48_{routing}_beam4"] = P.search(G48, c48 if routing else None, X48t, Q48t, 10, 64, routing=routing,
                                               beam=4)
    torch.cuda.synchronize()
    res = {}
    for key, v in out.items():
        res[key + "_ids"] = v[0].cpu().numpy()
        res[key + "_dists"] = v[1].cpu().numpy()
    return res


if __name__ == "__main__":
    import paper_2402_11354_gb300 as P
    P.load(build_if_missing=False)
    res = battery(P)
    np.savez(sys.argv[1], **res)
    print(json.dumps({"version": P.version(), "violations": P.check_read()}))
