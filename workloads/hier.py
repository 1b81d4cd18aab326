"""Upper layers of an HNSW-style hierarchy over a workload's base graph (the paper's
indexes are HNSW graphs with M = 32, Sec. 6.1 and its experimental setup).

Each node draws a level l = floor(-ln U / ln M), U uniform in (0, 1], from a seeded
generator (HNSW's level rule with m_L = 1 / ln M), so layer l >= 1 holds about n / M^l
nodes.  Every upper layer is a graph of its own nodes built by the same builder as the
base graph (exact kNN candidates, relative-neighbourhood pruning, reverse edges,
connectivity repair); layers with fewer than `min_nodes` nodes are dropped, and the
descent starts at the top layer's entry (its node nearest the centroid).

The result is ordered top layer first, each layer a dict with
  ids  [n_l]        base row of each local node (ascending),
  nbrs [n_l, R_l]   local ids, -1 = empty slot,
  down [n_l]        local id of the node in the next lower upper layer (not on the lowest),
plus the top layer's entry as a local id."""
from __future__ import annotations

import numpy as np

from .graph import build_graph


def build_hierarchy(X: np.ndarray, R: int, seed: int, M: int = 32, min_nodes: int = 64,
                    device: str = "cpu") -> tuple[list[dict], int]:
    n = X.shape[0]
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random(n)  # (0, 1]
    level = np.floor(-np.log(u) / np.log(M)).astype(np.int64)
    layers = []
    lvl = 1
    while True:
        ids = np.nonzero(level >= lvl)[0].astype(np.int32)
        if len(ids) < min_nodes:
            break
        nb, entry = build_graph(np.ascontiguousarray(X[ids]), min(R, len(ids) - 1), device=device)
        layers.append({"ids": ids, "nbrs": nb.astype(np.int32), "entry": int(entry)})
        lvl += 1
    if not layers:
        raise ValueError("no upper layer has enough nodes (lower M or min_nodes)")
    for lo, hi in zip(layers[:-1], layers[1:]):
        hi["down"] = np.searchsorted(lo["ids"], hi["ids"]).astype(np.int32)
        assert np.array_equal(lo["ids"][hi["down"]], hi["ids"])
    layers = layers[::-1]
    return layers, layers[0]["entry"]
