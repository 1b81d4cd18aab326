"""Uneven query batches: thousands of queries with their own k and efs in one
persistent search launch (peos_search_batch), captured into a CUDA graph and
replayed, with the launch shape chosen by a small autotuner.

The launch shape (queries resident per CTA, visited-table slots per query, rows per
gather batch) changes only speed, never results: the visited table is lossy by design
(a forgotten node is re-evaluated and rejected again) and the gather width only
regroups the same per-row sums.  The beam width (nodes expanded per iteration) is also
tuned when the caller offers more than one: it changes the search itself (more nodes
expanded per iteration, usually a recall at least as high at the same efs), so a caller
that tunes it checks the recall of the shape it gets.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import torch

from . import peos as _p


@dataclass
class Shape:
    warps_per_cta: int = 0   # 0 = library default (8, lowered to fit shared memory)
    visited_slots: int = 0   # 0 = library default (16 x efs in 512..4096, lowered where shared memory
                             #     rather than registers would limit the resident CTAs)
    gather_rows: int = 0     # 0 = routing default (8 plain, 4 PEOs)
    beam: int = 1            # nodes expanded per iteration (1, 2 or 4)

    def kw(self) -> dict:
        return dict(warps_per_cta=self.warps_per_cta, visited_slots=self.visited_slots,
                    gather_rows=self.gather_rows, beam=self.beam)


@dataclass
class TuneResult:
    best: Shape
    ms: float
    table: list = field(default_factory=list)  # (shape, ms) for every candidate that ran


def candidate_shapes(ef_max: int, beams=(1,)) -> list[Shape]:
    """Launch shapes the tuner tries: queries per CTA x visited slots x gather rows
    (x beam widths, when more than one is offered)."""
    slots = [0] + [s for s in (1024, 2048, 4096) if s >= 2 * ef_max]
    return [Shape(w, s, g, b) for w, s, g, b in itertools.product((2, 4, 8), slots, (4, 8), beams)]


def autotune(graph, codes, base, queries: torch.Tensor, k_max: int, ef_max: int, k_per_query=None,
             ef_per_query=None, rerank=None, candidates: list[Shape] | None = None, reps: int = 3,
             beams=(1,), **search_kw) -> TuneResult:
    """Time each candidate shape on the given batch (a representative sample of the
    workload) with CUDA events and return the fastest.  Shapes the library rejects
    (shared memory beyond the per-CTA limit, a beam width the variant lacks) are skipped."""
    cands = candidates or candidate_shapes(ef_max, beams)
    nq = queries.shape[0]
    stream = torch.cuda.current_stream()
    ids = torch.empty((nq, k_max), dtype=torch.int32, device=queries.device)
    dists = torch.empty((nq, k_max), dtype=torch.float32, device=queries.device)
    table = []
    for sh in cands:
        kw = dict(search_kw, **sh.kw())
        try:
            ws_bytes = _p.batch_workspace_size(graph, codes, base, nq, k_max, ef_max, rerank, **kw)
        except _p.PeosError:
            continue
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device=queries.device)

        def run():
            _p.search_batch(graph, codes, base, queries, k_max, ef_max, k_per_query, ef_per_query, workspace=ws,
                            rerank=rerank, out=(ids, dists, None), **kw)
        run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            run()
        e1.record(stream)
        torch.cuda.synchronize()
        table.append((sh, e0.elapsed_time(e1) / reps))
    if not table:
        raise RuntimeError("no candidate launch shape fits this device")
    best = min(table, key=lambda t: t[1])
    return TuneResult(best[0], best[1], table)


class BatchPlan:
    """Fixed device buffers for batches of up to `capacity` queries, one persistent
    search launch per batch, optionally captured into a CUDA graph.

    load() copies a batch (queries, per-query k and efs) into the plan's buffers on the
    current stream; run() replays the captured graph (or calls the library directly);
    results are views of the plan's output buffers."""

    def __init__(self, graph, codes, base, d: int, capacity: int, k_max: int, ef_max: int, rerank=None,
                 shape: Shape | None = None, device="cuda", **search_kw):
        self.graph, self.codes, self.base, self.rerank = graph, codes, base, rerank
        self.capacity, self.k_max, self.ef_max = capacity, k_max, ef_max
        self.shape = shape or Shape()
        self.kw = dict(search_kw, **self.shape.kw())
        dev = torch.device(device)
        self.queries = torch.zeros((capacity, d), dtype=torch.float32, device=dev)
        self.k_q = torch.full((capacity,), k_max, dtype=torch.int32, device=dev)
        self.ef_q = torch.full((capacity,), ef_max, dtype=torch.int32, device=dev)
        self.ids = torch.empty((capacity, k_max), dtype=torch.int32, device=dev)
        self.dists = torch.empty((capacity, k_max), dtype=torch.float32, device=dev)
        nbytes = _p.batch_workspace_size(graph, codes, base, capacity, k_max, ef_max, rerank, **self.kw)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        self.cuda_graph = None

    def load(self, queries: torch.Tensor, k_per_query: torch.Tensor, ef_per_query: torch.Tensor):
        n = queries.shape[0]
        if n != self.capacity:
            raise ValueError("a plan runs batches of exactly its capacity (pad with repeated queries)")
        self.queries.copy_(queries, non_blocking=True)
        self.k_q.copy_(k_per_query, non_blocking=True)
        self.ef_q.copy_(ef_per_query, non_blocking=True)

    def _launch(self):
        _p.search_batch(self.graph, self.codes, self.base, self.queries, self.k_max, self.ef_max, self.k_q,
                        self.ef_q, workspace=self.workspace, rerank=self.rerank, out=(self.ids, self.dists, None),
                        **self.kw)

    def capture(self):
        """Capture one batch launch into a CUDA graph (after one direct call, which
        loads the kernels and sets their attributes outside the capture)."""
        self._launch()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self._launch()
        self.cuda_graph = g
        return self

    def run(self):
        if self.cuda_graph is not None:
            self.cuda_graph.replay()
        else:
            self._launch()
        return self.ids, self.dists
