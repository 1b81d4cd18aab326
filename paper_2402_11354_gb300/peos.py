"""Python binding of the PEOs C ABI (include/peos.h): argument marshalling only.

Every step of the search and of the index build runs in the CUDA library
libpeos.so; torch tensors only carry device memory and streams.  There is no
CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

PEOS_OK = 0
STATUS_NAMES = {0: "PEOS_OK", 1: "PEOS_E_INVAL", 2: "PEOS_E_NOMEM", 3: "PEOS_E_CUDA", 4: "PEOS_E_OVERFLOW",
                5: "PEOS_E_TIMEOUT", 6: "PEOS_E_UNSUPPORTED"}
COUNTER_NAMES = ["expansions", "edges", "visited_skip", "a_reject", "a_accept", "h_tests", "h_pass", "n_dist",
                 "inserts", "status", "full_expansions"]
NCOUNTERS = len(COUNTER_NAMES)
F32, BF16, FP8E4M3 = 0, 1, 2
DTYPES = {"f32": F32, "bf16": BF16, "e4m3": FP8E4M3}


class PeosError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("R", ctypes.c_int32), ("entry", ctypes.c_int32), ("nbrs", ctypes.c_void_p)]


class _Matrix(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("scales", ctypes.c_void_p), ("n", ctypes.c_int64), ("d", ctypes.c_int32),
                ("dtype", ctypes.c_int32)]


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("ef", ctypes.c_int32), ("eps", ctypes.c_float), ("routing", ctypes.c_int32),
                ("test_mode", ctypes.c_int32), ("eta_mode", ctypes.c_int32), ("max_expansions", ctypes.c_int32),
                ("visited_slots", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32), ("gather_rows", ctypes.c_int32),
                ("entries", ctypes.c_void_p), ("frame", ctypes.c_int32), ("beam", ctypes.c_int32)]


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("R", ctypes.c_int32), ("L", ctypes.c_int32), ("m", ctypes.c_int32),
                ("d", ctypes.c_int32), ("entry", ctypes.c_int32), ("record_stride", ctypes.c_size_t),
                ("node_proj_stride", ctypes.c_int32), ("records", ctypes.c_void_p), ("node_proj", ctypes.c_void_p),
                ("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("perm", ctypes.c_void_p), ("kind", ctypes.c_int32),
                ("norms", ctypes.c_void_p), ("scalar_bits", ctypes.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpeos.so (building it first if it is missing or stale and nvcc is available)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("PEOS_LIBRARY") or _build.LIB
    if build_if_missing and not os.environ.get("PEOS_LIBRARY"):
        try:
            path = _build.build()
        except RuntimeError:
            if not os.path.exists(path):
                raise
    if not os.path.exists(path):
        raise RuntimeError(f"PEOs CUDA library not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    lib.peos_last_error.restype = ctypes.c_char_p
    lib.peos_version.restype = ctypes.c_char_p
    for name in ("peos_build_codes", "peos_codes_free", "peos_codes_get_info", "peos_codes_export", "peos_search",
                 "peos_search_rerank", "peos_quantize", "peos_search_host", "peos_search_noalloc",
                 "peos_trace_enable", "peos_trace_read", "peos_search_batch", "peos_search_batch_workspace_size",
                 "peos_server_create", "peos_server_submit", "peos_server_replay", "peos_server_poll",
                 "peos_server_stats", "peos_server_destroy", "peos_knn_tensor",
                 "peos_release_workspace", "peos_edge_stats", "peos_projections", "peos_knn_bruteforce",
                 "peos_dim_permutation", "peos_build_codes_permuted", "peos_hier_entry", "peos_build_simhash", "peos_search_host_async",
                 "peos_selftest_bounded_wait", "peos_crc32", "peos_codes_save", "peos_codes_load", "peos_codes_graph", "peos_check_read",
                 "peos_build_codes_compact"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(rc: int):
    if rc != PEOS_OK:
        raise PeosError(rc, load().peos_last_error().decode())


def _stream(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 2):
        raise TypeError(f"{name} must be a 2-D float32 CUDA tensor")
    return t.contiguous()


def _matrix(t: torch.Tensor) -> _Matrix:
    return _Matrix(t.data_ptr() if t.numel() else None, None, t.shape[0], t.shape[1], F32)


@dataclass
class StoredBase:
    """Base vectors in reduced-precision storage: data [n, d] (torch.bfloat16, or uint8
    E4M3 codes) and, for E4M3, one FP32 scale per row (element = scale * value(code))."""
    data: torch.Tensor
    scales: torch.Tensor | None
    dtype: str  # "bf16" or "e4m3"

    @property
    def shape(self):
        return self.data.shape

    def nbytes(self) -> int:
        return self.data.numel() * self.data.element_size() + (0 if self.scales is None else 4 * self.scales.numel())


def _base(base) -> tuple[_Matrix, object]:
    """peos_matrix for a search base: an FP32 tensor or a StoredBase.  Returns the struct
    and the objects it points into (kept alive by the caller)."""
    if isinstance(base, StoredBase):
        t = base.data
        if not (t.is_cuda and t.dim() == 2 and t.is_contiguous()):
            raise TypeError("StoredBase.data must be a contiguous 2-D CUDA tensor")
        code = DTYPES[base.dtype]
        if code == BF16 and t.dtype != torch.bfloat16:
            raise TypeError("bf16 storage must be a torch.bfloat16 tensor")
        if code == FP8E4M3 and t.dtype not in (torch.uint8, torch.float8_e4m3fn):
            raise TypeError("e4m3 storage must be uint8 codes or torch.float8_e4m3fn")
        sc = base.scales
        if code == FP8E4M3:
            if sc is None or not (sc.is_cuda and sc.dtype == torch.float32 and sc.is_contiguous()):
                raise TypeError("e4m3 storage needs per-row float32 CUDA scales")
        M = _Matrix(t.data_ptr() if t.numel() else None, sc.data_ptr() if (sc is not None and code == FP8E4M3) else None,
                    t.shape[0], t.shape[1], code)
        return M, base
    t = _dev_f32(base, "base")
    return _matrix(t), t


def quantize(base: torch.Tensor, dtype: str, stream=None) -> StoredBase:
    """Reduced-precision copy of an FP32 base on the device (bf16, or e4m3 with per-row scales)."""
    base = _dev_f32(base, "base")
    n, d = base.shape
    code = DTYPES.get(dtype)
    if code == BF16:
        data = torch.empty((n, d), dtype=torch.bfloat16, device=base.device)
        scales = None
    elif code == FP8E4M3:
        data = torch.empty((n, d), dtype=torch.uint8, device=base.device)
        scales = torch.empty(n, dtype=torch.float32, device=base.device)
    else:
        raise ValueError("dtype must be 'bf16' or 'e4m3'")
    M = _matrix(base)
    _check(load().peos_quantize(ctypes.byref(M), ctypes.c_int32(code), ctypes.c_void_p(data.data_ptr() if n else 0),
                                ctypes.c_void_p(scales.data_ptr() if scales is not None and n else 0),
                                _stream(stream)))
    return StoredBase(data, scales, dtype)


@dataclass
class Graph:
    """Graph index on the device: nbrs [n, R] int32 (-1 = empty slot) and the entry node."""
    nbrs: torch.Tensor
    entry: int

    @property
    def n(self) -> int:
        return self.nbrs.shape[0]

    @property
    def R(self) -> int:
        return self.nbrs.shape[1]

    def c(self) -> _Graph:
        if not (self.nbrs.is_cuda and self.nbrs.dtype == torch.int32 and self.nbrs.is_contiguous()):
            raise TypeError("Graph.nbrs must be a contiguous int32 CUDA tensor")
        return _Graph(self.n, self.R, int(self.entry), self.nbrs.data_ptr())

    @staticmethod
    def from_numpy(nbrs: np.ndarray, entry: int, device="cuda") -> "Graph":
        return Graph(torch.from_numpy(np.ascontiguousarray(nbrs, dtype=np.int32)).to(device), int(entry))


class Codes:
    """PEOs index data owned by the library (peos_build_codes / peos_codes_free)."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = _Info()
        _check(load().peos_codes_get_info(self._h, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in _Info._fields_}

    def arrays(self) -> dict:
        """Host copies of the index arrays (records split into their fields)."""
        inf = self.info()
        n, R, L, m, d = inf["n"], inf["R"], inf["L"], inf["m"], inf["d"]
        if inf["kind"] == 1:  # SimHash: ||e||, ids, K sign bits per edge, node table, S
            K, W = m, m // 64
            raw = np.empty((n, inf["record_stride"]), dtype=np.uint8)
            tv = np.empty((n, K), dtype=np.float32)
            S = np.empty((K, d), dtype=np.float32)
            _check(load().peos_codes_export(self._h, ctypes.c_void_p(raw.ctypes.data),
                                            ctypes.c_void_p(tv.ctypes.data), None, ctypes.c_void_p(S.ctypes.data)))
            en = np.ascontiguousarray(raw[:, :16 * R].copy().view(np.float32).reshape(n, R, 4)[:, :, 0])
            ids = raw[:, 16 * R:20 * R].copy().view(np.int32)
            off = (20 * R + 15) // 16 * 16
            bits = raw[:, off:off + 8 * W * R].copy().view(np.uint64).reshape(n, W, R).transpose(0, 2, 1)
            return dict(ids=ids, en=en, bits=np.ascontiguousarray(bits), tv=tv, S=S, record_stride=inf["record_stride"])
        stride = inf["record_stride"]
        raw = np.empty((n, stride), dtype=np.uint8)
        tstride = inf["node_proj_stride"]
        tvp = np.empty((n, tstride), dtype=np.float32)
        A = np.empty((L, m, d // L), dtype=np.float32)
        B = np.empty((m, d), dtype=np.float32)
        _check(load().peos_codes_export(self._h, ctypes.c_void_p(raw.ctypes.data), ctypes.c_void_p(tvp.ctypes.data),
                                        ctypes.c_void_p(A.ctypes.data), ctypes.c_void_p(B.ctypes.data)))
        tv = np.ascontiguousarray(tvp[:, :(L + 1) * m]).reshape(n, L + 1, m)
        sb = inf["scalar_bits"]
        extra = {}
        if sb == 32:
            scal = raw[:, :16 * R].copy().view(np.float32).reshape(n, R, 4)
            ids_off = 16 * R
        else:  # the node's steps, then per edge 4 signed integers (the fourth unused) and the
            # FP32 node term: 16-bit as sv[R] then q[R], 8-bit as {q, sv} pairs; the search
            # reads q * step
            steps = raw[:, :16].copy().view(np.float32)[:, :3]
            if sb == 16:
                sv = raw[:, 16:16 + 4 * R].copy().view(np.float32)
                q_off = (16 + 4 * R + 7) // 8 * 8
                q = raw[:, q_off:q_off + 8 * R].copy().view(np.int16).reshape(n, R, 4)
                ids_off = q_off + 8 * R
            else:
                pairs = raw[:, 16:16 + 8 * R].copy().reshape(n, R, 8)
                q = np.ascontiguousarray(pairs[:, :, :4]).view(np.int8).reshape(n, R, 4)
                sv = np.ascontiguousarray(pairs[:, :, 4:]).view(np.float32).reshape(n, R)
                ids_off = 16 + 8 * R
            q = q[:, :, :3].astype(np.int32)
            scal = np.concatenate([(q.astype(np.float32) * steps[:, None, :]).astype(np.float32), sv[:, :, None]],
                                  axis=2)
            extra = dict(steps=np.ascontiguousarray(steps), q=np.ascontiguousarray(q))
        enorm, wreg, cres, sv = (np.ascontiguousarray(scal[:, :, i]) for i in range(4))
        ids = raw[:, ids_off:ids_off + 4 * R].copy().view(np.int32)
        codes = unpack_codes(raw[:, (ids_off + 4 * R + 15) // 16 * 16:], R, L, m)
        codes[ids < 0] = 0  # empty slots carry no codes
        return dict(ids=ids, enorm=enorm, wreg=wreg, cres=cres, sv=sv, codes=np.ascontiguousarray(codes), tv=tv, A=A,
                    B=B, record_stride=stride, **extra)

    def save(self, path: str):
        """Write the handle to an index file (peos_codes_save); load it with load_codes."""
        _check(load().peos_codes_save(self._h, os.fsencode(path)))

    def graph(self, stream=None) -> Graph:
        """The graph the index was built on (edge ids from its records, its entry node)."""
        inf = self.info()
        nbrs = torch.empty((inf["n"], inf["R"]), dtype=torch.int32, device="cuda")
        entry = ctypes.c_int32()
        _check(load().peos_codes_graph(self._h, ctypes.c_void_p(nbrs.data_ptr()), ctypes.byref(entry),
                                       _stream(stream)))
        torch.cuda.current_stream().synchronize() if stream is None else None
        return Graph(nbrs, entry.value)

    def free(self):
        if self._h:
            _check(load().peos_codes_free(self._h))
            self._h = None

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.peos_codes_free(self._h)
        except Exception:
            pass


def load_codes(path: str) -> Codes:
    """Read an index file written by Codes.save into a new handle on the current device
    (every field and section checksum is checked: PeosError on a damaged file)."""
    h = ctypes.c_void_p()
    _check(load().peos_codes_load(os.fsencode(path), ctypes.byref(h)))
    return Codes(h)


def crc32(data: bytes) -> int:
    """CRC-32 (zlib / IEEE 802.3) as the index files use it."""
    out = ctypes.c_uint32()
    buf = ctypes.create_string_buffer(bytes(data), len(data))
    _check(load().peos_crc32(buf, ctypes.c_size_t(len(data)), ctypes.byref(out)))
    return out.value


def code_bits(m: int) -> int:
    b = 1
    while (1 << b) < m:
        b += 1
    return b + 1


def unpack_codes(raw: np.ndarray, R: int, L: int, m: int) -> np.ndarray:
    """Packed record codes -> signed codes [n, R, L+1] (sgn * (j + 1))."""
    bits = code_bits(m)
    cpw = 64 // bits
    W = (L + 1 + cpw - 1) // cpw
    n = raw.shape[0]
    words = np.ascontiguousarray(raw[:, :8 * W * R]).view(np.uint64).reshape(n, W, R)
    out = np.zeros((n, R, L + 1), dtype=np.int8)
    for c in range(L + 1):
        w, t = divmod(c, cpw)
        code = (words[:, w, :] >> np.uint64(t * bits)) & np.uint64((1 << bits) - 1)
        j = (code & np.uint64((1 << (bits - 1)) - 1)).astype(np.int16) + 1
        neg = (code >> np.uint64(bits - 1)).astype(bool)
        out[:, :, c] = np.where(neg, -j, j)
    return out


def dim_permutation(graph: Graph, base: torch.Tensor, L: int, stream=None) -> torch.Tensor:
    """Appendix D.1's dimension permutation of `base` over the graph's edges (int32 [d],
    device): entry i*(d/L) + t is the coordinate that becomes coordinate t of subspace i."""
    base = _dev_f32(base, "base")
    perm = torch.empty(base.shape[1], dtype=torch.int32, device=base.device)
    g = graph.c()
    M = _matrix(base)
    _check(load().peos_dim_permutation(ctypes.byref(g), ctypes.byref(M), ctypes.c_int32(L),
                                       ctypes.c_void_p(perm.data_ptr()), _stream(stream)))
    return perm


def build_codes(graph: Graph, base: torch.Tensor, L: int, m: int, seed: int, stream=None,
                perm: torch.Tensor | None = None, scalar_bits: int = 32) -> Codes:
    """Sec. 4.2 steps (1)-(3) for every edge, plus the node projection tables; with `perm`
    (int32 [d], device) in the permuted coordinates of Appendix D.1; with scalar_bits 16
    or 8 the compact index (edge scalars quantised per node, peos_build_codes_compact)."""
    base = _dev_f32(base, "base")
    h = ctypes.c_void_p()
    g = graph.c()
    M = _matrix(base)
    if scalar_bits != 32:
        if perm is not None:
            raise ValueError("the compact index has no dimension permutation")
        _check(load().peos_build_codes_compact(ctypes.byref(g), ctypes.byref(M), ctypes.c_int32(L), ctypes.c_int32(m),
                                               ctypes.c_uint64(seed), ctypes.c_int32(scalar_bits), _stream(stream),
                                               ctypes.byref(h)))
    elif perm is None:
        _check(load().peos_build_codes(ctypes.byref(g), ctypes.byref(M), ctypes.c_int32(L), ctypes.c_int32(m),
                                       ctypes.c_uint64(seed), _stream(stream), ctypes.byref(h)))
    else:
        if not (perm.is_cuda and perm.dtype == torch.int32 and perm.numel() == base.shape[1]):
            raise TypeError("perm must be an int32 CUDA tensor of d entries")
        perm = perm.contiguous()
        _check(load().peos_build_codes_permuted(ctypes.byref(g), ctypes.byref(M), ctypes.c_int32(L),
                                                ctypes.c_int32(m), ctypes.c_uint64(seed),
                                                ctypes.c_void_p(perm.data_ptr()), _stream(stream), ctypes.byref(h)))
    return Codes(h)


def build_simhash(graph: Graph, base: torch.Tensor, K: int, seed: int, stream=None) -> Codes:
    """Index data of the SimHash routing test (K sign bits per edge, node table); search
    it with routing=2."""
    base = _dev_f32(base, "base")
    h = ctypes.c_void_p()
    g = graph.c()
    M = _matrix(base)
    _check(load().peos_build_simhash(ctypes.byref(g), ctypes.byref(M), ctypes.c_int32(K), ctypes.c_uint64(seed),
                                     _stream(stream), ctypes.byref(h)))
    return Codes(h)


def _params(k, ef, eps, routing, test_mode, eta_mode, max_expansions, visited_slots, warps_per_cta,
            gather_rows=0, entries=None, frame=0, beam=0) -> _Params:
    return _Params(int(k), int(ef), float(eps), int(routing), int(test_mode), int(eta_mode), int(max_expansions),
                   int(visited_slots), int(warps_per_cta), int(gather_rows), entries, int(frame), int(beam))


def _entries(entries, nq: int, host: bool = False):
    """Pointer to per-query entry nodes (int32 [nq]: a CUDA tensor, or host memory for the
    host-buffer call), or None."""
    if entries is None:
        return None
    if host:
        if isinstance(entries, torch.Tensor):
            if entries.is_cuda or entries.dtype != torch.int32 or not entries.is_contiguous() or entries.numel() != nq:
                raise TypeError("entries must be a contiguous int32 host array of nq values")
            return entries.data_ptr()
        arr = np.asarray(entries)
        if arr.dtype != np.int32 or not arr.flags.c_contiguous or arr.size != nq:
            raise TypeError("entries must be a contiguous int32 host array of nq values")
        return arr.ctypes.data
    if not (isinstance(entries, torch.Tensor) and entries.is_cuda and entries.dtype == torch.int32
            and entries.is_contiguous() and entries.numel() == nq):
        raise TypeError("entries must be a contiguous int32 CUDA tensor of nq values")
    return entries.data_ptr() if nq else None


def search(graph: Graph, codes: Codes | None, base, queries: torch.Tensor, k: int, ef: int,
           eps: float = 0.2, routing: int = 1, test_mode: int = 0, eta_mode: int = 0, max_expansions: int = 0,
           visited_slots: int = 0, warps_per_cta: int = 0, counters: bool = False, out=None, stream=None,
           rerank: torch.Tensor | None = None, gather_rows: int = 0, entries: torch.Tensor | None = None,
           frame: int = 0, beam: int = 0):
    """Batched search (device tensors in and out).  `base` is an FP32 tensor or a StoredBase
    (reduced precision); `rerank` (FP32 base) re-ranks each final list exactly before the
    top k are taken; `entries` (int32 [nq], e.g. from hier_entry) gives each query its own
    entry node; `beam` = nodes expanded per iteration (0/1, 2 or 4).
    Returns (ids [nq,k] int32, dists [nq,k] f32, counters|None)."""
    Mb, keep = _base(base)
    queries = _dev_f32(queries, "queries")
    nq = queries.shape[0]
    if out is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
        cnt = torch.zeros((nq, NCOUNTERS), dtype=torch.int32, device=queries.device) if counters else None
    else:
        ids, dists, cnt = out
    g = graph.c()
    Mq = _matrix(queries)
    P = _params(k, ef, eps, routing, test_mode, eta_mode, max_expansions, visited_slots, warps_per_cta, gather_rows,
                _entries(entries, nq), frame, beam)
    h = codes.handle if codes is not None else None
    args = (ctypes.byref(Mq), ctypes.byref(P), ctypes.c_void_p(ids.data_ptr() if nq else 0),
            ctypes.c_void_p(dists.data_ptr() if nq else 0),
            ctypes.c_void_p(cnt.data_ptr() if cnt is not None and nq else 0), _stream(stream))
    if rerank is None:
        _check(load().peos_search(ctypes.byref(g), h, ctypes.byref(Mb), *args))
    else:
        rr = _dev_f32(rerank, "rerank")
        Mr = _matrix(rr)
        _check(load().peos_search_rerank(ctypes.byref(g), h, ctypes.byref(Mb), ctypes.byref(Mr), *args))
    del keep
    return ids, dists, cnt


def search_noalloc(graph: Graph, codes: Codes | None, base: torch.Tensor, queries: torch.Tensor, k: int, ef: int,
                   eps: float = 0.2, routing: int = 1, test_mode: int = 0, eta_mode: int = 0, max_expansions: int = 0,
                   visited_slots: int = 0, warps_per_cta: int = 0, counters: bool = False, out=None, stream=None,
                   gather_rows: int = 0, entries: torch.Tensor | None = None, beam: int = 0):
    """Like search(), for callers that cannot allocate device memory while serving: the
    library uses a fixed scratch array in its own device image instead of pool memory.
    Calls on one device share that array and must not overlap on the GPU."""
    Mb, keep = _base(base)
    queries = _dev_f32(queries, "queries")
    nq = queries.shape[0]
    if out is None:
        ids = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
        dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
        cnt = torch.zeros((nq, NCOUNTERS), dtype=torch.int32, device=queries.device) if counters else None
    else:
        ids, dists, cnt = out
    g = graph.c()
    Mq = _matrix(queries)
    P = _params(k, ef, eps, routing, test_mode, eta_mode, max_expansions, visited_slots, warps_per_cta,
                gather_rows, _entries(entries, nq), 0, beam)
    _check(load().peos_search_noalloc(ctypes.byref(g), codes.handle if codes is not None else None, ctypes.byref(Mb),
                                      ctypes.byref(Mq), ctypes.byref(P), ctypes.c_void_p(ids.data_ptr() if nq else 0),
                                      ctypes.c_void_p(dists.data_ptr() if nq else 0),
                                      ctypes.c_void_p(cnt.data_ptr() if cnt is not None and nq else 0),
                                      _stream(stream)))
    return ids, dists, cnt


def search_host(graph: Graph, codes: Codes | None, base: torch.Tensor, queries: np.ndarray, k: int, ef: int,
                eps: float = 0.2, routing: int = 1, test_mode: int = 0, eta_mode: int = 0, max_expansions: int = 0,
                visited_slots: int = 0, warps_per_cta: int = 0, counters: bool = False, out=None, stream=None,
                gather_rows: int = 0, entries=None, wait: bool = True, beam: int = 0):
    """Search with queries and results in host memory (numpy or pinned torch CPU tensors);
    the library copies in, searches and copies out, and returns after the stream drains.
    With wait=False the work is only enqueued (peos_search_host_async): the buffers must be
    pinned and stay untouched until the stream is synchronised."""
    Mb, keep = _base(base)
    if isinstance(queries, torch.Tensor):
        qp = queries.data_ptr()
        nq = queries.shape[0]
    else:
        queries = np.ascontiguousarray(queries, dtype=np.float32)
        qp = queries.ctypes.data
        nq = queries.shape[0]
    if out is None:
        ids = np.empty((nq, k), dtype=np.int32)
        dists = np.empty((nq, k), dtype=np.float32)
        cnt = np.zeros((nq, NCOUNTERS), dtype=np.int32) if counters else None
    else:
        ids, dists, cnt = out

    def ptr(a):
        if a is None:
            return None
        return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data

    g = graph.c()
    P = _params(k, ef, eps, routing, test_mode, eta_mode, max_expansions, visited_slots, warps_per_cta,
                gather_rows, _entries(entries, nq, host=True), 0, beam)
    fn = load().peos_search_host if wait else load().peos_search_host_async
    _check(fn(ctypes.byref(g), codes.handle if codes is not None else None, ctypes.byref(Mb),
                                   ctypes.c_void_p(qp), ctypes.c_int64(nq), ctypes.byref(P),
                                   ctypes.c_void_p(ptr(ids)), ctypes.c_void_p(ptr(dists)), ctypes.c_void_p(ptr(cnt)),
                                   _stream(stream)))
    return ids, dists, cnt


def batch_workspace_size(graph: Graph, codes: Codes | None, base, nq: int, k_max: int, ef_max: int,
                         rerank: torch.Tensor | None = None, **kw) -> int:
    """Bytes of device workspace a search_batch call of nq queries needs."""
    Mb, keep = _base(base)
    g = graph.c()
    P = _params(k_max, ef_max, kw.get("eps", 0.2), kw.get("routing", 1), kw.get("test_mode", 0),
                kw.get("eta_mode", 0), kw.get("max_expansions", 0), kw.get("visited_slots", 0),
                kw.get("warps_per_cta", 0), kw.get("gather_rows", 0), None, kw.get("frame", 0), kw.get("beam", 0))
    Mr = _matrix(_dev_f32(rerank, "rerank")) if rerank is not None else None
    out = ctypes.c_size_t()
    _check(load().peos_search_batch_workspace_size(ctypes.byref(g), codes.handle if codes is not None else None,
                                                   ctypes.byref(Mb), ctypes.byref(Mr) if Mr is not None else None,
                                                   ctypes.c_int64(nq), ctypes.byref(P), ctypes.byref(out)))
    return out.value


def search_batch(graph: Graph, codes: Codes | None, base, queries: torch.Tensor, k_max: int, ef_max: int,
                 k_per_query: torch.Tensor | None = None, ef_per_query: torch.Tensor | None = None,
                 workspace: torch.Tensor | None = None, rerank: torch.Tensor | None = None, eps: float = 0.2,
                 routing: int = 1, test_mode: int = 0, eta_mode: int = 0, max_expansions: int = 0,
                 visited_slots: int = 0, warps_per_cta: int = 0, gather_rows: int = 0, counters: bool = False,
                 out=None, stream=None, entries: torch.Tensor | None = None, frame: int = 0, beam: int = 0):
    """Uneven batch in one launch without allocation: query i uses its own efs and k
    (device int32 [nq] tensors; None = ef_max / k_max for all).  `workspace` is a uint8
    CUDA tensor of at least batch_workspace_size() bytes (allocated here when None).
    Returns (ids [nq, k_max], dists [nq, k_max], counters|None); slots >= k_i are -1 / inf."""
    Mb, keep = _base(base)
    queries = _dev_f32(queries, "queries")
    nq = queries.shape[0]
    for t, nm in ((k_per_query, "k_per_query"), (ef_per_query, "ef_per_query")):
        if t is not None and not (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous() and t.numel() == nq):
            raise TypeError(f"{nm} must be a contiguous int32 CUDA tensor of nq values")
    kw = dict(eps=eps, routing=routing, test_mode=test_mode, eta_mode=eta_mode, max_expansions=max_expansions,
              visited_slots=visited_slots, warps_per_cta=warps_per_cta, gather_rows=gather_rows, frame=frame,
              beam=beam)
    if workspace is None:
        workspace = torch.empty(batch_workspace_size(graph, codes, base, nq, k_max, ef_max, rerank, **kw),
                                dtype=torch.uint8, device=queries.device)
    if out is None:
        ids = torch.empty((nq, k_max), dtype=torch.int32, device=queries.device)
        dists = torch.empty((nq, k_max), dtype=torch.float32, device=queries.device)
        cnt = torch.zeros((nq, NCOUNTERS), dtype=torch.int32, device=queries.device) if counters else None
    else:
        ids, dists, cnt = out
    g = graph.c()
    Mq = _matrix(queries)
    P = _params(k_max, ef_max, eps, routing, test_mode, eta_mode, max_expansions, visited_slots, warps_per_cta,
                gather_rows, _entries(entries, nq), frame, beam)
    Mr = _matrix(_dev_f32(rerank, "rerank")) if rerank is not None else None

    def ptr(t):
        return ctypes.c_void_p(t.data_ptr() if t is not None and t.numel() else 0)
    _check(load().peos_search_batch(ctypes.byref(g), codes.handle if codes is not None else None, ctypes.byref(Mb),
                                    ctypes.byref(Mr) if Mr is not None else None, ctypes.byref(Mq), ctypes.byref(P),
                                    ptr(k_per_query), ptr(ef_per_query), ptr(ids), ptr(dists), ptr(cnt),
                                    ctypes.c_void_p(workspace.data_ptr()), ctypes.c_size_t(workspace.numel()),
                                    _stream(stream)))
    del keep
    return ids, dists, cnt


class _Layer(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("R", ctypes.c_int32), ("ids", ctypes.c_void_p), ("nbrs", ctypes.c_void_p),
                ("down", ctypes.c_void_p)]


class _Hierarchy(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int32), ("layers", ctypes.POINTER(_Layer)), ("top_entry", ctypes.c_int32)]


class Hierarchy:
    """Upper layers of an HNSW-style index on the device (peos_hierarchy): a list of
    layers top first, each a dict of numpy arrays ids [n_l], nbrs [n_l, R_l] (local ids)
    and, except on the lowest, down [n_l]; plus the top layer's entry (a local id)."""

    def __init__(self, layers: list, top_entry: int, device="cuda"):
        self.top_entry = int(top_entry)
        self.tensors = []
        for i, lay in enumerate(layers):
            t = {"ids": torch.from_numpy(np.ascontiguousarray(lay["ids"], dtype=np.int32)).to(device),
                 "nbrs": torch.from_numpy(np.ascontiguousarray(lay["nbrs"], dtype=np.int32)).to(device)}
            if i + 1 < len(layers):
                t["down"] = torch.from_numpy(np.ascontiguousarray(lay["down"], dtype=np.int32)).to(device)
            self.tensors.append(t)

    def c(self):
        arr = (_Layer * len(self.tensors))()
        for i, t in enumerate(self.tensors):
            arr[i] = _Layer(t["ids"].numel(), t["nbrs"].shape[1], t["ids"].data_ptr(), t["nbrs"].data_ptr(),
                            t["down"].data_ptr() if "down" in t else None)
        h = _Hierarchy(len(self.tensors), ctypes.cast(arr, ctypes.POINTER(_Layer)), self.top_entry)
        return h, arr


def hier_entry(hierarchy: Hierarchy, base, queries: torch.Tensor, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """Entry node of every query by greedy descent through the upper layers (int32 [nq], device)."""
    Mb, keep = _base(base)
    queries = _dev_f32(queries, "queries")
    nq = queries.shape[0]
    entries = out if out is not None else torch.empty(nq, dtype=torch.int32, device=queries.device)
    h, arr = hierarchy.c()
    Mq = _matrix(queries)
    _check(load().peos_hier_entry(ctypes.byref(h), ctypes.byref(Mb), ctypes.byref(Mq),
                                  ctypes.c_void_p(entries.data_ptr() if nq else 0), _stream(stream)))
    del keep, arr
    return entries


def knn_bruteforce(base: torch.Tensor, queries: torch.Tensor, k: int, stream=None):
    """Exact K-NN (FP32 sums of squared differences, ties by id) on the device."""
    base = _dev_f32(base, "base")
    queries = _dev_f32(queries, "queries")
    nq = queries.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
    Mb, Mq = _matrix(base), _matrix(queries)
    _check(load().peos_knn_bruteforce(ctypes.byref(Mb), ctypes.byref(Mq), ctypes.c_int32(k),
                                      ctypes.c_void_p(ids.data_ptr() if nq else 0),
                                      ctypes.c_void_p(dists.data_ptr() if nq else 0), _stream(stream)))
    return ids, dists


def knn_tensor(base: torch.Tensor, queries: torch.Tensor, k: int, stream=None):
    """Exact-rerank K-NN on the tensor cores (BF16 scores, FP32 exact distances of the
    candidates); 1 <= k <= 96.  Synchronous."""
    base = _dev_f32(base, "base")
    queries = _dev_f32(queries, "queries")
    nq = queries.shape[0]
    ids = torch.empty((nq, k), dtype=torch.int32, device=queries.device)
    dists = torch.empty((nq, k), dtype=torch.float32, device=queries.device)
    Mb, Mq = _matrix(base), _matrix(queries)
    _check(load().peos_knn_tensor(ctypes.byref(Mb), ctypes.byref(Mq), ctypes.c_int32(k),
                                  ctypes.c_void_p(ids.data_ptr() if nq else 0),
                                  ctypes.c_void_p(dists.data_ptr() if nq else 0), _stream(stream)))
    return ids, dists


def edge_stats(codes: Codes, query: torch.Tensor, v: int, dv: float, delta2: float, eps: float = 0.2,
               eta_mode: int = 0, stream=None) -> dict:
    """PEOs statistics (A, H, T, pass, kind) of every out-edge of node v for one query (device code of the search)."""
    R = codes.info()["R"]
    q = query.contiguous().view(-1)
    if not (q.is_cuda and q.dtype == torch.float32):
        raise TypeError("query must be a float32 CUDA tensor")
    outs = [torch.zeros(R, dtype=torch.float32, device=q.device) for _ in range(3)] + \
           [torch.zeros(R, dtype=torch.int32, device=q.device) for _ in range(2)]
    _check(load().peos_edge_stats(codes.handle, ctypes.c_void_p(q.data_ptr()), ctypes.c_int32(v), ctypes.c_float(dv),
                                  ctypes.c_float(delta2), ctypes.c_float(eps), ctypes.c_int32(eta_mode),
                                  *[ctypes.c_void_p(o.data_ptr()) for o in outs], _stream(stream)))
    torch.cuda.current_stream().synchronize() if stream is None else None
    names = ["A", "H", "T", "passed", "kind"]
    return {nm: o.cpu().numpy() for nm, o in zip(names, outs)}


def selftest_bounded_wait(limit_us: int = 1000, stream=None) -> bool:
    """Run one bounded device wait, limited to `limit_us` microseconds, on an mbarrier
    nothing arrives on; True when it gave up (the failure detection works) and the device
    is still usable."""
    gave_up = ctypes.c_int32(-1)
    _check(load().peos_selftest_bounded_wait(ctypes.c_int64(limit_us), ctypes.byref(gave_up), _stream(stream)))
    return gave_up.value == 1


CHECK_KINDS = ["candidate", "expanded", "list_write", "list_order", "list_duplicate"]


def check_read() -> dict | None:
    """Violation counts of a self-checked library (built with checked=True), read and
    zeroed; None for a normal build."""
    buf = (ctypes.c_uint64 * 8)()
    rc = load().peos_check_read(buf)
    if rc == 6:  # PEOS_E_UNSUPPORTED: a normal build
        return None
    _check(rc)
    return {k: int(buf[i]) for i, k in enumerate(CHECK_KINDS)}


def projections(seed: int, d: int, L: int, m: int):
    """Host-side random vectors of Sec. 4.2 step (2): A [L, m, d/L], B [m, d] (FP32)."""
    A = np.zeros((L, m, d // L), dtype=np.float32)
    B = np.zeros((m, d), dtype=np.float32)
    _check(load().peos_projections(ctypes.c_uint64(seed), ctypes.c_int32(d), ctypes.c_int32(L), ctypes.c_int32(m),
                                   ctypes.c_void_p(A.ctypes.data), ctypes.c_void_p(B.ctypes.data)))
    return A, B


class _ServerConfig(ctypes.Structure):
    _fields_ = [("max_batch", ctypes.c_int32), ("streams", ctypes.c_int32), ("memory_budget", ctypes.c_size_t),
                ("k_max", ctypes.c_int32), ("ef_max", ctypes.c_int32), ("params", _Params)]


class _ServerResult(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("k", ctypes.c_int32), ("status", ctypes.c_int32),
                ("arrival_ns", ctypes.c_int64), ("admit_ns", ctypes.c_int64), ("complete_ns", ctypes.c_int64)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("pending", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("batched_queries", ctypes.c_uint64),
                ("admission_waits", ctypes.c_uint64), ("arena_bytes", ctypes.c_size_t),
                ("arena_used", ctypes.c_size_t), ("arena_peak", ctypes.c_size_t),
                ("batches_in_flight", ctypes.c_int32), ("last_error", ctypes.c_int32)]


class Server:
    """Continuous-batching search server (peos_server_*): graph, codes and base stay
    resident; requests are admitted by device memory and run in up to `streams`
    concurrent batch launches.  Results come back through poll()."""

    def __init__(self, graph: Graph, codes: Codes | None, base, k_max: int, ef_max: int, max_batch: int = 1024,
                 streams: int = 4, memory_budget: int = 256 << 20, rerank: torch.Tensor | None = None,
                 eps: float = 0.2, routing: int = 1, test_mode: int = 0, eta_mode: int = 0, max_expansions: int = 0,
                 visited_slots: int = 0, warps_per_cta: int = 0, gather_rows: int = 0, beam: int = 0):
        self._keep = (graph, codes, base, rerank)
        Mb, self._base_keep = _base(base)
        self._Mb = Mb
        self._Mr = _matrix(_dev_f32(rerank, "rerank")) if rerank is not None else None
        self._g = graph.c()
        self.d = Mb.d
        self.k_max = k_max
        cfg = _ServerConfig(max_batch, streams, memory_budget, k_max, ef_max,
                            _params(k_max, ef_max, eps, routing, test_mode, eta_mode, max_expansions, visited_slots,
                                    warps_per_cta, gather_rows, None, 0, beam))
        h = ctypes.c_void_p()
        _check(load().peos_server_create(ctypes.byref(self._g), codes.handle if codes is not None else None,
                                         ctypes.byref(self._Mb), ctypes.byref(self._Mr) if self._Mr else None,
                                         ctypes.c_int32(self.d), ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h

    def submit(self, request_id: int, query: np.ndarray, k: int, ef: int):
        q = np.ascontiguousarray(query, dtype=np.float32).reshape(-1)
        _check(load().peos_server_submit(self._h, ctypes.c_uint64(request_id), ctypes.c_void_p(q.ctypes.data),
                                         ctypes.c_int32(k), ctypes.c_int32(ef)))

    def replay(self, request_ids, queries: np.ndarray, k, ef, arrival_ns):
        """Submit request i at arrival_ns[i] after this call, from a native generator thread."""
        ids = np.ascontiguousarray(request_ids, dtype=np.uint64)
        q = np.ascontiguousarray(queries, dtype=np.float32)
        kk = np.ascontiguousarray(k, dtype=np.int32)
        ee = np.ascontiguousarray(ef, dtype=np.int32)
        at = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        _check(load().peos_server_replay(self._h, ctypes.c_int64(len(ids)), ctypes.c_void_p(ids.ctypes.data),
                                         ctypes.c_void_p(q.ctypes.data), ctypes.c_void_p(kk.ctypes.data),
                                         ctypes.c_void_p(ee.ctypes.data), ctypes.c_void_p(at.ctypes.data)))

    def poll(self, max_results: int = 4096, wait_us: int = 1000) -> dict:
        """Finished requests: dict of arrays (request_id, k, status, arrival_ns, admit_ns,
        complete_ns, ids [n, k_max], dists [n, k_max])."""
        res = (_ServerResult * max_results)()
        ids = np.empty((max_results, self.k_max), dtype=np.int32)
        dists = np.empty((max_results, self.k_max), dtype=np.float32)
        n = ctypes.c_int32()
        _check(load().peos_server_poll(self._h, ctypes.c_int32(max_results), res, ctypes.c_void_p(ids.ctypes.data),
                                       ctypes.c_void_p(dists.ctypes.data), ctypes.byref(n), ctypes.c_int32(wait_us)))
        n = n.value
        out = {f: np.array([getattr(res[i], f) for i in range(n)]) for f, _ in _ServerResult._fields_}
        out["ids"], out["dists"] = ids[:n], dists[:n]
        return out

    def stats(self) -> dict:
        st = _ServerStats()
        _check(load().peos_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in _ServerStats._fields_}

    def close(self):
        if self._h:
            _check(load().peos_server_destroy(self._h))
            self._h = None

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.peos_server_destroy(self._h)
        except Exception:
            pass


STAGES = ("setup", "search", "rerank")


def trace_enable(on: bool = True):
    """Record CUDA events around the stages of every later search call (device-time tracing)."""
    _check(load().peos_trace_enable(ctypes.c_int32(1 if on else 0)))


def trace_read() -> dict:
    """Wait for the traced calls and return {"calls": n, "<stage>_ms": summed device ms, ...}
    since the last read."""
    ms = (ctypes.c_double * len(STAGES))()
    calls = ctypes.c_int64()
    _check(load().peos_trace_read(ms, ctypes.byref(calls)))
    out = {"calls": calls.value}
    out.update({f"{s}_ms": ms[i] for i, s in enumerate(STAGES)})
    return out


def release_workspace():
    _check(load().peos_release_workspace())


def version() -> str:
    return load().peos_version().decode()
