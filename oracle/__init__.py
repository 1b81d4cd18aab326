"""PEOs oracle: plain CPU reference of the PEOs routing hot path (arXiv 2402.11354).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
never imports, links or calls it, and this package never imports the product.

The arithmetic lives in ``peos_oracle.c`` (plain sequential FP32 for the method,
FP64 for reference distances); this module only compiles it with gcc and
marshals numpy arrays.  See the header of ``peos_oracle.c`` for which function
follows which passage of the paper.

Parity pins (tests/test_oracle_*.py) tie every function to something outside the
oracle: numpy's own Philox4x64-10, textbook normal quantiles, the Gamma closed
form of Lemma 5.4, Monte Carlo moments of Eq. (combination), FP64 brute force,
and the paper's printed values (Lemma 5.4's 0.978, Table 6).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "peos_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libpeos_oracle.so")

N_COUNTERS = 10
COUNTER_NAMES = ["expansions", "edges", "visited_skip", "a_reject", "a_accept", "h_tests", "h_pass",
                 "n_dist", "inserts", "status"]
KIND_NAMES = {0: "reject_A>=1", 1: "accept_A<=0", 2: "H_test", 3: "degenerate", 4: "not_full", 5: "no_test"}


# -ffp-contract=off keeps a*b+c two roundings
_CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared"]


def compile_source(src: str, out: str) -> None:
    """Compile a C source of the oracle into the shared library `out` with the oracle's flags."""
    subprocess.check_call(["gcc", *_CFLAGS, "-o", out, src, "-lm"])


def build(force: bool = False) -> str:
    """Compile peos_oracle.c with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    compile_source(_SRC, tmp)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("ef", ctypes.c_int32), ("routing", ctypes.c_int32),
                ("test_mode", ctypes.c_int32), ("frame", ctypes.c_int32),
                ("max_expansions", ctypes.c_int32), ("trace_cap", ctypes.c_int32),
                ("z_eps", ctypes.c_float), ("c_eta", ctypes.c_float), ("beam", ctypes.c_int32)]


class _SimHash(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("S", ctypes.c_void_p), ("bits", ctypes.c_void_p), ("en", ctypes.c_void_p),
                ("acrit", ctypes.c_void_p)]


_lib = None


def load_library(path: str):
    """Load a compiled oracle library and declare the return types of its entry points."""
    so = ctypes.CDLL(path)
    so.orc_norm_ppf.restype = ctypes.c_double
    so.orc_norm_ppf.argtypes = [ctypes.c_double]
    so.orc_eta.restype = ctypes.c_double
    so.orc_eta.argtypes = [ctypes.c_int, ctypes.c_int]
    so.orc_dist2_f32.restype = ctypes.c_float
    so.orc_num_threads.restype = ctypes.c_int
    return so


def lib():
    global _lib
    if _lib is None:
        _lib = load_library(build())
    return _lib


@contextlib.contextmanager
def using_library(path: str):
    """Route every call of this module to another compiled copy of the oracle (a test
    that plants a mistake in a copy of the source runs the pins against it)."""
    global _lib
    saved = _lib
    _lib = load_library(path)
    try:
        yield
    finally:
        _lib = saved


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(ctypes.c_int(int(t)))


def num_threads() -> int:
    return int(lib().orc_num_threads())


def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block: 4 counter words, 2 key words -> 4 output words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def projections(seed: int, d: int, L: int, m: int):
    """Random vectors of Sec. 4.2 step (2): A [L, m, d/L] and B [m, d], FP32."""
    A = np.zeros((L, m, d // L), dtype=np.float32)
    B = np.zeros((m, d), dtype=np.float32)
    rc = lib().orc_projections(ctypes.c_uint64(seed), ctypes.c_int(d), ctypes.c_int(L), ctypes.c_int(m), _p(A), _p(B))
    if rc:
        raise ValueError(f"orc_projections failed ({rc})")
    return A, B


def norm_ppf(p: float) -> float:
    return float(lib().orc_norm_ppf(float(p)))


def eta(m: int, mode: int = 0) -> float:
    """sqrt(2 ln m) (mode 0) or the finite-m mean of max_j |g_j| (mode 1)."""
    return float(lib().orc_eta(int(m), int(mode)))


def test_constants(L: int, m: int, eps: float, eta_mode: int = 0):
    """(z_eps, c_eta) in FP32: z = Phi^{-1}(eps), c = sqrt(L) * eta."""
    z = np.float32(norm_ppf(eps))
    c = np.float32(np.sqrt(float(L)) * eta(m, eta_mode))
    return float(z), float(c)


def build_codes(X, nbrs, L: int, m: int, A, B, with_cres: bool = False):
    """Edge records of Sec. 4.2 steps (1) and (3) for every edge of the graph.
    Returns codes [n, R, L+1] int8, enorm [n, R], wreg [n, R] (and, with_cres, also
    cres = sqrt(L) w_res [n, R])."""
    X = _f32(X)
    nbrs = _i32(nbrs)
    n, d = X.shape
    R = nbrs.shape[1]
    codes = np.zeros((n, R, L + 1), dtype=np.int8)
    enorm = np.zeros((n, R), dtype=np.float32)
    wreg = np.zeros((n, R), dtype=np.float32)
    cres = np.zeros((n, R), dtype=np.float32)
    rc = lib().orc_build_codes(_p(X), ctypes.c_int64(n), ctypes.c_int(d), _p(nbrs), ctypes.c_int(R), ctypes.c_int(L),
                               ctypes.c_int(m), _p(_f32(A)), _p(_f32(B)), _p(codes), _p(enorm), _p(wreg), _p(cres))
    if rc:
        raise ValueError(f"orc_build_codes failed ({rc})")
    return (codes, enorm, wreg, cres) if with_cres else (codes, enorm, wreg)


def quantize_scalars(nbrs, bits: int, enorm, wreg, cres):
    """The compact index's edge scalars (orc_quantize_scalars): returns the dequantised
    (enorm, wreg, cres), the per-node steps [n, 3] and the stored integers [n, R, 3]
    (kinds in the order ||e||, w_reg, sqrt(L) w_res)."""
    nbrs = _i32(nbrs)
    n, R = nbrs.shape
    arrs = [np.array(_f32(a), dtype=np.float32, copy=True) for a in (enorm, wreg, cres)]
    steps = np.zeros((n, 3), dtype=np.float32)
    q = np.zeros((n, R, 3), dtype=np.int32)
    rc = lib().orc_quantize_scalars(ctypes.c_int64(n), _p(nbrs), ctypes.c_int(R), ctypes.c_int(bits),
                                    *[_p(a) for a in arrs], _p(steps), _p(q))
    if rc:
        raise ValueError(f"orc_quantize_scalars failed ({rc})")
    return (*arrs, steps, q)


def node_proj(X, L: int, m: int, A, B):
    """Projection table of every row of X: [n, L+1, m] (slot 0 = b_j, slot i = a^i_j)."""
    X = _f32(X)
    n, d = X.shape
    T = np.zeros((n, L + 1, m), dtype=np.float32)
    rc = lib().orc_node_proj(_p(X), ctypes.c_int64(n), ctypes.c_int(d), ctypes.c_int(L), ctypes.c_int(m),
                             _p(_f32(A)), _p(_f32(B)), _p(T))
    if rc:
        raise ValueError(f"orc_node_proj failed ({rc})")
    return T


def dim_permutation(X, nbrs, L: int) -> np.ndarray:
    """Dimension permutation of Appendix D.1: perm[i*d' + t] is the original coordinate
    that becomes coordinate t of subspace i (int32 [d])."""
    X = _f32(X)
    nbrs = _i32(nbrs)
    n, d = X.shape
    perm = np.zeros(d, dtype=np.int32)
    rc = lib().orc_dim_permutation(_p(X), ctypes.c_int64(n), ctypes.c_int(d), _p(nbrs), ctypes.c_int(nbrs.shape[1]),
                                   ctypes.c_int(L), _p(perm))
    if rc:
        raise ValueError(f"orc_dim_permutation failed ({rc})")
    return perm


def dist2_f32(a, b) -> float:
    a = _f32(a)
    b = _f32(b)
    return float(lib().orc_dist2_f32(_p(a), _p(b), ctypes.c_int(a.shape[0])))


class Index:
    """Per-node index data for the oracle's PEOs search, built eagerly or lazily.

    Lazy mode allocates full-size arrays but builds a node's codes and weights only
    when the search first expands it, so a handful of sampled queries can be searched
    on a million-node graph without building every edge.  The eager index also holds
    every node's projection table tv [n, L+1, m] (orc_node_proj), which the search does
    not use: it is there to compare stored tables against."""

    def __init__(self, X, nbrs, entry: int, L: int, m: int, seed: int, lazy: bool = False, perm=None,
                 scalar_bits: int = 32):
        self.X = _f32(X)
        # with a dimension permutation (Appendix D.1) the codes and projection tables live
        # in permuted coordinates: they come from the rows X[:, perm]; exact distances
        # keep using X
        self.perm = None if perm is None else _i32(perm)
        self.Xi = self.X if perm is None else np.ascontiguousarray(self.X[:, self.perm])
        self.nbrs = _i32(nbrs)
        self.entry = int(entry)
        self.n, self.d = self.X.shape
        self.R = self.nbrs.shape[1]
        self.L, self.m, self.seed = L, m, seed
        self.A, self.B = projections(seed, self.d, L, m)
        if lazy:
            self.codes = np.zeros((self.n, self.R, L + 1), dtype=np.int8)
            self.enorm = np.zeros((self.n, self.R), dtype=np.float32)
            self.wreg = np.zeros((self.n, self.R), dtype=np.float32)
            self.cres = np.zeros((self.n, self.R), dtype=np.float32)
            self.tv = None
            self.ready = np.zeros(self.n, dtype=np.uint8)
        else:
            self.codes, self.enorm, self.wreg, self.cres = build_codes(self.Xi, self.nbrs, L, m, self.A, self.B,
                                                                       with_cres=True)
            self.tv = node_proj(self.Xi, L, m, self.A, self.B)
            self.ready = None
        # the compact index (8- or 16-bit edge scalars): the search reads the dequantised values
        self.scalar_bits = scalar_bits
        self.steps = self.qscal = None
        if scalar_bits != 32:
            if lazy:
                raise ValueError("compact scalars need the eager index")
            self.enorm, self.wreg, self.cres, self.steps, self.qscal = quantize_scalars(
                self.nbrs, scalar_bits, self.enorm, self.wreg, self.cres)

    def search(self, Q, k: int, ef: int, routing: int = 1, eps: float = 0.1, eta_mode: int = 0,
               test_mode: int = 0, frame: int = 0, max_expansions: int = 1 << 30,
               trace_cap: int = 0, base=None, rerank=None, entries=None, beam: int = 1):
        """Search with this index's codes; `base` replaces the vectors the search reads
        (e.g. dequantised reduced-precision storage), `rerank` re-ranks R in FP32,
        `entries` gives each query its own entry node, `beam` expands that many nodes
        per iteration."""
        return search(self.X if base is None else base, self.nbrs, self.entry, Q, k, ef, routing=routing, index=self,
                      eps=eps, eta_mode=eta_mode, test_mode=test_mode, frame=frame,
                      max_expansions=max_expansions, trace_cap=trace_cap, rerank=rerank, entries=entries,
                      beam=beam)

    def edge_stats(self, q, v: int, dv: float, delta2: float, eps: float = 0.1, eta_mode: int = 0,
                   frame: int = 0, p: int = -1, test_mode: int = 0):
        """Test statistics (A, H, T, pass, kind) of every out-edge of v for query q, in frame
        T or (frame=1) frame Q, where p = the list's efs-th entry (frame Q only)."""
        if self.ready is not None and not self.ready[v]:
            raise ValueError("edge_stats needs node v built (eager index or after a search touched v)")
        z, c = test_constants(self.L, self.m, eps, eta_mode)
        P = _Params(1, 1, 1, test_mode, frame, 1, 0, z, c, 1)
        outs = [np.zeros(self.R, dtype=np.float32) for _ in range(3)] + [np.zeros(self.R, dtype=np.int32)
                                                                         for _ in range(2)]
        q = _f32(q)
        rc = lib().orc_edge_stats(_p(self.X), _p(self.Xi), ctypes.c_int64(self.n), ctypes.c_int(self.d),
                                  _p(self.nbrs), ctypes.c_int(self.R), ctypes.c_int(self.L), ctypes.c_int(self.m),
                                  _p(self.A), _p(self.B), _p(self.codes), _p(self.enorm), _p(self.wreg),
                                  _p(self.cres), _p(q), _p(self.perm),
                                  ctypes.c_int32(v), ctypes.c_float(dv), ctypes.c_float(delta2), ctypes.c_int32(p),
                                  ctypes.byref(P),
                                  *[_p(o) for o in outs])
        if rc:
            raise ValueError(f"orc_edge_stats failed ({rc})")
        return dict(A=outs[0], H=outs[1], T=outs[2], passed=outs[3], kind=outs[4])


def quantize(X, dtype: str):
    """Reduced-precision storage: dtype "bf16" (round to nearest even) or "e4m3" (per-row
    scale max|x|/448, nearest even, saturating).  Returns (codes, scales, dequantised FP32)."""
    X = _f32(X)
    n, d = X.shape
    code = {"bf16": 1, "e4m3": 2}[dtype]
    codes = np.zeros((n, d), dtype=np.uint16 if code == 1 else np.uint8)
    scales = np.zeros(n, dtype=np.float32)
    deq = np.zeros((n, d), dtype=np.float32)
    rc = lib().orc_quantize(_p(X), ctypes.c_int64(n), ctypes.c_int(d), ctypes.c_int(code), _p(codes), _p(scales),
                            _p(deq))
    if rc:
        raise ValueError(f"orc_quantize failed ({rc})")
    return codes, scales, deq


def search(X, nbrs, entry: int, Q, k: int, ef: int, routing: int = 0, index: Index | None = None,
           eps: float = 0.1, eta_mode: int = 0, test_mode: int = 0, frame: int = 0,
           max_expansions: int = 1 << 30, trace_cap: int = 0, rerank=None, entries=None,
           simhash: SimHash | None = None, beam: int = 1):
    """Algorithm 1 with plain routing (routing=0) or the PEOs test (routing=1).

    X is the base the search reads (FP32, or the dequantised values of a reduced-precision
    store); `rerank` (optional FP32 base) recomputes the distances of the final list R
    exactly and sorts it again before the top k are taken.  `entries` (optional, one per
    query) replaces the single entry node (a hierarchical entry, hier_entries).
    routing=2 is the SimHash test (Sec. 3.1) with the data of `simhash`.  `beam` = W nodes
    expanded per iteration (1..8; W = 1 is Algorithm 1's pop-one loop).
    Returns dict(ids [nq,k], dists [nq,k] (squared l2, FP32), counters [nq,10],
    trace_v/trace_dv/trace_d2 [nq, trace_cap] when trace_cap > 0)."""
    X = _f32(X)
    nbrs = _i32(nbrs)
    Q = _f32(Q).reshape(-1, X.shape[1])
    n, d = X.shape
    nq = Q.shape[0]
    R = nbrs.shape[1]
    if routing == 1:
        if index is None:
            raise ValueError("PEOs routing needs an Index")
        L, m = index.L, index.m
        z, c = test_constants(L, m, eps, eta_mode)
        codes, enorm, wreg, cres, ready, A, B = (index.codes, index.enorm, index.wreg, index.cres, index.ready,
                                                 index.A, index.B)
    else:
        L, m, z, c = 1, 2, 0.0, 0.0
        codes = enorm = wreg = cres = ready = A = B = None
    sh = None
    if routing == 2:
        if simhash is None:
            raise ValueError("SimHash routing needs a SimHash")
        sh = simhash.c(eps)
    P = _Params(k, ef, routing, test_mode, frame, max_expansions, trace_cap, z, c, beam)
    ids = np.zeros((nq, k), dtype=np.int32)
    dists = np.zeros((nq, k), dtype=np.float32)
    cnt = np.zeros((nq, N_COUNTERS), dtype=np.int64)
    tr = [None, None, None]
    if trace_cap > 0:
        tr = [np.full((nq, trace_cap), -1, dtype=np.int32), np.zeros((nq, trace_cap), dtype=np.float32),
              np.zeros((nq, trace_cap), dtype=np.float32)]
    rc = lib().orc_search(_p(X), ctypes.c_int64(n), ctypes.c_int(d), _p(nbrs), ctypes.c_int(R), ctypes.c_int32(entry),
                          _p(codes), _p(enorm), _p(wreg), _p(cres), _p(ready), _p(A), _p(B),
                          ctypes.c_int(L),
                          ctypes.c_int(m), _p(Q), ctypes.c_int64(nq), ctypes.byref(P), _p(ids), _p(dists), _p(cnt),
                          _p(tr[0]), _p(tr[1]), _p(tr[2]), _p(None if rerank is None else _f32(rerank)),
                          _p(index.Xi if index is not None else None),
                          _p(index.perm if index is not None and routing == 1 else None),
                          _p(None if entries is None else _i32(entries)),
                          ctypes.byref(sh) if sh is not None else None)
    if rc:
        raise ValueError(f"orc_search failed ({rc})")
    out = dict(ids=ids, dists=dists, counters=cnt)
    if trace_cap > 0:
        out.update(trace_v=tr[0], trace_dv=tr[1], trace_d2=tr[2])
    return out


def simhash_acrit(K: int, eps: float) -> np.ndarray:
    """Thresholds of the SimHash test: pass iff A <= acrit[#Col] (FP32 [K+1])."""
    out = np.zeros(K + 1, dtype=np.float32)
    rc = lib().orc_simhash_acrit(ctypes.c_int(K), ctypes.c_double(eps), _p(out))
    if rc:
        raise ValueError(f"orc_simhash_acrit failed ({rc})")
    return out


class SimHash:
    """Per-edge SimHash data of the residual remedy (Sec. 3.1): K sign bits of S_i . e
    and ||e|| per edge; S = the K x d random matrix B of projections(seed, d, 1, K)."""

    def __init__(self, X, nbrs, K: int, seed: int):
        X = _f32(X)
        nbrs = _i32(nbrs)
        n, d = X.shape
        R = nbrs.shape[1]
        self.K, self.seed = K, seed
        self.S = np.ascontiguousarray(projections(seed, d, 1, K)[1])
        self.bits = np.zeros((n, R, K // 64), dtype=np.uint64)
        self.en = np.zeros((n, R), dtype=np.float32)
        rc = lib().orc_simhash_build(_p(X), ctypes.c_int64(n), ctypes.c_int(d), _p(nbrs), ctypes.c_int(R),
                                     ctypes.c_int(K), _p(self.S), _p(self.bits), _p(self.en))
        if rc:
            raise ValueError(f"orc_simhash_build failed ({rc})")

    def c(self, eps: float):
        self.acrit = simhash_acrit(self.K, eps)
        return _SimHash(self.K, self.S.ctypes.data, self.bits.ctypes.data, self.en.ctypes.data,
                        self.acrit.ctypes.data)


def greedy_layer(X, Q, ids, nbrs, cur):
    """One upper layer of the hierarchical entry: greedy descent with a list of one.
    ids [n_l] base rows of the layer's nodes, nbrs [n_l, R_l] local ids, cur [nq] local
    start nodes.  Returns (local end nodes [nq], hops [nq])."""
    X = _f32(X)
    Q = _f32(Q).reshape(-1, X.shape[1])
    ids = _i32(ids)
    nbrs = _i32(nbrs)
    cur = _i32(cur).copy()
    hops = np.zeros(len(cur), dtype=np.int64)
    rc = lib().orc_greedy_layer(_p(X), ctypes.c_int(X.shape[1]), _p(Q), ctypes.c_int64(Q.shape[0]),
                                ctypes.c_int64(len(ids)), ctypes.c_int(nbrs.shape[1]), _p(ids), _p(nbrs), _p(cur),
                                _p(hops))
    if rc:
        raise ValueError(f"orc_greedy_layer failed ({rc})")
    return cur, hops


def hier_entries(X, Q, layers, top_entry: int):
    """Entry node of every query: greedy descent from `top_entry` (a local id of the top
    layer) through `layers` (ordered top first; each a dict with ids [n_l], nbrs
    [n_l, R_l] in local ids and, except for the lowest upper layer, down [n_l] = the
    node's local id in the layer below).  Returns (base ids [nq], total hops [nq])."""
    Q = _f32(Q).reshape(-1, _f32(X).shape[1])
    cur = np.full(Q.shape[0], int(top_entry), dtype=np.int32)
    hops = np.zeros(Q.shape[0], dtype=np.int64)
    for i, lay in enumerate(layers):
        cur, h = greedy_layer(X, Q, lay["ids"], lay["nbrs"], cur)
        hops += h
        if i + 1 < len(layers):
            cur = np.asarray(lay["down"], dtype=np.int32)[cur]
    return np.asarray(layers[-1]["ids"], dtype=np.int32)[cur], hops


def knn_f64(X, Q, k: int):
    """Exact K-NN by brute force, FP64 distances, ties by id."""
    X = _f32(X)
    Q = _f32(Q).reshape(-1, X.shape[1])
    nq = Q.shape[0]
    ids = np.zeros((nq, k), dtype=np.int32)
    dists = np.zeros((nq, k), dtype=np.float64)
    rc = lib().orc_knn_f64(_p(X), ctypes.c_int64(X.shape[0]), ctypes.c_int(X.shape[1]), _p(Q), ctypes.c_int64(nq),
                           ctypes.c_int(k), _p(ids), _p(dists))
    if rc:
        raise ValueError(f"orc_knn_f64 failed ({rc})")
    return ids, dists


def build_graph(X, R: int, Kc: int | None = None, ucap: int | None = None):
    """Exact-kNN + relative-neighbourhood graph with reverse edges and connectivity
    repair (FP64).  O(n^2 d): small n only.  Returns (nbrs [n, R] int32, entry)."""
    X = _f32(X)
    n = X.shape[0]
    Kc = 2 * R if Kc is None else Kc
    ucap = 4 * R if ucap is None else ucap
    nbrs = np.full((n, R), -1, dtype=np.int32)
    entry = ctypes.c_int32(0)
    rc = lib().orc_build_graph(_p(X), ctypes.c_int64(n), ctypes.c_int(X.shape[1]), ctypes.c_int(R), ctypes.c_int(Kc),
                               ctypes.c_int(ucap), _p(nbrs), ctypes.byref(entry))
    if rc:
        raise ValueError(f"orc_build_graph failed ({rc})")
    return nbrs, int(entry.value)


def recall_at_k(found, truth) -> float:
    """Mean |found_i ∩ truth_i| / k over queries."""
    found = np.asarray(found)
    truth = np.asarray(truth)
    k = truth.shape[1]
    hits = sum(len(set(f[:k].tolist()) & set(t.tolist())) for f, t in zip(found, truth))
    return hits / float(truth.shape[0] * k)
