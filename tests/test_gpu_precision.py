"""GPU parity of the precision form: reduced-precision storage of the base (BF16, or
FP8-E4M3 with one scale per row), FP32 accumulation, and the exact FP32 re-rank of the
final lists, through the C ABI, against the oracle on the same seeded inputs.

Bars: quantised codes and scales bit-exact; on the stored rows the search results
follow the oracle's search over the dequantised rows (top-k ids identical on >= 99% of
queries, distances within 1e-5 relative, recall within 0.3 points; bit-exact where the
arithmetic is exact: integer data in BF16 with plain routing); the re-ranked results
follow the oracle's re-rank the same way."""
import numpy as np
import pytest
import torch

import oracle
import parity
import workloads
from conftest import Case

pytestmark = pytest.mark.gpu

_cases = {}


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


def glove_case():
    """GloVe-shaped angular data (d=100, R=48, L=10, m=16) at 20,000 points, 300 queries."""
    if "glove" not in _cases:
        _cases["glove"] = Case(workloads.scaled(workloads.CONFIGS["glove"], 20_000, 300))
    return _cases["glove"]


def sift_case():
    if "sift" not in _cases:
        _cases["sift"] = Case(workloads.scaled(workloads.CONFIGS["sift"], 20_000, 200))
    return _cases["sift"]


class Dev:
    def __init__(self, P, case):
        self.X = torch.from_numpy(case.X).cuda()
        self.Q = torch.from_numpy(case.Q).cuda()
        self.G = P.Graph.from_numpy(case.nbrs, case.entry)
        self.codes = P.build_codes(self.G, self.X, case.cfg.L, case.cfg.m, case.cfg.proj_seed)


_devs = {}


def dev(P, case):
    if id(case) not in _devs:
        _devs[id(case)] = Dev(P, case)
    return _devs[id(case)]


def _special_rows(d):
    rng = np.random.default_rng(5)
    X = (rng.standard_normal((300, d)) * np.exp(3 * rng.standard_normal((300, 1)))).astype(np.float32)
    X[0] = 0.0                      # all-zero row: scale 1
    X[1] = 0.0
    X[1, 3] = -1e-30                # one tiny negative entry
    X[2, :] = 448.0                 # already at the top of the range
    X[3] = np.linspace(-1e-3, 1e5, d, dtype=np.float32)  # wide dynamic range: subnormal codes
    return X


def _compare(gpu_ids, gpu_d, orc, gt_ids, exact=False):
    parity.search_parity(gpu_ids, gpu_d, orc, gt=gt_ids, exact=exact)


@pytest.mark.parametrize("dtype", ["bf16", "e4m3"])
@pytest.mark.parametrize("d", [100, 128, 960])
def test_quantize_bitwise(P, dtype, d):
    X = _special_rows(d)
    st = P.quantize(torch.from_numpy(X).cuda(), dtype)
    torch.cuda.synchronize()
    codes, scales, _ = oracle.quantize(X, dtype)
    if dtype == "bf16":
        got = st.data.view(torch.int16).cpu().numpy().view(np.uint16)
        assert st.scales is None
    else:
        got = st.data.cpu().numpy()
        assert np.array_equal(st.scales.cpu().numpy().view(np.uint32), scales.view(np.uint32))
    assert np.array_equal(got, codes)


@pytest.mark.parametrize("dtype", ["bf16", "e4m3"])
@pytest.mark.parametrize("routing", [0, 1])
def test_search_on_stored_rows(P, dtype, routing):
    case = glove_case()
    D = dev(P, case)
    cfg = case.cfg
    st = P.quantize(D.X, dtype)
    _, _, deq = oracle.quantize(case.X, dtype)
    ef = 64
    ids, dists, cnt = P.search(D.G, D.codes, st, D.Q, cfg.k, ef, eps=cfg.eps, routing=routing, counters=True)
    orc = case.index.search(case.Q, cfg.k, ef, routing=routing, eps=cfg.eps, base=deq)
    _compare(ids.cpu().numpy(), dists.cpu().numpy(), orc, case.gt_ids)
    assert np.all(cnt.cpu().numpy()[:, 9] == 0)


@pytest.mark.parametrize("dtype", ["bf16", "e4m3"])
@pytest.mark.parametrize("routing", [0, 1])
def test_rerank_parity(P, dtype, routing):
    case = glove_case()
    D = dev(P, case)
    cfg = case.cfg
    st = P.quantize(D.X, dtype)
    _, _, deq = oracle.quantize(case.X, dtype)
    for ef in (16, 64, 300):
        ids, dists, _ = P.search(D.G, D.codes, st, D.Q, cfg.k, ef, eps=cfg.eps, routing=routing, rerank=D.X)
        orc = case.index.search(case.Q, cfg.k, ef, routing=routing, eps=cfg.eps, base=deq, rerank=case.X)
        _compare(ids.cpu().numpy(), dists.cpu().numpy(), orc, case.gt_ids)


def test_bf16_of_integer_data_is_exact(P):
    """Integers 0..255 are exact in BF16, so BF16 storage of SIFT-shaped data gives the FP32
    results bit for bit, and both meet the bars against the oracle (plain routing: bit for bit)."""
    case = sift_case()
    D = dev(P, case)
    st = P.quantize(D.X, "bf16")
    for routing in (0, 1):
        a = P.search(D.G, D.codes, D.X, D.Q, 10, 48, eps=0.2, routing=routing)
        b = P.search(D.G, D.codes, st, D.Q, 10, 48, eps=0.2, routing=routing)
        c = P.search(D.G, D.codes, st, D.Q, 10, 48, eps=0.2, routing=routing, rerank=D.X)
        for x, y in ((a, b), (a, c)):
            assert torch.equal(x[0], y[0]) and torch.equal(x[1].view(torch.int32), y[1].view(torch.int32))
        orc = case.index.search(case.Q, 10, 48, routing=routing, eps=0.2)
        _compare(b[0].cpu().numpy(), b[1].cpu().numpy(), orc, case.gt_ids, exact=routing == 0)


def test_e4m3_rerank_integer_data_exact_distances(P):
    """On integer data the FP32 re-rank distances are exact: wherever the ids agree with the
    oracle's, the distances agree bit for bit."""
    case = sift_case()
    D = dev(P, case)
    st = P.quantize(D.X, "e4m3")
    _, _, deq = oracle.quantize(case.X, "e4m3")
    ids, dists, _ = P.search(D.G, D.codes, st, D.Q, 10, 64, eps=0.2, routing=1, rerank=D.X)
    orc = case.index.search(case.Q, 10, 64, routing=1, eps=0.2, base=deq, rerank=case.X)
    ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
    parity.search_parity(ids, dists, orc)
    same = np.all(ids == orc["ids"], axis=1)
    assert np.array_equal(dists[same].view(np.uint32), orc["dists"][same].view(np.uint32))
    # every re-ranked distance is the exact distance of its id
    exact = ((case.Q[:, None, :].astype(np.float64) - case.X[ids].astype(np.float64)) ** 2).sum(-1)
    assert np.array_equal(dists, exact.astype(np.float32))


def test_rerank_of_fp32_search_changes_nothing(P):
    """Re-ranking an FP32 search with its own base recomputes the same distances (same
    per-lane sums and reduction tree), so ids and distances are unchanged bit for bit."""
    case = glove_case()
    D = dev(P, case)
    for routing in (0, 1):
        a = P.search(D.G, D.codes, D.X, D.Q, 10, 40, eps=0.2, routing=routing)
        b = P.search(D.G, D.codes, D.X, D.Q, 10, 40, eps=0.2, routing=routing, rerank=D.X)
        assert torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))


def test_stored_rows_through_other_entry_points(P):
    case = glove_case()
    D = dev(P, case)
    st = P.quantize(D.X, "e4m3")
    a = P.search(D.G, D.codes, st, D.Q, 10, 64, eps=0.2, routing=1)
    b = P.search_noalloc(D.G, D.codes, st, D.Q, 10, 64, eps=0.2, routing=1)
    c = P.search_host(D.G, D.codes, st, case.Q, 10, 64, eps=0.2, routing=1)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
    assert np.array_equal(a[0].cpu().numpy(), c[0]) and np.array_equal(a[1].cpu().numpy(), c[1])


def test_rerank_short_lists(P):
    """Lists shorter than k (a graph where the entry reaches few nodes) and k = ef."""
    rng = np.random.default_rng(3)
    n, d = 50, 16
    X = rng.standard_normal((n, d)).astype(np.float32)
    nbrs = np.full((n, 4), -1, dtype=np.int32)
    nbrs[0, :3] = [1, 2, 3]
    nbrs[2, 0] = 4
    Q = rng.standard_normal((7, d)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    G = P.Graph.from_numpy(nbrs, 0)
    st = P.quantize(Xd, "e4m3")
    _, _, deq = oracle.quantize(X, "e4m3")
    for k, ef in ((10, 10), (3, 8), (1, 1)):
        ids, dists, _ = P.search(G, None, st, torch.from_numpy(Q).cuda(), k, ef, routing=0, rerank=Xd)
        orc = oracle.search(deq, nbrs, 0, Q, k, ef, routing=0, rerank=X)
        ids, dists = ids.cpu().numpy(), dists.cpu().numpy()
        assert np.array_equal(ids, orc["ids"])
        fin = np.isfinite(orc["dists"])
        assert np.array_equal(np.isfinite(dists), fin)
        assert np.allclose(dists[fin], orc["dists"][fin], rtol=1e-5, atol=0)


def test_precision_invalid_arguments(P):
    case = glove_case()
    D = dev(P, case)
    st = P.quantize(D.X, "e4m3")
    bf = P.quantize(D.X, "bf16")
    with pytest.raises(TypeError):
        P.search(D.G, D.codes, P.StoredBase(st.data, None, "e4m3"), D.Q, 10, 16)
    with pytest.raises(P.PeosError, match="rerank"):
        P.search(D.G, D.codes, st, D.Q, 10, 16, rerank=D.X[:100].contiguous())
    import ctypes
    from paper_2402_11354_gb300 import peos as B
    lib = B.load()
    g = D.G.c()
    Mq = B._matrix(D.Q)
    prm = B._params(10, 16, 0.2, 1, 0, 0, 0, 0, 0)
    out = torch.empty((D.Q.shape[0], 10), dtype=torch.int32, device="cuda")
    outd = torch.empty((D.Q.shape[0], 10), dtype=torch.float32, device="cuda")

    def call(Mb, Mr=None, Mq=Mq):
        return lib.peos_search_rerank(ctypes.byref(g), D.codes.handle, ctypes.byref(Mb),
                                      ctypes.byref(Mr) if Mr is not None else None, ctypes.byref(Mq),
                                      ctypes.byref(prm), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(outd.data_ptr()), None, B._stream(None))

    n, d = D.X.shape
    no_scales = B._Matrix(st.data.data_ptr(), None, n, d, B.FP8E4M3)
    assert call(no_scales) == 1
    bf_scaled = B._Matrix(bf.data.data_ptr(), st.scales.data_ptr(), n, d, B.BF16)
    assert call(bf_scaled) == 1
    good = B._Matrix(st.data.data_ptr(), st.scales.data_ptr(), n, d, B.FP8E4M3)
    bad_q = B._Matrix(bf.data.data_ptr(), None, n, d, B.BF16)
    assert call(good, Mq=bad_q) == 1                      # queries must be FP32
    assert call(good, Mr=B._matrix(D.X[:100])) == 1       # re-rank base of another shape
    assert call(good, Mr=bad_q) == 1                      # re-rank base must be FP32
    assert call(good, Mr=B._matrix(D.X)) == 0
    torch.cuda.synchronize()
    with pytest.raises(TypeError):
        P.build_codes(D.G, bf.data, 10, 16, 1)            # codes come from the FP32 rows
    M = B._Matrix(bf.data.data_ptr(), None, n, d, B.BF16)
    h = ctypes.c_void_p()
    assert lib.peos_build_codes(ctypes.byref(g), ctypes.byref(M), 10, 16, ctypes.c_uint64(1), B._stream(None),
                                ctypes.byref(h)) == 1
    with pytest.raises(ValueError):
        P.quantize(D.X, "int4")
    assert lib.peos_quantize(ctypes.byref(B._matrix(D.X)), 0, ctypes.c_void_p(st.data.data_ptr()), None,
                             B._stream(None)) == 1
