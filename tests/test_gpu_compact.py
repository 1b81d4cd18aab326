"""GPU parity of the compact index (edge scalars in 16 or 8 bits, per-node linear steps;
the paper's standard 16-bit form and its PEOs (Compact), Sec. 4.3 and Sec. 6.4) against
the oracle on the same seeded inputs: the records' steps, integers, ids and codes bit for
bit, the node terms (kept in FP32, from the stored weights) and the searches within the
bars of tests/parity.py."""
import numpy as np
import pytest
import torch

import oracle
import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


@pytest.fixture(scope="module", params=[16, 8])
def env(request, P, sift20k):
    bits = request.param
    case = sift20k
    cfg = case.cfg
    X = torch.from_numpy(case.X).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    codes = P.build_codes(G, X, cfg.L, cfg.m, cfg.proj_seed, scalar_bits=bits)
    ix = oracle.Index(case.X, case.nbrs, case.entry, cfg.L, cfg.m, cfg.proj_seed, scalar_bits=bits)
    return bits, case, X, G, codes, ix


def test_records(P, env):
    bits, case, X, G, codes, ix = env
    arr = codes.arrays()
    assert codes.info()["scalar_bits"] == bits
    assert arr["record_stride"] == {16: 800, 8: 672}[bits]  # R = 32, L = 8, m = 16 (FP32 scalars: 896)
    assert np.array_equal(arr["ids"], case.nbrs)
    assert np.array_equal(arr["codes"], ix.codes)
    assert np.array_equal(arr["steps"].view(np.uint32), ix.steps.view(np.uint32))
    assert np.array_equal(arr["q"], ix.qscal)
    for name in ("enorm", "wreg", "cres"):
        assert np.array_equal(arr[name].view(np.uint32), getattr(ix, name).view(np.uint32)), name
    # the node term comes from the stored (quantised) weights
    sv_ref, sv_scale = parity.node_terms(ix.tv, ix.codes, ix.wreg, ix.cres)
    assert np.all(parity.close(arr["sv"], sv_ref, sv_scale))


@pytest.mark.parametrize("eps", [0.1, 0.3])
@pytest.mark.parametrize("ef", [16, 64])
def test_search_integer_data(P, env, eps, ef):
    bits, case, X, G, codes, ix = env
    Q = torch.from_numpy(case.Q).cuda()
    ids, dists, cnt = P.search(G, codes, X, Q, 10, ef, eps=eps, routing=1, counters=True)
    want = ix.search(case.Q, 10, ef, routing=1, eps=eps)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids)
    parity.counters_parity(cnt.cpu().numpy(), want["counters"], 0)


def test_forms_outside_the_compact_search_are_rejected(P, env):
    bits, case, X, G, codes, ix = env
    Q = torch.from_numpy(case.Q).cuda()
    with pytest.raises(P.PeosError, match="in frame T"):
        P.search(G, codes, X, Q, 10, 32, routing=1, frame=1)
    with pytest.raises(P.PeosError, match="FP32 scalars"):
        P.edge_stats(codes, Q[0], 0, 1.0, 2.0)
    with pytest.raises(P.PeosError, match="scalar_bits"):
        P.build_codes(G, X, 8, 16, 1, scalar_bits=12)
    # plain routing ignores the codes' scalars
    a = P.search(G, codes, X, Q, 10, 32, routing=0)[0].cpu().numpy()
    b = P.search(G, None, X, Q, 10, 32, routing=0)[0].cpu().numpy()
    assert np.array_equal(a, b)


def test_index_file_roundtrip(P, env, tmp_path):
    bits, case, X, G, codes, ix = env
    path = str(tmp_path / f"compact{bits}.idx")
    codes.save(path)
    back = P.load_codes(path)
    assert back.info()["scalar_bits"] == bits
    Q = torch.from_numpy(case.Q).cuda()
    x = P.search(G, codes, X, Q, 10, 32, routing=1)
    G2 = back.graph()
    assert np.array_equal(G2.nbrs.cpu().numpy(), case.nbrs) and G2.entry == case.entry
    y = P.search(G2, back, X, Q, 10, 32, routing=1)
    assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1])


def test_reduced_precision_storage(P, env):
    """BF16 holds the integers 0..255 exactly, so BF16 storage gives the FP32 results bit
    for bit; FP8-E4M3 storage with the FP32 re-rank follows the oracle's search over the
    dequantised rows."""
    bits, case, X, G, codes, ix = env
    Q = torch.from_numpy(case.Q).cuda()
    a = P.search(G, codes, X, Q, 10, 48, eps=0.2, routing=1)
    b = P.search(G, codes, P.quantize(X, "bf16"), Q, 10, 48, eps=0.2, routing=1)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1].view(torch.int32), b[1].view(torch.int32))
    _, _, deq = oracle.quantize(case.X, "e4m3")
    ids, dists, _ = P.search(G, codes, P.quantize(X, "e4m3"), Q, 10, 64, eps=0.2, routing=1, rerank=X)
    want = ix.search(case.Q, 10, 64, routing=1, eps=0.2, base=deq, rerank=case.X)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids)


@pytest.mark.parametrize("bits", [16, 8])
def test_two_edges_per_lane_float_data(P, bits):
    """R = 48 (two edges per lane), d = 100, L = 10 on GloVe-shaped unit vectors: the
    compact records match the oracle's bit for bit and the searches meet the bars."""
    import workloads
    from workloads.graph import build_graph
    cfg = workloads.scaled(workloads.CONFIGS["glove"], 6000, 150)
    X, Q = workloads.generate(cfg)
    nbrs, entry = build_graph(X, 48)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    G = P.Graph.from_numpy(nbrs, entry)
    codes = P.build_codes(G, Xt, 10, 16, 5, scalar_bits=bits)
    ix = oracle.Index(X, nbrs, entry, 10, 16, 5, scalar_bits=bits)
    arr = codes.arrays()
    assert arr["record_stride"] == {16: 1184, 8: 992}[bits]
    assert np.array_equal(arr["steps"].view(np.uint32), ix.steps.view(np.uint32))
    assert np.array_equal(arr["q"], ix.qscal)
    gt, _ = oracle.knn_f64(X, Q, 10)
    ids, dists, _ = P.search(G, codes, Xt, Qt, 10, 64, routing=1, eps=0.2)
    want = ix.search(Q, 10, 64, routing=1, eps=0.2)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=gt)
