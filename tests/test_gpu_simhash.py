"""GPU parity of the SimHash routing test (Sec. 3.1, Lemma 4.1, the baseline the paper
compares PEOs with) against the oracle on the same seeded inputs: the per-edge bits and
norms bit for bit, the node tables S_i . v (the library's own) within 1e-5 relative of their
FP64 values, and the searches within the bars of tests/parity.py (the library takes the bits
of q - v from S_i . q - S_i . v, the oracle from S_i . (q - v))."""
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


@pytest.fixture(scope="module", params=[64, 128])
def env(request, P, sift20k):
    K = request.param
    case = sift20k
    X = torch.from_numpy(case.X).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    codes = P.build_simhash(G, X, K, seed=31)
    sh = oracle.SimHash(case.X, case.nbrs, K, seed=31)
    return case, X, G, codes, sh


def test_build_bitwise(P, env):
    case, X, G, codes, sh = env
    arr = codes.arrays()
    assert np.array_equal(arr["ids"], case.nbrs)
    assert np.array_equal(arr["S"], sh.S)
    assert np.array_equal(arr["bits"], sh.bits)
    assert np.array_equal(arr["en"].view(np.uint32), sh.en.view(np.uint32))
    X64 = case.X.astype(np.float64)
    tv = X64 @ sh.S.astype(np.float64).T
    scale = np.linalg.norm(X64, axis=1)[:, None] * np.linalg.norm(sh.S.astype(np.float64), axis=1)[None, :]
    assert np.all(parity.close(arr["tv"], tv, scale))


@pytest.mark.parametrize("eps", [0.1, 0.3])
@pytest.mark.parametrize("ef", [16, 64])
def test_search_integer_data(P, env, eps, ef):
    case, X, G, codes, sh = env
    Q = torch.from_numpy(case.Q).cuda()
    ids, dists, cnt = P.search(G, codes, X, Q, 10, ef, eps=eps, routing=2, counters=True)
    want = oracle.search(case.X, case.nbrs, case.entry, case.Q, 10, ef, routing=2, simhash=sh, eps=eps)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids)
    c = cnt.cpu().numpy()
    parity.counters_parity(c, want["counters"], 0)
    assert np.all(c[:, 9] == 0)
    # the test screens: fewer exact distances than plain routing at the same efs
    plain = P.search(G, None, X, Q, 10, ef, routing=0, counters=True)[2].cpu().numpy()
    assert c[:, 7].sum() < plain[:, 7].sum()


def test_modes_and_rejections(P, env, sift20k):
    case, X, G, codes, sh = env
    Q = torch.from_numpy(case.Q).cuda()
    a = P.search(G, codes, X, Q, 10, 32, routing=2, test_mode=2)[0].cpu().numpy()
    b = P.search(G, None, X, Q, 10, 32, routing=0)[0].cpu().numpy()
    assert np.array_equal(a, b)  # every neighbour passes: plain routing
    with pytest.raises(P.PeosError, match="SimHash codes"):
        P.search(G, None, X, Q, 10, 32, routing=2)
    pe = P.build_codes(G, X, 8, 16, 1)
    with pytest.raises(P.PeosError, match="SimHash codes"):
        P.search(G, pe, X, Q, 10, 32, routing=2)
    with pytest.raises(P.PeosError, match="PEOs codes"):
        P.search(G, codes, X, Q, 10, 32, routing=1)
    with pytest.raises(P.PeosError, match="FP32"):
        P.search(G, codes, P.quantize(X, "bf16"), Q, 10, 32, routing=2)
    with pytest.raises(P.PeosError, match="K must be"):
        P.build_simhash(G, X, 96, 1)
    with pytest.raises(P.PeosError, match="PEOs codes"):
        P.edge_stats(codes, Q[0], 0, 1.0, 2.0)
