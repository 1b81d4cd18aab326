"""GPU parity of the PEOs test in the paper-literal frame Q (table of q' = q / ||q|| once
per query, A_r of Eq. A_r) against the oracle's frame Q on the same seeded inputs, within
the bars of tests/parity.py.  The library forms v.q and p.q from the search's distances
and squared norms; the oracle takes plain dot products."""
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


@pytest.fixture(scope="module")
def env(P, sift20k):
    case = sift20k
    X = torch.from_numpy(case.X).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    codes = P.build_codes(G, X, case.cfg.L, case.cfg.m, case.cfg.proj_seed)
    return case, X, G, codes


@pytest.mark.parametrize("ef", [16, 64, 200])
@pytest.mark.parametrize("eps", [0.1, 0.2])
def test_frame_q_search(P, env, ef, eps):
    case, X, G, codes = env
    Q = torch.from_numpy(case.Q).cuda()
    ids, dists, cnt = P.search(G, codes, X, Q, 10, ef, eps=eps, routing=1, frame=1, counters=True)
    want = case.index.search(case.Q, 10, ef, routing=1, eps=eps, frame=1)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids)
    c = cnt.cpu().numpy()
    parity.counters_parity(c, want["counters"], 0)
    assert np.all(c[:, 9] == 0) and c[:, 5].sum() > 0


def test_frame_q_with_permuted_codes(P, env):
    case, X, G, codes = env
    cfg = case.cfg
    perm = oracle.dim_permutation(case.X, case.nbrs, cfg.L)
    ix = oracle.Index(case.X, case.nbrs, case.entry, cfg.L, cfg.m, cfg.proj_seed, perm=perm)
    pc = P.build_codes(G, X, cfg.L, cfg.m, cfg.proj_seed, perm=torch.from_numpy(perm).cuda())
    ids, dists, _ = P.search(G, pc, X, torch.from_numpy(case.Q).cuda(), 10, 48, eps=0.2, routing=1, frame=1)
    want = ix.search(case.Q, 10, 48, routing=1, eps=0.2, frame=1)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids)


def test_frame_q_modes_and_checks(P, env):
    case, X, G, codes = env
    Q = torch.from_numpy(case.Q).cuda()
    a = P.search(G, codes, X, Q, 10, 32, routing=1, frame=1, test_mode=2)[0].cpu().numpy()
    b = P.search(G, None, X, Q, 10, 32, routing=0)[0].cpu().numpy()
    assert np.array_equal(a, b)
    with pytest.raises(P.PeosError, match="frame"):
        P.search(G, codes, X, Q, 10, 32, routing=0, frame=1)
    with pytest.raises(P.PeosError, match="frame"):
        P.search(G, codes, X, Q, 10, 32, routing=1, frame=2)
    with pytest.raises(P.PeosError, match="FP32"):
        P.search(G, codes, P.quantize(X, "bf16"), Q, 10, 32, routing=1, frame=1)
    assert codes.info()["norms"]


@pytest.mark.parametrize("ef", [16, 64])
def test_quantile_table(P, env, ef):
    """test_mode 3: frame Q with the quantile table (variance at its bin's upper edge)."""
    case, X, G, codes = env
    Q = torch.from_numpy(case.Q).cuda()
    ids, dists, cnt = P.search(G, codes, X, Q, 10, ef, eps=0.2, routing=1, frame=1, test_mode=3, counters=True)
    want = case.index.search(case.Q, 10, ef, routing=1, eps=0.2, frame=1, test_mode=3)
    parity.search_parity(ids.cpu().numpy(), dists.cpu().numpy(), want, gt=case.gt_ids)
    parity.counters_parity(cnt.cpu().numpy(), want["counters"], 0)
    with pytest.raises(P.PeosError, match="quantile table"):
        P.search(G, codes, X, Q, 10, ef, routing=1, frame=0, test_mode=3)
