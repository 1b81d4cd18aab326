"""GPU tests of the tensor-core brute force (peos_knn_tensor: tcgen05 BF16 scores, exact
FP32 distances of the candidates) against the exact FFMA brute force and the oracle's
FP64 brute force.

Integer-valued data below 256 make the BF16 scores exact, so ids and distances must
equal the exact brute force bit for bit; on float data the ranking may differ only at
near-ties, which the candidates' slack absorbs."""
import numpy as np
import pytest
import torch

import oracle
import workloads
from conftest import get_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


@pytest.mark.parametrize("n,nq,k", [(1000, 1, 1), (3000, 129, 10), (20_000, 200, 64), (5000, 70, 96)])
def test_integer_data_exact(P, n, nq, k):
    cfg = workloads.scaled(workloads.CONFIGS["sift"], n, nq)
    X, Q = workloads.generate(cfg)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    ti, td = P.knn_tensor(Xt, Qt, k)
    ei, ed = P.knn_bruteforce(Xt, Qt, k)
    assert torch.equal(ti, ei)
    assert torch.equal(td, ed)


@pytest.mark.parametrize("name,d", [("glove", 100), ("gist", 960)])
def test_float_data_matches_fp64(P, name, d):
    cfg = workloads.scaled(workloads.CONFIGS[name], 5000, 150)
    X, Q = workloads.generate(cfg)
    assert X.shape[1] == d
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    ti, td = P.knn_tensor(Xt, Qt, 10)
    gi, gd = oracle.knn_f64(X, Q, 10)
    ti, td = ti.cpu().numpy(), td.cpu().numpy()
    assert oracle.recall_at_k(ti, gi) >= 0.999
    # distances are exact FP32 sums of the returned rows
    exact = ((Q[:, None, :].astype(np.float64) - X[ti].astype(np.float64)) ** 2).sum(-1)
    assert np.allclose(td, exact, rtol=1e-5, atol=1e-6)


def test_large_base_sampled(P):
    case = get_case("sift", 20_000, 200)
    Xt, Qt = torch.from_numpy(case.X).cuda(), torch.from_numpy(case.Q).cuda()
    ti, _ = P.knn_tensor(Xt, Qt, 10)
    assert np.array_equal(ti.cpu().numpy(), case.gt_ids)


def test_arguments(P):
    X = torch.rand((500, 64), device="cuda")
    with pytest.raises(P.PeosError):
        P.knn_tensor(X, X[:10].contiguous(), 97)     # k above the tensor path's limit
    with pytest.raises(P.PeosError):
        P.knn_tensor(X, torch.rand((10, 32), device="cuda"), 5)
