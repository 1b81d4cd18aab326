"""Failure detection without a GPU fault: a device wait on an mbarrier that nothing
arrives on gives up once its time limit passed, the host reads the outcome, and the
device keeps working (a tensor-core brute force right after it is exact)."""
import time

import pytest
import torch

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


@pytest.mark.parametrize("limit_us", [1, 1000, 200_000])
def test_bounded_wait_gives_up_and_the_device_stays_usable(P, limit_us):
    P.selftest_bounded_wait(1)  # warm the launch path
    t0 = time.perf_counter()
    assert P.selftest_bounded_wait(limit_us)
    waited = time.perf_counter() - t0
    assert waited >= limit_us * 1e-6  # it waited for its limit, not a fixed number of polls
    assert waited < limit_us * 1e-6 + 1.0  # and gave up soon after it
    cfg = workloads.scaled(workloads.CONFIGS["sift"], 3000, 50)
    X, Q = workloads.generate(cfg)
    Xt, Qt = torch.from_numpy(X).cuda(), torch.from_numpy(Q).cuda()
    ti, _ = P.knn_tensor(Xt, Qt, 10)
    ei, _ = P.knn_bruteforce(Xt, Qt, 10)
    assert torch.equal(ti, ei)


def test_bounded_wait_arguments(P):
    with pytest.raises(P.PeosError):
        P.selftest_bounded_wait(0)
    with pytest.raises(P.PeosError):
        P.selftest_bounded_wait(2_000_001)
