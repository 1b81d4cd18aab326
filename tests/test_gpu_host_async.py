"""The asynchronous host-buffer search (peos_search_host_async): batches enqueued on two
streams with pinned buffers give exactly the results of the synchronous call and of the
device-buffer call, and the counters come back too."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2402_11354_gb300 as P
    P.load()
    return P


def test_async_host_search_on_two_streams(P, sift20k):
    case = sift20k
    X = torch.from_numpy(case.X).cuda()
    G = P.Graph.from_numpy(case.nbrs, case.entry)
    codes = P.build_codes(G, X, case.cfg.L, case.cfg.m, case.cfg.proj_seed)
    nq, k = len(case.Q), 10
    want, wd, wc = P.search(G, codes, X, torch.from_numpy(case.Q).cuda(), k, 32, eps=0.2, routing=1, counters=True)
    want, wd, wc = want.cpu().numpy(), wd.cpu().numpy(), wc.cpu().numpy()
    sync = P.search_host(G, codes, X, case.Q, k, 32, eps=0.2, routing=1)[0]
    assert np.array_equal(sync, want)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    bufs = [(torch.from_numpy(case.Q).pin_memory(), torch.empty((nq, k), dtype=torch.int32).pin_memory(),
             torch.empty((nq, k), dtype=torch.float32).pin_memory(),
             torch.empty((nq, P.NCOUNTERS), dtype=torch.int32).pin_memory()) for _ in streams]
    for i in range(6):
        q, ids, d, c = bufs[i % 2]
        s = streams[i % 2]
        if i >= 2:
            s.synchronize()
            assert np.array_equal(ids.numpy(), want) and np.array_equal(d.numpy(), wd)
            assert np.array_equal(c.numpy()[:, 0], wc[:, 0])
            ids.fill_(-7)
        P.search_host(G, codes, X, q, k, 32, eps=0.2, routing=1, out=(ids, d, c), stream=s, wait=False)
    for s in streams:
        s.synchronize()
    for q, ids, d, c in bufs:
        assert np.array_equal(ids.numpy(), want)
