"""Shared fixtures.  Tests marked `gpu` need a CUDA device and the compiled library;
everything else runs on the CPU (oracle pins, host logic, ABI exports)."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled PEOs library")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


def _gpu_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _gpu_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


class Case:
    """A small workload: base X, queries Q, graph, entry, ground truth, oracle index."""

    def __init__(self, cfg, with_index=True):
        import oracle
        import workloads
        from workloads.graph import build_graph
        self.cfg = cfg
        self.X, self.Q = workloads.generate(cfg)
        self.nbrs, self.entry = build_graph(self.X, cfg.R)
        self.gt_ids, self.gt_d = oracle.knn_f64(self.X, self.Q, cfg.k)
        self.index = oracle.Index(self.X, self.nbrs, self.entry, cfg.L, cfg.m, cfg.proj_seed) if with_index else None


_cases = {}


def get_case(name: str, n: int, nq: int):
    import workloads
    key = (name, n, nq)
    if key not in _cases:
        _cases[key] = Case(workloads.scaled(workloads.CONFIGS[name], n, nq))
    return _cases[key]


@pytest.fixture(scope="session")
def tiny():
    """The tiny config at full size: 10,000 x 128, 100 queries, R=32, L=8, m=16."""
    import workloads
    key = ("tiny", 10_000, 100)
    if key not in _cases:
        _cases[key] = Case(workloads.CONFIGS["tiny"])
    return _cases[key]


@pytest.fixture(scope="session")
def sift20k():
    """SIFT-shaped integer data at 20,000 points, 200 queries (several tiles, ragged tail)."""
    return get_case("sift", 20_000, 200)


@pytest.fixture(scope="session")
def rng():
    return np.random.default_rng(12345)
