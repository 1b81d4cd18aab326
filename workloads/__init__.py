"""Seeded synthetic workloads shaped like the paper's datasets (Table 1), plus the
proximity graph both the CUDA path and the oracle search.

This module generates inputs only; it holds none of the PEOs arithmetic.  The
paper's datasets (SIFT, GloVe, DEEP, GIST) are not available, so each config
draws vectors with the shape and value statistics of one of them:

  tiny   10,000 x 128 FP32, 50-component Gaussian mixture (centres N(0, I), sigma 0.3),
         100 queries, R=32, L=8, m=16, k=10, ef=64, eps=0.1
  sift   1,000,000 x 128, integer values 0..255 stored as FP32: a 1,000-cluster mixture in a
         16-dim latent space (overlapping clusters), mapped linearly to 128 dims with small
         isotropic noise, rectified, scaled, clipped to 0..255 and rounded (skewed, many zeros,
         low intrinsic dimension like local image descriptors); 10,000 queries; R=32, L=8, m=16
  glove  1,200,000 x 100, unit-normalised, heavy-tailed per-dimension scales, 2,000 clusters in a
         20-dim latent space; 10,000 queries; R=48, L=10, m=16
  deep   10,000,000 x 96, unit-normalised, 10,000 clusters in a 16-dim latent space; 100,000
         queries; R=32, L=8, m=16
  gist   1,000,000 x 960, non-negative values in [0, 1) (rectified, scaled by 0.1), 5,000 clusters
         in a 24-dim latent space; R=32, L=24, m=16
  sift-hard  the sift recipe with a 32-dim latent space and a cluster spread of 2 (overlapping
         clusters, a higher intrinsic dimension: recall@10 of 0.95 needs efs in the tens to
         hundreds, the regime of the paper's Sec. 6 curves)

Seeds: data 1000 + config index, queries 2000 + config index, projections 3000 + config
index.  Queries are drawn from the same mixture as the base, independently of it.
"""
from __future__ import annotations

import hashlib
import os
from dataclasses import dataclass, field, replace

import numpy as np


@dataclass(frozen=True)
class Config:
    name: str
    index: int
    n: int
    d: int
    nq: int
    R: int
    L: int
    m: int
    k: int
    ef: int
    eps: float
    ef_sweep: tuple = ()
    extra: dict = field(default_factory=dict, compare=False, hash=False)

    @property
    def data_seed(self) -> int:
        return 1000 + self.index

    @property
    def query_seed(self) -> int:
        return 2000 + self.index

    @property
    def proj_seed(self) -> int:
        return 3000 + self.index


CONFIGS = {
    "tiny": Config("tiny", 0, 10_000, 128, 100, 32, 8, 16, 10, 64, 0.1,
                   tuple(range(10, 64, 2)) + tuple(range(64, 257, 16)) + (320, 384, 512, 768, 1024)),
    "sift": Config("sift", 1, 1_000_000, 128, 10_000, 32, 8, 16, 10, 64, 0.2,
                   tuple(range(10, 33)) + (40, 48, 64, 96, 128, 192, 256)),
    "glove": Config("glove", 2, 1_200_000, 100, 10_000, 48, 10, 16, 10, 64, 0.2,
                    tuple(range(10, 64, 2)) + tuple(range(64, 129, 8)) + (160, 192, 256)),
    "deep": Config("deep", 3, 10_000_000, 96, 100_000, 32, 8, 16, 10, 64, 0.2),
    "gist": Config("gist", 4, 1_000_000, 960, 10_000, 32, 24, 16, 10, 64, 0.2,
                   tuple(range(10, 64, 2)) + tuple(range(64, 129, 8)) + (160, 192, 256)),
    "sift-hard": Config("sift-hard", 5, 1_000_000, 128, 10_000, 32, 8, 16, 10, 64, 0.2,
                        tuple(range(16, 64, 4)) + tuple(range(64, 257, 16)) + (288, 320, 384, 448, 512),
                        extra={"latent": 32, "spread": 2.0}),
}


def scaled(cfg: Config, n: int, nq: int | None = None) -> Config:
    """Same recipe at another size (tests): clusters scale with n so the points per cluster stay fixed."""
    return replace(cfg, n=n, nq=cfg.nq if nq is None else nq)


# --------------------------------------------------------------------------- recipes
def _mixture_tiny(rng, n, d, n_clusters, centres):
    lab = rng.integers(0, n_clusters, size=n)
    return (centres[lab] + 0.3 * rng.standard_normal((n, d))).astype(np.float32)


SIFT_LATENT = 16        # intrinsic dimension of the descriptor manifold
SIFT_SPREAD = 0.5       # cluster spread in latent units (neighbouring clusters overlap)
SIFT_NOISE = 0.15       # isotropic noise in the 128-d space, latent units
SIFT_SHIFT = 0.1        # rectification threshold (sets the fraction of zeros)
SIFT_GAIN = 48.0        # latent unit -> descriptor value


def _sift_params(rng, n_clusters, d, latent=SIFT_LATENT):
    centres = rng.standard_normal((n_clusters, latent))
    M = rng.standard_normal((latent, d)) / np.sqrt(latent)
    return centres, M


def _sift_points(rng, n, centres, M, spread=SIFT_SPREAD):
    nc, r = centres.shape
    d = M.shape[1]
    lab = rng.integers(0, nc, size=n)
    out = np.empty((n, d), dtype=np.float32)
    step = 1 << 16
    for s in range(0, n, step):
        e = min(n, s + step)
        z = centres[lab[s:e]] + spread * rng.standard_normal((e - s, r))
        y = z @ M + SIFT_NOISE * rng.standard_normal((e - s, d)) - SIFT_SHIFT
        out[s:e] = np.rint(np.clip(SIFT_GAIN * np.maximum(y, 0.0), 0.0, 255.0))
    return out


def _latent_params(rng, n_clusters, d, latent):
    """Cluster centres in a `latent`-dim space (N(0, I)) and a fixed map to d dims."""
    centres = rng.standard_normal((n_clusters, latent))
    M = rng.standard_normal((latent, d)) / np.sqrt(latent)
    return centres, M


def _latent_points(rng, n, centres, M, spread, noise):
    """y = (centre + spread * N(0, I)) M + noise * N(0, I): overlapping clusters on a
    low-dimensional manifold, in blocks of rows."""
    nc, r = centres.shape
    d = M.shape[1]
    lab = rng.integers(0, nc, size=n)
    step = max(1, (1 << 24) // d)
    for s in range(0, n, step):
        e = min(n, s + step)
        z = centres[lab[s:e]] + spread * rng.standard_normal((e - s, r))
        yield s, e, z @ M + noise * rng.standard_normal((e - s, d))


def _glove_points(rng, n, centres, M, scales):
    out = np.empty((n, M.shape[1]), dtype=np.float32)
    for s, e, y in _latent_points(rng, n, centres, M, 0.5, 0.15):
        y = y * scales
        out[s:e] = y / np.linalg.norm(y, axis=1, keepdims=True)
    return out


def _deep_points(rng, n, centres, M):
    out = np.empty((n, M.shape[1]), dtype=np.float32)
    for s, e, y in _latent_points(rng, n, centres, M, 0.5, 0.15):
        out[s:e] = y / np.linalg.norm(y, axis=1, keepdims=True)
    return out


def _gist_points(rng, n, centres, M):
    out = np.empty((n, M.shape[1]), dtype=np.float32)
    for s, e, y in _latent_points(rng, n, centres, M, 0.5, 0.15):
        out[s:e] = np.clip(0.1 * np.maximum(y - 0.1, 0.0), 0.0, 1.0)
    return out


def _recipe(cfg: Config):
    """The config's mixture parameters, drawn from its data seed: returns (crng, points)
    where crng continues the data stream (it draws the base next) and points(rng, n)
    draws n vectors of the recipe."""
    crng = np.random.default_rng(cfg.data_seed)
    if cfg.name == "tiny":
        n_cl = 50
        centres = crng.standard_normal((n_cl, cfg.d))
        return crng, lambda rng, n: _mixture_tiny(rng, n, cfg.d, n_cl, centres)
    if cfg.name in ("sift", "sift-hard"):
        centres, M = _sift_params(crng, max(1, round(cfg.n / 1000)), cfg.d, cfg.extra.get("latent", SIFT_LATENT))
        spread = cfg.extra.get("spread", SIFT_SPREAD)
        return crng, lambda rng, n: _sift_points(rng, n, centres, M, spread)
    if cfg.name == "glove":
        scales = np.exp(0.75 * crng.standard_normal(cfg.d))
        centres, M = _latent_params(crng, max(1, round(cfg.n / 600)), cfg.d, 20)
        return crng, lambda rng, n: _glove_points(rng, n, centres, M, scales)
    if cfg.name == "deep":
        centres, M = _latent_params(crng, max(1, round(cfg.n / 1000)), cfg.d, 16)
        return crng, lambda rng, n: _deep_points(rng, n, centres, M)
    if cfg.name == "gist":
        centres, M = _latent_params(crng, max(1, round(cfg.n / 200)), cfg.d, 24)
        return crng, lambda rng, n: _gist_points(rng, n, centres, M)
    raise KeyError(cfg.name)


def generate(cfg: Config):
    """Base vectors X [n, d] and queries Q [nq, d] (FP32) of a config, fully determined by its seeds."""
    crng, points = _recipe(cfg)
    X = points(crng, cfg.n)
    Q = points(np.random.default_rng(cfg.query_seed), cfg.nq)
    return X, Q


def queries(cfg: Config, nq: int) -> np.ndarray:
    """nq further queries of the config's recipe (same mixture as its base), from a seed of
    their own (not the config's query set)."""
    _, points = _recipe(cfg)
    return points(np.random.default_rng(cfg.query_seed + 10_000), nq)


def stats(X: np.ndarray) -> dict:
    """Realised statistics written beside each dataset."""
    nrm = np.linalg.norm(X.astype(np.float64), axis=1)
    return dict(mean=float(X.mean()), zero_frac=float((X == 0).mean()), norm_mean=float(nrm.mean()),
                norm_std=float(nrm.std()), min=float(X.min()), max=float(X.max()))


# --------------------------------------------------------------------------- cache
def cache_dir() -> str:
    d = os.environ.get("PEOS_CACHE") or os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                                      "_cache")
    os.makedirs(d, exist_ok=True)
    return d


def _save_atomic(path: str, arr: np.ndarray) -> None:
    """Write a cache file under a private name, then rename it into place: processes
    building the same workload at once (one per GPU) never read a half-written file."""
    tmp = f"{path}.{os.getpid()}.tmp.npy"
    np.save(tmp, arr)
    os.replace(tmp, path)


def _key(cfg: Config, what: str) -> str:
    h = hashlib.sha1(repr((cfg.name, cfg.n, cfg.d, cfg.nq, cfg.R, what, 2)).encode()).hexdigest()[:12]
    return os.path.join(cache_dir(), f"{cfg.name}_{cfg.n}_{what}_{h}.npy")


def dataset(cfg: Config, use_cache: bool = True):
    """(X, Q), cached on disk for the large configs."""
    px, pq = _key(cfg, "X"), _key(cfg, "Q")
    if use_cache and os.path.exists(px) and os.path.exists(pq):
        return np.load(px, mmap_mode=None), np.load(pq)
    X, Q = generate(cfg)
    if use_cache and cfg.n >= 200_000:
        _save_atomic(px, X)
        _save_atomic(pq, Q)
    return X, Q


def load_graph(cfg: Config, X: np.ndarray, device: str | None = None, use_cache: bool = True, verbose: bool = False):
    """(nbrs [n, R] int32, entry) of the config's graph; GPU-built for large n when a GPU is present."""
    from .graph import build_graph
    import torch

    pg = _key(cfg, f"G{cfg.R}")
    if use_cache and os.path.exists(pg):
        arr = np.load(pg)
        return np.ascontiguousarray(arr[1:]).astype(np.int32), int(arr[0, 0])
    if device is None:
        device = "cuda" if (torch.cuda.is_available() and cfg.n > 50_000) else "cpu"
    nbrs, entry = build_graph(X, cfg.R, device=device, verbose=verbose)
    if use_cache and cfg.n >= 200_000:
        head = np.full((1, cfg.R), entry, dtype=np.int32)
        _save_atomic(pg, np.concatenate([head, nbrs], 0))
    return nbrs, entry
