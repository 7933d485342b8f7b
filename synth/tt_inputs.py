"""Seeded generators for TT-cores, TT-matrix cores, index tuples and weights.

Core layout (the library's ABI layout): one array per core k of shape
``(batch, r_{k-1}, n_k, r_k)`` for TT-vectors and ``(batch, r_{k-1}, m_k, n_k, r_k)`` for
TT-matrices, with ``r_0 = r_d = 1`` (the TT definition of Section 1 of the paper).
Everything is drawn in float64 from ``numpy.random.default_rng(seed)``; callers round to
float32 / bfloat16 themselves when a reduced-precision run needs it.

The workload recipes below mirror the paper's benchmark objects (Section 4: random TT
tensors with d=10, modes 10, TT-rank 10) and the five configurations of the hot path
(tiny brute-force case, tensor completion, batched Gram / matvec, uneven batches,
projection at scale). "N(0, 1/sqrt(r))" is read as standard deviation 1/sqrt(r).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "tt_ranks", "random_tt", "random_ttm", "random_indices", "loguniform_ranks",
    "Config1", "Config2", "Config3a", "Config3b", "Config4", "Config5",
    "config1", "config2", "config3a", "config3b", "config4", "config5",
]


def tt_ranks(d: int, r: int) -> list[int]:
    """(1, r, ..., r, 1): d+1 ranks with the boundary ranks fixed to one."""
    if d < 1:
        raise ValueError("d must be >= 1")
    return [1] + [int(r)] * (d - 1) + [1]


def random_tt(rng: np.random.Generator, batch: int, n, ranks, std: float = 1.0):
    """A batch of TT-vectors with i.i.d. N(0, std^2) cores, one array per core."""
    d = len(ranks) - 1
    n = [int(n)] * d if np.isscalar(n) else [int(v) for v in n]
    return [rng.normal(0.0, std, size=(batch, ranks[k], n[k], ranks[k + 1]))
            for k in range(d)]


def random_ttm(rng: np.random.Generator, batch: int, m, n, ranks, std: float = 1.0):
    """A batch of TT-matrices (row modes m, column modes n) with i.i.d. N(0, std^2) cores."""
    d = len(ranks) - 1
    m = [int(m)] * d if np.isscalar(m) else [int(v) for v in m]
    n = [int(n)] * d if np.isscalar(n) else [int(v) for v in n]
    return [rng.normal(0.0, std, size=(batch, ranks[k], m[k], n[k], ranks[k + 1]))
            for k in range(d)]


def random_indices(rng: np.random.Generator, N: int, n) -> np.ndarray:
    """N index tuples, uniform per mode, with replacement; int32, layout [d][N] (SoA)."""
    n = [int(v) for v in n]
    return np.stack([rng.integers(0, nk, size=N, dtype=np.int64) for nk in n]).astype(np.int32)


def loguniform_ranks(rng: np.random.Generator, lo: int, hi: int, size: int) -> np.ndarray:
    """r = floor(exp(U(ln lo, ln(hi+1)))), clipped to [lo, hi]."""
    u = rng.uniform(math.log(lo), math.log(hi + 1), size=size)
    return np.clip(np.floor(np.exp(u)).astype(np.int64), lo, hi)


# ---------------------------------------------------------------------------------------
# Workload recipes
# ---------------------------------------------------------------------------------------

@dataclass
class Config1:
    """Tiny brute-force case: two batches of 8 TTs (d=4, n=3, r=2, N(0,1)), a TT point X of
    the same shape, 1000 uniform index tuples with targets noise, 8 projection weights."""
    A: list
    B: list
    X: list
    idx: np.ndarray
    noise: np.ndarray
    c: np.ndarray
    d: int = 4
    n: int = 3
    r: int = 2


def config1(seed: int = 1) -> Config1:
    rng = np.random.default_rng(seed)
    d, n, r = 4, 3, 2
    ranks = tt_ranks(d, r)
    A = random_tt(rng, 8, n, ranks, 1.0)
    B = random_tt(rng, 8, n, ranks, 1.0)
    X = random_tt(rng, 1, n, ranks, 1.0)
    idx = random_indices(rng, 1000, [n] * d)
    noise = rng.normal(0.0, 0.01, size=1000)
    c = rng.normal(0.0, 1.0, size=8)
    return Config1(A, B, X, idx, noise, c)


@dataclass
class Config2:
    """Tensor completion: target T of rank 4 (d=10, n=10, std 1/sqrt(4)), model X of rank 8
    (std 1/sqrt(8)), N uniform observed tuples, additive noise sigma*N(0,1) for the targets
    y = T(i) + noise (the caller evaluates T at the tuples)."""
    T: list
    X: list
    idx: np.ndarray
    noise: np.ndarray
    d: int
    n: int
    r_target: int
    r_model: int


def config2(seed: int = 2, N: int = 1_000_000, d: int = 10, n: int = 10,
            r_target: int = 4, r_model: int = 8, sigma: float = 0.01) -> Config2:
    rng = np.random.default_rng(seed)
    T = random_tt(rng, 1, n, tt_ranks(d, r_target), 1.0 / math.sqrt(r_target))
    X = random_tt(rng, 1, n, tt_ranks(d, r_model), 1.0 / math.sqrt(r_model))
    idx = random_indices(rng, N, [n] * d)
    noise = rng.normal(0.0, sigma, size=N)
    return Config2(T, X, idx, noise, d, n, r_target, r_model)


@dataclass
class Config3a:
    """Batched Gram: bA vs bB TT-vectors, d=10, n=10, r=10, std 1/sqrt(r)."""
    A: list
    B: list


def config3a(seed: int = 3, bA: int = 100, bB: int = 100, d: int = 10, n: int = 10,
             r: int = 10) -> Config3a:
    rng = np.random.default_rng(seed)
    ranks = tt_ranks(d, r)
    A = random_tt(rng, bA, n, ranks, 1.0 / math.sqrt(r))
    B = random_tt(rng, bB, n, ranks, 1.0 / math.sqrt(r))
    return Config3a(A, B)


@dataclass
class Config3b:
    """Batched matvec: b TT-matrices (d=10, 4x4 modes, r=10) zipped with b TT-vectors
    (n=4, r=10); std 1/sqrt(r)."""
    A: list
    x: list


def config3b(seed: int = 4, batch: int = 100, d: int = 10, m: int = 4, n: int = 4,
             r: int = 10) -> Config3b:
    rng = np.random.default_rng(seed)
    ranks = tt_ranks(d, r)
    A = random_ttm(rng, batch, m, n, ranks, 1.0 / math.sqrt(r))
    x = random_tt(rng, batch, n, ranks, 1.0 / math.sqrt(r))
    return Config3b(A, x)


@dataclass
class Config4Group:
    d: int
    n: int
    ranks: np.ndarray          # per-object constant TT-rank, shape [objects]
    cores: list = field(default_factory=list)  # per object: list of d core arrays (r0,n,r1)


@dataclass
class Config4:
    """Uneven batches: G groups of S objects; (d, n) drawn per group (d in [4,16],
    n in [2,16]); a constant rank per object, log-uniform in [2,64]; std 1/sqrt(r)."""
    groups: list


def config4(seed: int = 5, groups: int = 8, per_group: int = 64, d_lo: int = 4,
            d_hi: int = 16, n_lo: int = 2, n_hi: int = 16, r_lo: int = 2,
            r_hi: int = 64) -> Config4:
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(groups):
        d = int(rng.integers(d_lo, d_hi + 1))
        n = int(rng.integers(n_lo, n_hi + 1))
        rs = loguniform_ranks(rng, r_lo, r_hi, per_group)
        g = Config4Group(d=d, n=n, ranks=rs)
        for r in rs:
            cores = random_tt(rng, 1, n, tt_ranks(d, int(r)), 1.0 / math.sqrt(int(r)))
            g.cores.append([c[0] for c in cores])
        out.append(g)
    return Config4(out)


@dataclass
class Config5:
    """Projection at scale: X of rank 32 (d=20, n=16, std 1/sqrt(32)); b TTs of rank 8
    (std 1/sqrt(8)) to be projected and summed with weights c ~ N(0,1)."""
    X: list
    Z: list
    c: np.ndarray


def config5(seed: int = 6, batch: int = 1000, d: int = 20, n: int = 16, rX: int = 32,
            rZ: int = 8) -> Config5:
    rng = np.random.default_rng(seed)
    X = random_tt(rng, 1, n, tt_ranks(d, rX), 1.0 / math.sqrt(rX))
    Z = random_tt(rng, batch, n, tt_ranks(d, rZ), 1.0 / math.sqrt(rZ))
    c = rng.normal(0.0, 1.0, size=batch)
    return Config5(X, Z, c)
