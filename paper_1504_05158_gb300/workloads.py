"""Seeded synthetic QAP instances shaped like the paper's workloads.

The paper runs on QAPLIB instances (section 4.1), which are not available here;
these generators stand in for their shapes: dense uniform matrices (like the
tai*a family) and grid Manhattan distances with sparse flows (like the sko/esc
families). Every instance is symmetric with a zero diagonal and non-negative
integer entries (section 2.1). This module holds input generation only, none of
the method's arithmetic: both the CUDA path and the CPU oracle take its outputs
as inputs. NumPy's PCG64 generator keeps the streams identical on every machine.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Instance:
    name: str
    F: np.ndarray  # n x n int32 flows between facilities
    D: np.ndarray  # n x n int32 distances between locations

    @property
    def n(self) -> int:
        return int(self.F.shape[0])


def _symmetric_from_upper(n: int, upper: np.ndarray) -> np.ndarray:
    M = np.zeros((n, n), np.int32)
    iu = np.triu_indices(n, 1)
    M[iu] = upper
    return M + M.T


def dense_uniform(n: int, seed: int, lo: int = 0, hi: int = 99, name: str | None = None) -> Instance:
    """F and D symmetric, zero diagonal, off-diagonal integers uniform in [lo, hi];
    the F pairs are drawn first, then the D pairs (upper triangle, row-major)."""
    rng = np.random.default_rng(seed)
    m = n * (n - 1) // 2
    fu = rng.integers(lo, hi + 1, size=m, dtype=np.int64)
    du = rng.integers(lo, hi + 1, size=m, dtype=np.int64)
    return Instance(name or f"dense{n}_s{seed}", _symmetric_from_upper(n, fu),
                    _symmetric_from_upper(n, du))


def grid_manhattan(n: int, rows: int | None = None, cols: int | None = None) -> np.ndarray:
    """Manhattan distances between the first n cells of a rows x cols grid, cell l at
    (l // cols, l % cols). Default shape: rows = floor(sqrt n), cols = ceil(n / rows)."""
    if rows is None:
        rows = max(1, int(math.isqrt(n)))
    if cols is None:
        cols = -(-n // rows)
    idx = np.arange(n)
    r, c = idx // cols, idx % cols
    return (np.abs(r[:, None] - r[None, :]) + np.abs(c[:, None] - c[None, :])).astype(np.int32)


def sparse_flow(n: int, rng: np.random.Generator, density: float = 0.3) -> np.ndarray:
    """Symmetric flows: each pair nonzero with probability `density`; nonzero values
    floor(exp(U ln 100)) for U uniform in [0, 1), i.e. log-uniform in [1, 99]."""
    m = n * (n - 1) // 2
    nz = rng.random(m) < density
    vals = np.floor(np.exp(rng.random(m) * math.log(100.0))).astype(np.int64)
    vals = np.clip(vals, 1, 99)
    return _symmetric_from_upper(n, np.where(nz, vals, 0))


def grid_sparse(n: int, seed: int, rows: int | None = None, cols: int | None = None,
                density: float = 0.3, name: str | None = None) -> Instance:
    rng = np.random.default_rng(seed)
    F = sparse_flow(n, rng, density)
    D = grid_manhattan(n, rows, cols)
    return Instance(name or f"grid{n}_s{seed}", F, D)


# ---------------------------------------------------------------- named workloads

def tiny9(seed: int = 1) -> Instance:
    """n = 9, off-diagonal entries uniform in [0, 9] (brute-forceable: 9! = 362 880)."""
    return dense_uniform(9, seed, 0, 9, name="tiny9")


def dense30(seed: int = 30) -> Instance:
    return dense_uniform(30, seed, 0, 99, name="dense30")


def grid64(seed: int = 64) -> Instance:
    """n = 64: D = Manhattan distances on an 8 x 8 grid, F 30 % dense log-uniform flows."""
    return grid_sparse(64, seed, rows=8, cols=8, name="grid64")


def uneven_batch(count: int = 64, seed: int = 4096, n_lo: int = 20, n_hi: int = 128) -> list[Instance]:
    """`count` instances with n uniform in [n_lo, n_hi]; even indices dense uniform in
    [0, 99], odd indices grid distances with 30 % sparse flows."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    out = []
    for i, n in enumerate(ns):
        n = int(n)
        if i % 2 == 0:
            out.append(dense_uniform(n, seed + 1 + i, name=f"b{i}_dense{n}"))
        else:
            out.append(grid_sparse(n, seed + 1 + i, name=f"b{i}_grid{n}"))
    return out


@dataclass
class Request:
    arrival_s: float
    instance: Instance
    swarms: int
    swarm_size: int
    iterations: int
    seed: int


def serving_stream(rate_hz: float = 50.0, duration_s: float = 60.0, seed: int = 5000,
                   sizes=(32, 64, 100, 150), p_lo: int = 4096, p_hi: int = 16384,
                   iterations: int = 150) -> list[Request]:
    """Poisson arrivals; each request a fresh instance with n drawn from `sizes`, the
    generator chosen 50/50, and a population of p_lo..p_hi particles in 8..32 swarms."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    i = 0
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t >= duration_s:
            break
        n = int(rng.choice(sizes))
        swarms = int(rng.integers(8, 33))
        total = int(rng.integers(p_lo, p_hi + 1))
        ss = max(1, total // swarms)
        gen_seed = seed * 1000 + i
        inst = dense_uniform(n, gen_seed) if rng.random() < 0.5 else grid_sparse(n, gen_seed)
        reqs.append(Request(t, inst, swarms, ss, iterations, gen_seed))
        i += 1
    return reqs


def random_perms(count: int, n: int, seed: int) -> np.ndarray:
    """`count` uniformly random permutations of 0..n-1 (rows), as int32."""
    rng = np.random.default_rng(seed)
    return np.argsort(rng.random((count, n)), axis=1).astype(np.int32)


def random_asymmetric(n: int, seed: int, hi: int = 20) -> Instance:
    """General instance (asymmetric, nonzero diagonal) for the general-form checks."""
    rng = np.random.default_rng(seed)
    return Instance(f"asym{n}_s{seed}", rng.integers(0, hi + 1, (n, n)).astype(np.int32),
                    rng.integers(0, hi + 1, (n, n)).astype(np.int32))
