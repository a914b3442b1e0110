"""Seeded synthetic QAP instances.

This module only draws inputs (flow matrix A, distance matrix B, start
permutation p0, request mixes). It holds none of the annealing arithmetic and
imports nothing but numpy, so the CUDA path and the CPU oracle can both be fed
from it.

The instance family is the one section 4 of Paul (arXiv:1208.2675) measures on:
built like Taillard's "Taixxa" instances, with A and B symmetric, zero diagonal,
and off-diagonal entries drawn independently and uniformly.
"""
from __future__ import annotations

import numpy as np


def _sym_uniform(rng: np.random.Generator, N: int, low: int, high: int) -> np.ndarray:
    """Symmetric N x N int32, zero diagonal, upper triangle uniform in [low, high]."""
    M = np.zeros((N, N), dtype=np.int32)
    iu = np.triu_indices(N, 1)
    vals = rng.integers(low, high + 1, size=len(iu[0]), dtype=np.int64).astype(np.int32)
    M[iu] = vals
    M.T[iu] = vals
    return M


def taixxa_like(N: int, seed: int, low: int = 0, high: int = 99):
    """(A, B, p0): uniform symmetric flows and distances in [low, high], random p0."""
    rng = np.random.default_rng([int(seed), int(N), 0x51A])
    A = _sym_uniform(rng, N, low, high)
    B = _sym_uniform(rng, N, low, high)
    p0 = rng.permutation(N).astype(np.int32)
    return A, B, p0


def grid_manhattan(side: int) -> np.ndarray:
    """Distances between the points of a side x side grid, L1 metric; i = side*y + x."""
    idx = np.arange(side * side)
    x, y = idx % side, idx // side
    D = np.abs(x[:, None] - x[None, :]) + np.abs(y[:, None] - y[None, :])
    return D.astype(np.int32)


def sparse_flows(N: int, density: float, low: int, high: int,
                 rng: np.random.Generator) -> np.ndarray:
    """Symmetric flows: each i<j pair nonzero with probability `density`, value U{low..high}."""
    A = np.zeros((N, N), dtype=np.int32)
    iu = np.triu_indices(N, 1)
    nz = rng.random(len(iu[0])) < density
    vals = rng.integers(low, high + 1, size=len(iu[0]), dtype=np.int64).astype(np.int32)
    vals = np.where(nz, vals, 0).astype(np.int32)
    A[iu] = vals
    A.T[iu] = vals
    return A


def grid_instance(side: int, seed: int, density: float = 0.3, low: int = 1, high: int = 10):
    """Structured instance: B = Manhattan distances on a side x side grid, sparse A."""
    N = side * side
    rng = np.random.default_rng([int(seed), int(N), 0x6D1])
    A = sparse_flows(N, density, low, high, rng)
    B = grid_manhattan(side)
    p0 = rng.permutation(N).astype(np.int32)
    return A, B, p0


def batch_sizes(count: int, n_lo: int, n_hi: int, seed: int) -> np.ndarray:
    """Problem sizes of a batch of independent chains, N ~ U{n_lo..n_hi}."""
    rng = np.random.default_rng([int(seed), 0xBA7])
    return rng.integers(n_lo, n_hi + 1, size=count).astype(np.int32)


def request_mix(count: int, rate: float, n_lo: int, n_hi: int,
                i_lo: float, i_hi: float, seed: int):
    """A Poisson stream of solve requests.

    Returns (arrival_s, N, iters): exponential inter-arrival times at `rate` per
    second, N log-uniform in [n_lo, n_hi], iteration counts log-uniform in
    [i_lo, i_hi].
    """
    rng = np.random.default_rng([int(seed), 0x5E7])
    gaps = rng.exponential(1.0 / rate, size=count)
    arrival = np.cumsum(gaps) - gaps[0]
    N = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi + 1), size=count)).astype(np.int64)
    N = np.clip(N, n_lo, n_hi).astype(np.int32)
    iters = np.exp(rng.uniform(np.log(i_lo), np.log(i_hi), size=count)).astype(np.int64)
    return arrival, N, iters
