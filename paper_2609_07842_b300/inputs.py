"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method: it only draws particle
configurations of the shapes the paper simulates (identical particles in a
periodic cubic box at a number density rho, Sec. 2 "simulation parameters"
and Sec. 5) from numpy's PCG64 generator.  Both the CUDA path and the CPU
oracle receive the same arrays from here.
"""
from __future__ import annotations

import numpy as np


def box_length(n: int, rho: float) -> float:
    """Edge of the cubic box holding n particles at number density rho."""
    return float((n / rho) ** (1.0 / 3.0))


def uniform_positions(n: int, rho: float, seed: int) -> tuple[np.ndarray, float]:
    """n positions i.i.d. uniform in a cubic box at density rho; returns (pos[n,3], L)."""
    L = box_length(n, rho)
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = rng.uniform(0.0, L, size=(n, 3))
    return np.ascontiguousarray(pos), L


def clustered_positions(n: int, rho: float, seed: int, cluster_size: int = 4,
                        spread: float = 0.9) -> tuple[np.ndarray, float]:
    """Small clusters at uniform random centres: a low-density fluid in which most
    particles have a few close neighbours, so that the smoothed counts fall in the
    switching window of low valencies.  Returns (pos[n,3], L)."""
    L = box_length(n, rho)
    rng = np.random.Generator(np.random.PCG64(seed))
    ncl = (n + cluster_size - 1) // cluster_size
    centres = rng.uniform(0.0, L, size=(ncl, 3))
    offs = rng.normal(0.0, spread / np.sqrt(3.0), size=(ncl * cluster_size, 3))
    pos = (np.repeat(centres, cluster_size, axis=0) + offs)[:n]
    pos = np.mod(pos, L)
    return np.ascontiguousarray(pos), L


def maxwell_velocities(n: int, kT: float, seed: int, mass: float = 1.0) -> np.ndarray:
    """Velocities drawn from the Maxwell-Boltzmann distribution at temperature kT."""
    rng = np.random.Generator(np.random.PCG64(seed))
    v = rng.normal(0.0, np.sqrt(kT / mass), size=(n, 3))
    return np.ascontiguousarray(v)


def quantile_valency(counts: np.ndarray, q: float) -> float:
    """A valency f that puts the q-quantile of the given counts inside the switching
    window [f, f + 1]: f = quantile - 0.5.  Used by tests so that the chain-rule
    terms are exercised on uniform fluids, whose counts sit far above small f."""
    return float(np.quantile(counts, q) - 0.5)


def sticker_chains(nchains: int, beads: int, rho: float, seed: int, bond: float = 1.0,
                   every: int = 4) -> tuple[np.ndarray, float, np.ndarray, np.ndarray]:
    """Linear bead-spring chains for the sticker model of Sec. 4: each chain a
    random walk of `beads` beads with steps of length `bond` in uniformly random
    directions, from a uniform random start in a cubic box at bead density rho.
    Beads whose index along the chain is a multiple of `every` are stickers
    (type 1), the others spacers (type 0).  Returns (pos[n,3] wrapped into the
    box, L, types[n] int32, bonds[m,2] int64 with consecutive beads of a chain)."""
    n = nchains * beads
    L = box_length(n, rho)
    rng = np.random.Generator(np.random.PCG64(seed))
    start = rng.uniform(0.0, L, size=(nchains, 1, 3))
    step = rng.normal(size=(nchains, beads - 1, 3))
    step *= bond / np.linalg.norm(step, axis=2, keepdims=True)
    walk = np.concatenate([np.zeros((nchains, 1, 3)), np.cumsum(step, axis=1)], axis=1)
    pos = np.mod((start + walk).reshape(n, 3), L)
    k = np.arange(n) % beads
    types = (k % every == 0).astype(np.int32)
    first = np.arange(n)[k < beads - 1]
    bonds = np.stack([first, first + 1], axis=1).astype(np.int64)
    return np.ascontiguousarray(pos), L, types, np.ascontiguousarray(bonds)
