"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws random numbers and tracks which orbital rows / sites are
occupied; it contains none of the method's arithmetic (no ratios, inverses,
operand differences or Pfaffians).  Both the CUDA path and the CPU oracle are
fed from here, so they see bit-identical inputs.

The paper's benchmarks (Sec. 4) use batches of random matrices (1024 matrices
for the one-step study, 16384 for the delayed study) and random QMC-like
moves; no public dataset is involved.  All generators use numpy's PCG64.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def gaussian(g: np.random.Generator, shape, var: float, complex_: bool) -> np.ndarray:
    """N(0, var) entries; complex entries have independent real and imaginary
    parts of variance var/2 each (so E|z|^2 = var)."""
    if not complex_:
        return g.standard_normal(shape) * np.sqrt(var)
    s = np.sqrt(var / 2.0)
    return g.standard_normal(shape) * s + 1j * (g.standard_normal(shape) * s)


def orbital_matrix(seed: int, m: int, n: int, var: float, complex_: bool = False) -> np.ndarray:
    """m x n orbital matrix Phi with N(0, var) entries."""
    return gaussian(rng(seed), (m, n), var, complex_)


def pairing_generator(seed: int, m: int, var: float, complex_: bool = False) -> np.ndarray:
    """m x m matrix G with N(0, var) entries; the pairing matrix is G - G^T."""
    return gaussian(rng(seed), (m, m), var, complex_)


def initial_occupation(seed: int, walkers: int, m: int, n: int, first_rows: bool = False) -> np.ndarray:
    """walkers x n int32: distinct orbital rows (or sites) per walker.

    ``first_rows`` gives every walker rows 0..n-1 in order; otherwise each
    walker gets a seeded random n-subset of 0..m-1 in random order."""
    if first_rows:
        return np.tile(np.arange(n, dtype=np.int32), (walkers, 1))
    g = rng(seed)
    occ = np.empty((walkers, n), dtype=np.int32)
    for w in range(walkers):
        occ[w] = g.permutation(m)[:n]
    return occ


def move_sequence(seed: int, occ0: np.ndarray, m: int, steps: int):
    """Random single-particle moves, every one assumed accepted.

    For each step and walker: a slot i uniform in [0, n) and a new row / site
    uniform among the m - n currently unoccupied ones (kept in a per-walker
    free list; the vacated row takes the chosen entry's place).  Returns
    ``(slot, new)``, each steps x walkers int32."""
    g = rng(seed)
    W, n = occ0.shape
    occ = occ0.astype(np.int64).copy()
    occupied = np.zeros((W, m), dtype=bool)
    occupied[np.arange(W)[:, None], occ] = True
    free = np.stack([np.flatnonzero(~occupied[w]) for w in range(W)]) if m > n else np.zeros((W, 0), np.int64)
    rows = np.arange(W)
    slot = np.empty((steps, W), dtype=np.int32)
    new = np.empty((steps, W), dtype=np.int32)
    for s in range(steps):
        i = g.integers(0, n, size=W)
        p = g.integers(0, m - n, size=W)
        nr = free[rows, p]
        free[rows, p] = occ[rows, i]
        occ[rows, i] = nr
        slot[s] = i
        new[s] = nr
    return slot, new


def multi_move_sequence(seed: int, occ0: np.ndarray, m: int, steps: int, k: int):
    """k simultaneous moves per step (e.g. two-electron moves, k = 2): k
    distinct slots and k distinct unoccupied rows, every move assumed
    accepted.  Returns (slot, new), each steps x walkers x k int32."""
    g = rng(seed)
    W, n = occ0.shape
    occ = occ0.astype(np.int64).copy()
    occupied = np.zeros((W, m), dtype=bool)
    occupied[np.arange(W)[:, None], occ] = True
    free = np.stack([np.flatnonzero(~occupied[w]) for w in range(W)])
    rows = np.arange(W)
    slot = np.empty((steps, W, k), dtype=np.int32)
    new = np.empty((steps, W, k), dtype=np.int32)
    for s in range(steps):
        sl = np.argsort(g.random((W, n)), axis=1)[:, :k]
        pk = np.argsort(g.random((W, m - n)), axis=1)[:, :k]
        for a in range(k):
            nr = free[rows, pk[:, a]]
            free[rows, pk[:, a]] = occ[rows, sl[:, a]]
            occ[rows, sl[:, a]] = nr
            slot[s, :, a] = sl[:, a]
            new[s, :, a] = nr
    return slot, new


def dense_operands(seed: int, walkers: int, n: int, k: int, var: float, complex_: bool = False):
    """Dense backflow-style operands: U (walkers x k x n, column a of U stored
    as a length-n vector) and V (walkers x k x n, row a of V)."""
    g = rng(seed)
    U = gaussian(g, (walkers, k, n), var, complex_)
    V = gaussian(g, (walkers, k, n), var, complex_)
    return U, V
