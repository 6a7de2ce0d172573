"""Seeded random draws used as inputs by both the oracle and the GPU path.

Every draw comes from NumPy's Philox bit generator with an explicit seed, so a test,
the oracle and the benchmark that ask for the same (kind, seed, shape) get the same
numbers. Nothing here models the atmosphere or the optics: the random numbers are
handed to the screen generators and test cases as plain inputs.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(int(seed)))


def screen_white_noise(S: int, seed: int) -> np.ndarray:
    """Complex white noise w = a + i b, a and b independent unit normals, shape (S, S)."""
    g = rng(seed)
    a = g.standard_normal((S, S))
    b = g.standard_normal((S, S))
    return a + 1j * b


def layer_seeds(base_seed: int, n_layers: int) -> list[int]:
    """Seed of layer l is base + l (loop-batched workloads use 1000*loop + l)."""
    return [int(base_seed) + l for l in range(n_layers)]


def random_opd_nm(Np: int, rms_nm: float, seed: int, n_waves: int = 24,
                  max_cycles: float = 6.0) -> np.ndarray:
    """Smooth random OPD map [nm]: a sum of n_waves plane waves with random
    frequency (|f| <= max_cycles across the pupil), phase and amplitude, scaled to
    the requested RMS over the full square. float64, shape (Np, Np)."""
    g = rng(seed)
    x = (np.arange(Np) - (Np - 1) / 2.0) / Np
    X, Y = np.meshgrid(x, x, indexing="ij")
    out = np.zeros((Np, Np))
    for _ in range(n_waves):
        fx, fy = g.uniform(-max_cycles, max_cycles, 2)
        ph = g.uniform(0, 2 * np.pi)
        amp = g.standard_normal()
        out += amp * np.cos(2 * np.pi * (fx * X + fy * Y) + ph)
    out -= out.mean()
    out *= rms_nm / max(out.std(), 1e-300)
    return out


def random_vector(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    return scale * rng(seed).standard_normal(n)


def random_matrix(rows: int, cols: int, seed: int, scale: float = 1.0) -> np.ndarray:
    return scale * rng(seed).standard_normal((rows, cols))


def uniform(n: int, seed: int, lo: float, hi: float) -> np.ndarray:
    return rng(seed).uniform(lo, hi, n)
