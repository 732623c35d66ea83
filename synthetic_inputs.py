"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no arithmetic of the method: it only draws the numbers that
are passed as *inputs* to both the CUDA path and the FP64 oracle (controls z,
network weights, minibatch orders).  The random fields m are not drawn here:
both sides generate them from the same counter-based Philox4x32-10 stream.

Seeds (fixed by convention):
  1  SAA sample set              4  training controls z
  2  held-out sample set         5  evaluation controls z
  3  training fields             6  network initialisation and minibatch shuffles
"""
from __future__ import annotations

import numpy as np

SEED_SAA = 1
SEED_HELDOUT = 2
SEED_TRAIN_FIELDS = 3
SEED_TRAIN_Z = 4
SEED_EVAL_Z = 5
SEED_NET = 6


def controls(seed: int, count: int, d_z: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """`count` control vectors z ~ U(lo, hi)^d_z as a (count, d_z) float64 array."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(lo, hi, size=(count, d_z))


def glorot_uniform_mlp(widths, seed: int = SEED_NET):
    """Glorot-uniform weights and zero biases for a dense net with layer widths
    `widths` = [n_in, h1, ..., n_out].  Returns lists (W_l of shape (out, in), b_l)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws, bs = [], []
    for fan_in, fan_out in zip(widths[:-1], widths[1:]):
        lim = np.sqrt(6.0 / (fan_in + fan_out))
        Ws.append(rng.uniform(-lim, lim, size=(fan_out, fan_in)))
        bs.append(np.zeros(fan_out))
    return Ws, bs


def epoch_orders(n_samples: int, epochs: int, seed: int = SEED_NET + 1000) -> np.ndarray:
    """One seeded permutation of range(n_samples) per epoch, shape (epochs, n_samples)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.stack([rng.permutation(n_samples) for _ in range(epochs)])


def random_state_like(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    """Standard-normal array (used for probe directions and synthetic states in tests)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(shape)
