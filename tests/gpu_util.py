"""Shared helpers for the GPU parity tests (no method arithmetic here)."""
import numpy as np


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (d if d > 0 else 1.0)


def bump_table(n, L, width):
    """1-D factors of the separable sources (the oracle builds G itself)."""
    x = np.arange(n) / (n - 1)
    return np.stack([np.exp(-((x - (j + 0.5) / L) ** 2) / (2 * width * width)) for j in range(L)])
