"""Philox4x32-10 counter-based generator and the normals the random field draws.

Oracle (test infrastructure only).  Written from the published definition of
Philox4x32 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the constants
0xD2511F53 / 0xCD9E8D57 and a Weyl key schedule 0x9E3779B9 / 0xBB67AE85.

The field's standard normals xi (Sec. 2: m ~ N(mbar, C)) are drawn per
(sample, mode pair):  counter = (block, sample_lo, sample_hi, 0x4B4C5158),
key = (seed_lo, seed_hi).  Each 128-bit output gives two uniforms with 52
random bits, u = (k + 1/2) 2^-52 (exact in float64, never 0 or 1), and the
Box-Muller transform turns them into normals 2*block and 2*block+1.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)
STREAM_TAG = 0x4B4C5158


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """ctr: (..., 4) uint32-valued, key: (..., 2) uint32-valued -> (..., 4) uint64 words < 2^32."""
    c = [np.asarray(ctr[..., i], dtype=np.uint64) & MASK32 for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint64) & MASK32
    k1 = np.asarray(key[..., 1], dtype=np.uint64) & MASK32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c[0]                      # < 2^64, exact in uint64
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


def uniform52(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Two 32-bit words -> a uniform in (0, 1) with 52 random bits."""
    k = ((a >> np.uint64(6)) << np.uint64(26)) | (b >> np.uint64(6))
    return (k.astype(np.float64) + 0.5) * 2.0 ** -52


def field_normals(seed: int, first_sample: int, n_samples: int, n_modes: int) -> np.ndarray:
    """Standard normals xi[s, q] for samples first_sample .. first_sample+n_samples-1 and
    flat mode index q in [0, n_modes)."""
    n_blocks = (n_modes + 1) // 2
    s = np.arange(first_sample, first_sample + n_samples, dtype=np.uint64)[:, None]
    blk = np.arange(n_blocks, dtype=np.uint64)[None, :]
    ctr = np.stack(np.broadcast_arrays(blk, s & MASK32, s >> np.uint64(32),
                                       np.uint64(STREAM_TAG) + 0 * blk), axis=-1)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint64)
    w = philox4x32_10(ctr, np.broadcast_to(key, ctr.shape[:-1] + (2,)))
    u1 = uniform52(w[..., 0], w[..., 1])
    u2 = uniform52(w[..., 2], w[..., 3])
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty((n_samples, 2 * n_blocks))
    out[:, 0::2] = r * np.cos(2.0 * np.pi * u2)
    out[:, 1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:, :n_modes]
