"""Counter-based initial orbitals (test infrastructure; FP64 oracle).

The paper does not say how fragment orbitals are started.  Reading: every
value is drawn from the SplitMix64 generator (Steele, Lea & Flood, OOPSLA
2014), used as a counter-based hash, so that the CUDA path can reproduce each
value independently from its own implementation of the same published
definition:

    key  = seed XOR ((f << 20 | i) << 32) XOR j         (f < 4096, i < 2^20, j < 2^32)
    z    = key + 0x9E3779B97F4A7C15           (mod 2^64)
    z    = (z XOR (z >> 30)) * 0xBF58476D1CE4E5B9
    z    = (z XOR (z >> 27)) * 0x94D049BB133111EB
    z    = z XOR (z >> 31)
    psi  = (z >> 11) * 2^-52 - 1               in [-1, 1)
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(key):
    """SplitMix64 output for an array of 64-bit keys (wrap-around arithmetic)."""
    with np.errstate(over="ignore"):
        z = np.asarray(key, dtype=np.uint64) + GAMMA
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def orbital_block(seed: int, f: int, n: int, npts: int):
    """Initial orbitals of fragment f: array [n][npts] with values in [-1, 1)."""
    if f >= 4096 or n > (1 << 20):
        raise ValueError("counter layout holds f < 4096 and i < 2^20")
    i = np.arange(n, dtype=np.uint64)
    j = np.arange(npts, dtype=np.uint64)
    hi = ((np.uint64(f) << np.uint64(20)) | i) << np.uint64(32)
    key = np.uint64(seed) ^ hi[:, None] ^ j[None, :]
    z = splitmix64(key)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0
