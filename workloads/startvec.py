"""Seeded start-vector values keyed by basis bit string.

Every basis state carries a 64-bit key (its bit string; for Hubbard models
key = up | dw << S).  The start vector component of a state is a function
of (seed, key) only, so any two orderings of the same basis see the same
vector.  The generator is the counter-based use of SplitMix64 (Steele, Lea
and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
the first output of a SplitMix64 stream whose state is seed XOR key, mapped
to a double in [-1, 1) from its top 53 bits.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 20260507

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(state) -> np.ndarray:
    """First SplitMix64 output for each 64-bit state (vectorised, uint64)."""
    z = np.asarray(state, dtype=np.uint64) + _GAMMA
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def start_values(keys, seed: int = DEFAULT_SEED) -> np.ndarray:
    """Unnormalised start-vector components U[-1, 1) for the given keys."""
    with np.errstate(over="ignore"):
        z = splitmix64(np.asarray(keys, dtype=np.uint64) ^ np.uint64(seed))
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0
