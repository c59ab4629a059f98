"""Oracle of the geo-anchor draw from a reference crop (TEST INFRASTRUCTURE ONLY: only
tests/ use it; the CUDA library never calls it).

Supp. "TDOM/DSM Reference Crop": the valid geo-anchors the solver uses are sampled from the
reference crop.  The paper does not say how.  Reading: a uniform draw without replacement
of n of the crop's valid pixels, made repeatable by a counter-based generator: pixel j gets
the key (upper 32 bits of the (j+1)-th output of SplitMix64 seeded with `seed`) * 2^32 + j,
and the n valid pixels with the smallest keys are drawn, listed in increasing pixel order.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014), written here from its published definition: the state advances by
0x9E3779B97F4A7C15 per output, and an output is the state mixed by
z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
(all modulo 2^64).  Plain Python integers, one pixel at a time.
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(seed: int, count: int) -> list:
    """The first `count` outputs of SplitMix64 started at state `seed`."""
    state = seed & _MASK
    out = []
    for _ in range(count):
        state = (state + _GAMMA) & _MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        out.append(z ^ (z >> 31))
    return out


def draw_keys(seed: int, n_pixels: int) -> list:
    """Key of every pixel: (upper 32 bits of its generator output) * 2^32 + pixel index."""
    return [((z >> 32) << 32) | j for j, z in enumerate(splitmix64(seed, n_pixels))]


def sample_anchors(valid, n_select: int, seed: int) -> np.ndarray:
    """Indices of the drawn pixels, increasing: the min(n_select, #valid) valid pixels with
    the smallest keys."""
    valid = np.asarray(valid).astype(bool).ravel()
    keys = draw_keys(seed, valid.size)
    cand = sorted((keys[j], j) for j in range(valid.size) if valid[j])
    chosen = [j for _, j in cand[:max(0, int(n_select))]]
    return np.array(sorted(chosen), dtype=np.int64)
