"""Counter-based random draws for the sketches (FP64 / exact integers, CPU).

Test infrastructure only: see the package docstring.

The paper's samplers draw rows uniformly (Sec. 3.3, uniform sampling),
from a leverage-based distribution (Lemma lev_est) and draw random sign flips
(Definition of the KSRFT).  It fixes no generator, so both implementations use
one counter-based generator from its published definition: Philox4x64-10
(Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11), written here with Python integers.

Draw contract (shared with the CUDA library, which implements it separately):
* key     = (seed mod 2^64, 0)
* counter = (s, k, tau, (purpose << 32) | stream)
  s = draw number (or entry index for signs), k = 1-based mode,
  tau = time step (0 = initialisation), purpose 0 = row index, 1 = sign.
* u = word 0 of Philox4x64-10(counter, key).
* uniform index on [0, I):   floor(u * I / 2^64).
* weighted index from p:    v = (u >> 11) * 2^-53; c = sequential left-to-right
  FP64 prefix sums of p; target = v * c[I-1]; index = min{i : target < c[i]}
  (if none, the last i with p[i] > 0).
* sign: +1 if u is even, else -1.
"""
from __future__ import annotations

import itertools
from typing import Sequence

import numpy as np

MASK64 = (1 << 64) - 1
# Philox4x64 round multipliers and Weyl key increments (Salmon et al., 2011).
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B

PURPOSE_INDEX = 0
PURPOSE_SIGN = 1


def philox4x64_10(counter: Sequence[int], key: Sequence[int]):
    """Ten Philox4x64 rounds: each multiplies words 0 and 2 by the round
    constants (128-bit product), swaps/xors with words 1 and 3 and the key,
    then bumps the key by the Weyl constants."""
    c0, c1, c2, c3 = (int(v) & MASK64 for v in counter)
    k0, k1 = (int(v) & MASK64 for v in key)
    for r in range(10):
        if r:
            k0 = (k0 + PHILOX_W0) & MASK64
            k1 = (k1 + PHILOX_W1) & MASK64
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def draw_u64(seed: int, s: int, k: int, tau: int, purpose: int, stream: int = 0) -> int:
    ctr = (s, k, tau, ((purpose & 0xFFFFFFFF) << 32) | (stream & 0xFFFFFFFF))
    return philox4x64_10(ctr, (seed & MASK64, 0))[0]


def uniform_indices(seed: int, m: int, I: int, k: int, tau: int, stream: int = 0) -> np.ndarray:
    """m draws with replacement, uniform on [0, I) (Eq. sampDS, probability 1/I)."""
    out = np.empty(m, dtype=np.int64)
    for s in range(m):
        u = draw_u64(seed, s, k, tau, PURPOSE_INDEX, stream)
        out[s] = (u * I) >> 64
    return out


def prefix_sums(p: Sequence[float]) -> np.ndarray:
    """Sequential left-to-right FP64 prefix sums c[i] = c[i-1] + p[i]."""
    return np.array(list(itertools.accumulate(float(v) for v in p)), dtype=np.float64)


def weighted_indices(seed: int, m: int, p: np.ndarray, k: int, tau: int,
                     stream: int = 0) -> np.ndarray:
    """m draws with replacement, index i with probability p[i] / sum(p)."""
    c = prefix_sums(p)
    total = c[-1]
    positive = np.nonzero(np.asarray(p) > 0)[0]
    last_pos = int(positive[-1]) if positive.size else len(p) - 1
    out = np.empty(m, dtype=np.int64)
    for s in range(m):
        u = draw_u64(seed, s, k, tau, PURPOSE_INDEX, stream)
        v = float(u >> 11) * (2.0 ** -53)
        target = v * total
        i = int(np.searchsorted(c, target, side="right"))   # first i with c[i] > target
        out[s] = i if i < len(p) else last_pos
    return out


def signs(seed: int, I: int, k: int, tau: int, stream: int = 0) -> np.ndarray:
    """Random sign flips d_i in {+1, -1} (Definition of the KSRFT, D_j)."""
    out = np.empty(I, dtype=np.float64)
    for i in range(I):
        u = draw_u64(seed, i, k, tau, PURPOSE_SIGN, stream)
        out[i] = 1.0 if (u & 1) == 0 else -1.0
    return out
