"""Seeded synthetic inputs for streaming tensor-ring tracking.

This module is the only code shared by the CPU oracle and the CUDA library's
tests and benchmark.  It draws random numbers and fixes the workload shapes;
it performs none of the method's arithmetic (no tensor-ring contraction, no
unfolding, no solve).  Building the noise-free tensor TR(G) from the cores is
left to the caller: the oracle does it on the CPU, the library on the GPU.

Workloads (the paper's experiments use Gaussian-core TR tensors, Sec. 4.2;
its real data sets are not available, so these shapes stand in for them):

* ``small``   20x20xT, T=100, ranks (3,3,3), noise 1e-3 relative Frobenius,
              init on 10 slices, updates of 10 slices.
* ``order4``  64x64x64xT, T=400, ranks all 8, noise at SNR 30 dB,
              init on 40 slices, updates of 10 slices, 5 sweeps per update.
* ``rand3``   512x512xT, T=200, ranks all 10, BF16 slabs, sketch size 2000,
              Philox seed 7, init on 40 slices, updates of 5 slices.
* ``masked5`` 32x32x32x32xT, T=100, ranks all 6, 30% of entries hidden.
* ``streams`` 256 independent order-3 streams, spatial dims in [16,128],
              ranks in {2..12}, 1-16 new slices per step.

Core layout used everywhere in Python: ``G[n]`` is a float64 array of shape
``(R_n, I_n, R_{n+1})`` indexed ``G[n][r_n, i_n, r_{n+1}]`` (paper, Sec. 1),
with ``R_{N+1} = R_1``.  Tensors are numpy arrays indexed ``X[i_1, ..., i_N]``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    dims: tuple            # spatial dims I_1..I_{N-1}
    T: int                 # total temporal length
    ranks: tuple           # R_1..R_N
    seed: int              # core seed; noise uses seed+100, init guess seed+200
    noise: float           # relative Frobenius noise level nu
    t_init: int
    t_new: int
    sweeps: int = 1
    slab_dtype: str = "f64"
    sketch_m: int = 0
    philox_seed: int = 0

    @property
    def order(self) -> int:
        return len(self.dims) + 1

    @property
    def steps(self) -> int:
        return (self.T - self.t_init) // self.t_new


WORKLOADS = {
    "small": Workload("small", (20, 20), 100, (3, 3, 3), 0, 1e-3, 10, 10),
    "order4": Workload("order4", (64, 64, 64), 400, (8, 8, 8, 8), 1,
                       10.0 ** (-30.0 / 20.0), 40, 10, sweeps=5, slab_dtype="f32"),
    "rand3": Workload("rand3", (512, 512), 200, (10, 10, 10), 2, 1e-3, 40, 5,
                      slab_dtype="bf16", sketch_m=2000, philox_seed=7),
    "masked5": Workload("masked5", (32, 32, 32, 32), 100, (6, 6, 6, 6, 6), 3, 0.0,
                        100, 0, slab_dtype="f32"),
}


def gaussian_cores(dims: Sequence[int], ranks: Sequence[int], seed: int) -> List[np.ndarray]:
    """i.i.d. N(0,1) cores G_n of shape (R_n, I_n, R_{n+1}), drawn G_1 first."""
    rng = np.random.default_rng(seed)
    N = len(dims)
    assert len(ranks) == N
    out = []
    for n in range(N):
        shape = (ranks[n], dims[n], ranks[(n + 1) % N])
        out.append(rng.standard_normal(shape))
    return out


def gaussian_tensor(shape: Sequence[int], seed: int) -> np.ndarray:
    """i.i.d. N(0,1) array of the given shape (numpy index order)."""
    return np.random.default_rng(seed).standard_normal(tuple(shape))


def add_noise(x_true: np.ndarray, e: np.ndarray, nu: float) -> np.ndarray:
    """X = X_true + nu * ||X_true||_F * E / ||E||_F  (relative Frobenius noise)."""
    if nu == 0.0:
        return x_true.copy()
    return x_true + nu * np.linalg.norm(x_true) * e / np.linalg.norm(e)


def bernoulli_keep_mask(shape: Sequence[int], hide_prob: float, seed: int) -> np.ndarray:
    """Boolean mask, True = entry observed; each entry hidden with prob hide_prob."""
    rng = np.random.default_rng(seed)
    return rng.random(tuple(shape)) >= hide_prob


def pack_mask_bits(mask: np.ndarray) -> np.ndarray:
    """Pack a boolean mask into uint32 words over the i_1-fastest linear index.

    Bit b of word w covers linear index 32*w + b; a set bit means observed.
    """
    flat = np.asarray(mask, dtype=bool).reshape(-1, order="F")
    nwords = (flat.size + 31) // 32
    padded = np.zeros(nwords * 32, dtype=np.uint64)
    padded[: flat.size] = flat
    weights = (np.uint64(1) << np.arange(32, dtype=np.uint64))
    words = (padded.reshape(nwords, 32) * weights).sum(axis=1)
    return words.astype(np.uint32)


def init_guess(w: Workload) -> List[np.ndarray]:
    """Initial guess for the initial decomposition: N(0,1) cores, seed+200."""
    return gaussian_cores(tuple(w.dims) + (w.t_init,), w.ranks, w.seed + 200)


@dataclasses.dataclass
class StreamSpec:
    dims: tuple
    ranks: tuple
    t_init: int
    t_news: tuple  # per step


def uneven_streams(count: int = 256, steps: int = 16, seed: int = 5,
                   dim_range=(16, 128), rank_range=(2, 12), tnew_range=(1, 16),
                   t_init: int = 32) -> List[StreamSpec]:
    """Independent order-3 streams of uneven sizes (batched-streams workload)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        dims = tuple(int(v) for v in rng.integers(dim_range[0], dim_range[1] + 1, size=2))
        ranks = tuple(int(v) for v in rng.integers(rank_range[0], rank_range[1] + 1, size=3))
        tn = tuple(int(v) for v in rng.integers(tnew_range[0], tnew_range[1] + 1, size=steps))
        out.append(StreamSpec(dims, ranks, t_init, tn))
    return out


def to_bf16_values(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even), as float64.

    Used to give the oracle the exact values a BF16 slab holds.
    """
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    rounded = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    out = rounded.astype(np.uint32).view(np.float32)
    nan = np.isnan(f)
    if nan.any():
        out = out.copy()
        out[nan] = np.nan
    return out.astype(np.float64)


def bf16_bits(x: np.ndarray) -> np.ndarray:
    """The uint16 bit patterns of to_bf16_values(x)."""
    f = to_bf16_values(x).astype(np.float32)
    return (f.view(np.uint32) >> np.uint32(16)).astype(np.uint16)
