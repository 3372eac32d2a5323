"""Helpers shared by the GPU tests (not a test module)."""
import numpy as np

import synth
from oracle import tr as otr


def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2307_00719_gb300 as p
    return p


def dev(X, dtype=None):
    """numpy tensor indexed [i_1..i_N] -> CUDA torch tensor with i_1 fastest."""
    import torch
    dtype = dtype or torch.float64
    t = torch.from_numpy(np.ascontiguousarray(np.asarray(X).transpose(list(range(X.ndim - 1, -1, -1)))))
    t = t.to(device="cuda", dtype=dtype)
    return t.permute(list(range(X.ndim - 1, -1, -1)))


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def problem(dims, T, ranks, seed, noise=1e-3):
    """Noisy Gaussian-core TR tensor (Sec. 4.2 synthetic data) and its true cores."""
    G = synth.gaussian_cores(tuple(dims) + (T,), ranks, seed)
    X = synth.add_noise(otr.tr_full(G), synth.gaussian_tensor(tuple(dims) + (T,), seed + 100), noise)
    return G, X


def perturbed_init(G, t_init, seed, scale=0.05):
    """Initial cores near the truth: G + scale * N(0,1), temporal core cut to t_init rows."""
    rng = np.random.default_rng(seed)
    out = [g + scale * rng.standard_normal(g.shape) for g in G]
    out[-1] = out[-1][:, :t_init, :]
    return out
