"""Full-size workloads on the GPU against the oracle (the launch configurations
bench.py times): the order-4 STR update and the 512x512 rSTR updates."""
import numpy as np
import pytest

import synth
from oracle import stream as ost
from oracle import tr as otr
from gpu_util import dev, lib, rel

pytestmark = pytest.mark.gpu


def _workload(w, steps):
    G = synth.gaussian_cores(tuple(w.dims) + (w.T,), w.ranks, w.seed)
    tmax = w.t_init + steps * w.t_new
    Gt = G[:-1] + [G[-1][:, :tmax, :]]
    Xt = otr.tr_full(Gt)
    E = synth.gaussian_tensor(Xt.shape, w.seed + 100)
    X = synth.add_noise(Xt, E, w.noise) if w.noise else Xt
    rng = np.random.default_rng(w.seed + 200)
    init = [g + 0.3 * rng.standard_normal(g.shape) for g in G]
    init[-1] = init[-1][:, :w.t_init, :]
    return X, init


def test_order4_update_full_size_fp32():
    """64x64x64 slabs of 10 slices, ranks 8, 5 sweeps, FP32 slab arithmetic (1e-5)."""
    import torch
    p = lib()
    w = synth.WORKLOADS["order4"]
    X, init = _workload(w, 2)
    ctx = p.str_init_cores(init, X0=dev(X[..., :w.t_init], torch.float32), compute="f32", sweeps=w.sweeps)
    ref = ost.str_init(X[..., :w.t_init], init)
    t = w.t_init
    for _ in range(2):
        ctx.update(dev(X[..., t:t + w.t_new], torch.float32))
        ost.str_update(ref, X[..., t:t + w.t_new], sweeps=w.sweeps)
        t += w.t_new
    for n in range(1, 5):
        assert rel(ctx.core(n), ref.cores[n - 1]) <= 1e-5
    e = ctx.fit_error(dev(X[..., :t], torch.float32))
    assert abs(e - otr.fit_error(X[..., :t], ref.cores)) <= 1e-5 * e


@pytest.mark.parametrize("sketch", ["uniform", "leverage", "ksrft"])
def test_rand3_update_full_size_bf16(sketch):
    """512x512 BF16 slabs of 5 slices, ranks 10, sketch size 2000: indices
    bit-exact, cores within 1e-5 of the oracle on the BF16-rounded data."""
    import torch
    p = lib()
    w = synth.WORKLOADS["rand3"]
    X, init = _workload(w, 1)
    X = synth.to_bf16_values(X)
    rng = np.random.default_rng(5)
    init = [g for g in init]
    ctx = p.str_init_cores(init, X0=dev(X[..., :w.t_init], torch.bfloat16), compute="f32", sketch=sketch,
                           m=w.sketch_m, seed=w.philox_seed)
    ref = ost.rstr_init(X[..., :w.t_init], init, sketch, w.sketch_m, w.philox_seed)
    t = w.t_init
    ctx.rupdate(dev(X[..., t:t + w.t_new], torch.bfloat16))
    ost.rstr_update(ref, X[..., t:t + w.t_new])
    for k in range(1, 4):
        assert np.array_equal(ctx.samples(k), ref.idxs[:, k - 1])
    for n in range(1, 4):
        assert rel(ctx.core(n), ref.cores[n - 1]) <= 1e-5
