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
    # the workload's normal equations are well conditioned: no solve needed the FP64 fallback
    assert ctx.stats()["fp64_fallbacks"] == 0


def test_order4_update_full_size_fp64():
    """The plain FP64 arm the bench times: 64x64x64 slabs of 10 slices, ranks 8,
    5 sweeps, FP64 slab arithmetic; cores, P_n, Q_n and the fit error within
    1e-10 of the oracle after two updates."""
    import torch
    p = lib()
    w = synth.WORKLOADS["order4"]
    X, init = _workload(w, 2)
    ctx = p.str_init_cores(init, X0=dev(X[..., :w.t_init], torch.float64), compute="f64", sweeps=w.sweeps)
    ref = ost.str_init(X[..., :w.t_init], init)
    t = w.t_init
    for _ in range(2):
        ctx.update(dev(X[..., t:t + w.t_new], torch.float64))
        ost.str_update(ref, X[..., t:t + w.t_new], sweeps=w.sweeps)
        t += w.t_new
    for n in range(1, 5):
        assert rel(ctx.core(n), ref.cores[n - 1]) <= 1e-10
    for n in range(1, 4):
        P, Q = ctx.pq(n)
        assert rel(P, ref.P[n - 1]) <= 1e-10 and rel(Q, ref.Q[n - 1]) <= 1e-10
    e = ctx.fit_error(dev(X[..., :t], torch.float64))
    assert abs(e - otr.fit_error(X[..., :t], ref.cores)) <= 1e-10 * e


def test_masked_loss_full_size_fp32():
    """The masked-loss workload the bench times: 32x32x32x32x100 FP32, ranks 6,
    30% of the entries hidden, noise 1e-2.  The loss within 1e-5 of the oracle's
    definition L = 1/2 sum M (X - TR(G))^2 and the gradients of the temporal
    core and of core 1, dL/dG_{n(2)} = -(M .* (X - TR(G)))_[n] G^{!=n}_[2], on
    the same FP32 values of X and of the cores.

    Gradient tolerance: the FP32 path forms each residual x - TR(G)(x) from a
    K-term dot product (K = R_1 R_{k+1} = 36) on the tensor cores, each factor
    carried as two TF32 pieces (hi + lo, 2^-22 relative) and the lo x lo product
    dropped, so a product carries about u = 3 * 2^-22 of rounding (12 u_32) and
    every residual about u sqrt(K) |x|; a gradient, a sum of residuals times
    subchain entries, then has relative error about u sqrt(K) ||X|| / ||M .* R||:
    ~100x the rounding of X for noise at 1e-2.  The test allows 8 times that,
    and at least 1e-5."""
    import torch
    from oracle import loss as olo
    p = lib()
    W = synth.WORKLOADS["masked5"]
    dims = tuple(W.dims) + (W.T,)
    G = synth.gaussian_cores(dims, W.ranks, W.seed)
    G = [g.astype(np.float32).astype(np.float64) for g in G]
    X = synth.add_noise(otr.tr_full(G), synth.gaussian_tensor(dims, W.seed + 100), 1e-2)
    X = X.astype(np.float32).astype(np.float64)
    mask = synth.bernoulli_keep_mask(dims, 0.3, W.seed)
    bits = torch.from_numpy(synth.pack_mask_bits(mask).view(np.int32)).cuda()
    cores = [torch.from_numpy(a).to("cuda", torch.float32) for a in p.cores_to_abi(G)]
    Xd = dev(X, torch.float32)
    loss = p.tr_masked_loss_fwd(cores, Xd, bits).item()
    grads = p.tr_masked_loss_bwd(cores, Xd, bits, 1.0)
    del Xd
    ref = olo.masked_loss(X, G, mask)
    assert abs(loss - ref) <= 1e-5 * ref
    res = (X - otr.tr_full(G)) * mask
    K = W.ranks[0] * W.ranks[3]
    tol = max(1e-5, 8 * 3 * 2.0 ** -22 * np.sqrt(K) * np.linalg.norm(X) / np.linalg.norm(res))
    del X
    for n in (5, 1):
        g_ref = -(otr.unfold_cyclic(res, n) @ otr.subchain_unfold(G, n))
        g_gpu = grads[n - 1].double().cpu().numpy().reshape(dims[n - 1], -1)   # rows i_n, column r_n + R_n r_{n+1}
        assert rel(g_gpu, g_ref) <= tol, (n, rel(g_gpu, g_ref), tol)


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
