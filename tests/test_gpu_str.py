"""STR (Alg. 4) on the GPU against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import stream as ost
from oracle import tr as otr
from gpu_util import dev, lib, perturbed_init, problem, rel

pytestmark = pytest.mark.gpu


def _run(dims, T, ranks, t_init, t_new, compute="f64", sweeps=1, slab="f64", seed=0, tol=1e-10,
         init=None, check_every=True, path=0):
    import torch
    p = lib()
    G, X = problem(dims, T, ranks, seed)
    if slab == "bf16":
        X = synth.to_bf16_values(X)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[slab]
    init = init or perturbed_init(G, t_init, seed + 7)
    ctx = p.str_init_cores(init, X0=dev(X[..., :t_init], tdt), compute=compute, sweeps=sweeps,
                           mttkrp_path=path)
    ref = ost.str_init(X[..., :t_init], init)
    worst = 0.0
    t = t_init
    while t + t_new <= T:
        ctx.update(dev(X[..., t:t + t_new], tdt))
        ost.str_update(ref, X[..., t:t + t_new], sweeps=sweeps)
        t += t_new
        if check_every or t + t_new > T:
            for n in range(1, len(ranks) + 1):
                worst = max(worst, rel(ctx.core(n), ref.cores[n - 1]))
            assert worst <= tol, f"core mismatch {worst:.3e} after t={t}"
    for n in range(1, len(ranks)):
        P, Q = ctx.pq(n)
        assert rel(P, ref.P[n - 1]) <= tol and rel(Q, ref.Q[n - 1]) <= tol
    e_gpu = ctx.fit_error(dev(X[..., :t], tdt))
    e_ref = otr.fit_error(X[..., :t], ref.cores)
    assert abs(e_gpu - e_ref) <= tol * e_ref
    assert ctx.time_rows() == t
    ctx.close()
    return worst


def test_small_config_fp64():
    """20x20xT, T=100, ranks (3,3,3), init 10 slices, 9 updates of 10 (FP64, 1e-10)."""
    w = synth.WORKLOADS["small"]
    G, X = problem(w.dims, w.T, w.ranks, w.seed, w.noise)
    init, _, _ = ost.tr_als_ne(X[..., :w.t_init], synth.init_guess(w), tol=1e-8, max_it=100)
    _run(w.dims, w.T, w.ranks, w.t_init, w.t_new, seed=w.seed, init=init)


def test_order4_sweeps_ragged_fp64():
    _run((6, 7, 5), 20, (2, 3, 2, 3), 8, 4, sweeps=3, seed=1)


def test_order5_fp64():
    _run((4, 3, 5, 3), 12, (2, 2, 3, 2, 2), 4, 4, seed=2)


def test_tile_tails_and_single_slice_fp64():
    """I_1 = 70 spans two 64-row tiles with a ragged tail; t_new = 1 slices."""
    _run((70, 9), 14, (3, 4, 2), 8, 1, seed=3, check_every=False)


@pytest.mark.parametrize("path", [0, 1])
def test_fp32_compute(path):
    _run((12, 10, 9), 16, (3, 3, 3, 3), 6, 5, compute="f32", slab="f32", sweeps=2, seed=4, tol=1e-5, path=path)


@pytest.mark.parametrize("path", [0, 1])
def test_bf16_slab_fp32_compute(path):
    _run((40, 36), 30, (4, 4, 4), 10, 5, compute="f32", slab="bf16", seed=5, tol=1e-5, path=path)


@pytest.mark.parametrize("slab", ["f32", "bf16"])
def test_tensor_core_path_every_mode(slab):
    """Dims that are multiples of 8 send every mode through the tcgen05 stage
    (mode 1 via the slab with its two fastest modes swapped); 128-row tiles end
    ragged; unequal ranks give padded N."""
    _run((16, 24, 8), 20, (3, 2, 4, 3), 8, 6, compute="f32", slab=slab, sweeps=2, seed=9, tol=1e-5)
    _run((64, 40), 23, (5, 4, 6), 7, 8, compute="f32", slab=slab, seed=10, tol=1e-5)


@pytest.mark.parametrize("R", [2, 3, 4, 5, 6, 7, 8])
def test_tensor_core_path_equal_ranks(R):
    """Equal TR-ranks take the stage-2 kernels specialised on the rank (2 x 2
    register blocks for 4 and 8, the warp-per-batch kernel for the others); the
    temporal mode's combinations span several chunks, batches and splits."""
    _run((16, 24, 8), 21, (R, R, R, R), 9, 6, compute="f32", slab="f32", sweeps=2, seed=11, tol=1e-5)


def test_tensor_core_path_order5_segments():
    """Order 5, equal ranks 5: stage 2 with both chain tables (A . Y . B per
    combination) where the runs of equal i_hi are 10 and 90 combinations long,
    so 32-combination batches straddle run boundaries."""
    _run((12, 10, 9, 7), 14, (5, 5, 5, 5, 5), 6, 4, compute="f32", slab="f32", sweeps=2, seed=12, tol=1e-5)


@pytest.mark.parametrize("compute,slab,tol", [("f64", "f64", 1e-10), ("f32", "f32", 1e-5)])
def test_tensor_train_boundary_ranks(compute, slab, tol):
    """TT specialisation (R_1 = R_{N+1} = 1): the ring closes through rank 1."""
    _run((16, 12, 8), 18, (1, 3, 2, 3), 6, 4, compute=compute, slab=slab, sweeps=2, seed=13, tol=tol)


def test_host_slab_matches_device_slab():
    import torch
    p = lib()
    G, X = problem((9, 8), 12, (2, 3, 2), 6)
    init = perturbed_init(G, 6, 1)
    a = p.str_init_cores(init, X0=dev(X[..., :6]))
    b = p.str_init_cores(init, X0=np.asfortranarray(X[..., :6]))
    a.update(dev(X[..., 6:]))
    b.update(np.asfortranarray(X[..., 6:]))
    for n in range(1, 4):
        assert np.array_equal(a.core(n), b.core(n))


def test_gpu_tr_als_ne_init_matches_oracle():
    """str_init runs TR-ALS-NE (Alg. 2) on the GPU; fixed iteration count (tol = 0)."""
    p = lib()
    G, X = problem((10, 9), 12, (2, 3, 2), 7)
    guess = synth.gaussian_cores((10, 9, 12), (2, 3, 2), 207)
    ctx = p.str_init(dev(X), (2, 3, 2), guess, init_max_it=6, init_tol=0.0)
    ref, _, _ = ost.tr_als_ne(X, guess, tol=0.0, max_it=6)
    for n in range(1, 4):
        assert rel(ctx.core(n), ref[n - 1]) <= 1e-9
    st = ost.str_init(X, ref)
    for n in range(1, 3):
        P, Q = ctx.pq(n)
        assert rel(P, st.P[n - 1]) <= 1e-9 and rel(Q, st.Q[n - 1]) <= 1e-9


def test_reconstruct_and_fit_error():
    import torch
    p = lib()
    G, X = problem((11, 7, 5), 9, (2, 3, 2, 3), 8)
    init = perturbed_init(G, 9, 2)
    ctx = p.str_init_cores(init, X0=dev(X))
    Xh = ctx.reconstruct(2, 7).cpu().numpy()
    ref = otr.tr_full([init[0], init[1], init[2], init[3][:, 2:7, :]])
    assert rel(Xh, ref) <= 1e-12
    e = ctx.fit_error(dev(X[..., 3:8]), t0=3)
    e_ref = otr.fit_error(X[..., 3:8], [init[0], init[1], init[2], init[3][:, 3:8, :]])
    assert abs(e - e_ref) <= 1e-12 * e_ref
