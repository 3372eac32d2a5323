"""rSTR (Alg. 5 with the schedules of Algs. 7-9) on the GPU against the oracle:
sample indices bit-exact (same Philox4x64-10 stream), cores within tolerance."""
import numpy as np
import pytest

import synth
from oracle import philox, stream as ost
from oracle import tr as otr
from gpu_util import dev, lib, perturbed_init, problem, rel

pytestmark = pytest.mark.gpu


def _run(sketch, dims, T, ranks, t_init, t_new, m, seed=7, compute="f64", slab="f64", rescale=1,
         tol=1e-10, stream_id=0):
    import torch
    p = lib()
    G, X = problem(dims, T, ranks, 11)
    if slab == "bf16":
        X = synth.to_bf16_values(X)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[slab]
    init = perturbed_init(G, t_init, 3)
    ctx = p.str_init_cores(init, X0=dev(X[..., :t_init], tdt), compute=compute, sketch=sketch, m=m,
                           seed=seed, rescale=rescale, stream_id=stream_id)
    ref = ost.rstr_init(X[..., :t_init], init, sketch, m, seed, rescale=bool(rescale), stream=stream_id)
    N = len(ranks)
    for k in range(1, N + 1):
        assert np.array_equal(ctx.samples(k), ref.idxs[:, k - 1]), f"init idxs mode {k}"
    for n in range(1, N):
        P, Q = ctx.pq(n)
        assert rel(P, ref.P[n - 1]) <= tol and rel(Q, ref.Q[n - 1]) <= tol
    t = t_init
    while t + t_new <= T:
        ctx.rupdate(dev(X[..., t:t + t_new], tdt))
        ost.rstr_update(ref, X[..., t:t + t_new])
        t += t_new
        for k in range(1, N + 1):
            got = ctx.samples(k)
            mism = int(np.sum(got != ref.idxs[:, k - 1]))
            assert mism == 0, f"{mism} index mismatches, mode {k}, t={t}"
        for n in range(1, N + 1):
            r = rel(ctx.core(n), ref.cores[n - 1])
            assert r <= tol, f"core {n} rel {r:.3e} at t={t}"
    e_gpu = ctx.fit_error(dev(X[..., :t], tdt))
    e_ref = otr.fit_error(X[..., :t], ref.cores)
    assert abs(e_gpu - e_ref) <= max(tol, 1e-12) * e_ref
    ctx.close()


@pytest.mark.parametrize("sketch", ["uniform", "leverage", "ksrft"])
def test_rstr_fp64_order3(sketch):
    _run(sketch, (14, 11), 22, (2, 3, 2), 8, 3, m=90)


@pytest.mark.parametrize("sketch", ["uniform", "leverage", "ksrft"])
def test_rstr_fp64_order4_no_rescale(sketch):
    _run(sketch, (6, 5, 7), 12, (2, 2, 3, 2), 4, 4, m=70, rescale=0, stream_id=5)


@pytest.mark.parametrize("compute,tol", [("f64", 1e-10), ("f32", 1e-5)])
def test_ksrft_power_of_two_lengths(compute, tol):
    """Every mode length a power of two: mixing, core mixing and unmixing all
    take the radix-2 FFT route (the other KSRFT tests use the direct DFT)."""
    _run("ksrft", (16, 32), 16, (2, 3, 2), 8, 4, m=120, compute=compute, tol=tol)


@pytest.mark.parametrize("sketch", ["uniform", "leverage", "ksrft"])
def test_rstr_bf16_slab_fp32(sketch):
    _run(sketch, (48, 40), 20, (3, 3, 3), 10, 5, m=200, compute="f32", slab="bf16", tol=1e-5)


def test_leverage_distribution_and_sampler_given_p():
    """GPU leverage distributions equal the oracle's SVD route to 1e-12, and the
    oracle's sampler fed the GPU's p reproduces the GPU's draws bit for bit."""
    p = lib()
    G, X = problem((30, 25), 12, (2, 3, 2), 12)
    init = perturbed_init(G, 12, 4)
    ctx = p.str_init_cores(init, X0=dev(X), sketch="leverage", m=500, seed=9)
    for k, rows in ((1, 30), (2, 25), (3, 12)):
        idx, pk = ctx.samples(k, with_p=True, p_rows=rows)
        pref = ost.leverage_probs(init[k - 1])
        assert rel(pk, pref) <= 1e-12
        again = philox.weighted_indices(9, 500, pk, k, 0)
        assert np.array_equal(idx, again)
