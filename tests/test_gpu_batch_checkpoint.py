"""Batched updates of independent streams and checkpoint/resume."""
import numpy as np
import pytest

import synth
from gpu_util import dev, lib, perturbed_init, problem

pytestmark = pytest.mark.gpu


def test_batch_equals_individual_updates():
    p = lib()
    specs = synth.uneven_streams(count=6, steps=3, seed=5, dim_range=(8, 40), rank_range=(2, 5),
                                 tnew_range=(1, 6), t_init=6)
    made = []
    for i, s in enumerate(specs):
        T = s.t_init + sum(s.t_news)
        G, X = problem(s.dims, T, s.ranks, 100 + i)
        init = perturbed_init(G, s.t_init, i)
        a = p.str_init_cores(init, X0=dev(X[..., :s.t_init]), compute="f32")
        b = p.str_init_cores(init, X0=dev(X[..., :s.t_init]), compute="f32")
        made.append((s, X, a, b))
    t = [s.t_init for s, _, _, _ in made]
    for step in range(3):
        slabs = [dev(X[..., t[i]:t[i] + s.t_news[step]], ) for i, (s, X, _, _) in enumerate(made)]
        p.str_update_batch([a for _, _, a, _ in made], slabs)
        for i, (s, X, a, b) in enumerate(made):
            b.update(slabs[i])
            t[i] += s.t_news[step]
    for s, X, a, b in made:
        for n in (1, 2, 3):
            assert np.array_equal(a.core(n), b.core(n))


def test_batch_graph_on_a_stream_equals_individual_updates():
    """On a non-default stream the batch runs every context's update as one
    branch of a captured graph (plain branches on the first step of a shape,
    capture on the next one per buffer parity, replays after): still
    bit-identical to updating each context on its own."""
    import torch
    p = lib()
    specs = synth.uneven_streams(count=5, steps=1, seed=8, dim_range=(8, 40), rank_range=(2, 5),
                                 tnew_range=(1, 6), t_init=6)
    steps = 6
    made = []
    for i, s in enumerate(specs):
        tn = s.t_news[0]
        T = s.t_init + steps * tn
        G, X = problem(s.dims, T, s.ranks, 300 + i)
        init = perturbed_init(G, s.t_init, i)
        a = p.str_init_cores(init, X0=dev(X[..., :s.t_init]), compute="f32", sweeps=2, t_capacity=T)
        b = p.str_init_cores(init, X0=dev(X[..., :s.t_init]), compute="f32", sweeps=2, t_capacity=T)
        made.append((s, tn, X, a, b))
    st = torch.cuda.Stream()
    for step in range(steps):
        slabs = [dev(X[..., s.t_init + step * tn:s.t_init + (step + 1) * tn]) for s, tn, X, _, _ in made]
        with torch.cuda.stream(st):
            p.str_update_batch([a for _, _, _, a, _ in made], slabs)
        st.synchronize()
        for i, (_, _, _, _, b) in enumerate(made):
            b.update(slabs[i])
    for s, tn, X, a, b in made:
        assert a.time_rows() == b.time_rows() == s.t_init + steps * tn
        for n in (1, 2, 3):
            assert np.array_equal(a.core(n), b.core(n))


@pytest.mark.parametrize("sketch", ["uniform", "leverage"])
def test_rstr_batch_on_a_stream_equals_individual_updates(sketch):
    """rSTR batches on a non-default stream run every context's step as a
    concurrent branch: bit-identical to one rstr_update per context."""
    import torch
    p = lib()
    specs = synth.uneven_streams(count=4, steps=1, seed=9, dim_range=(16, 40), rank_range=(2, 4),
                                 tnew_range=(2, 5), t_init=8)
    made = []
    for i, s in enumerate(specs):
        tn = s.t_news[0]
        T = s.t_init + 3 * tn
        G, X = problem(s.dims, T, s.ranks, 800 + i)
        init = perturbed_init(G, s.t_init, 810 + i)
        kw = dict(compute="f32", sketch=sketch, m=64, seed=11 + i, t_capacity=T)
        a = p.str_init_cores(init, X0=dev(X[..., :s.t_init]), **kw)
        b = p.str_init_cores(init, X0=dev(X[..., :s.t_init]), **kw)
        made.append((s, tn, X, a, b))
    st = torch.cuda.Stream()
    for step in range(3):
        slabs = [dev(X[..., s.t_init + step * tn:s.t_init + (step + 1) * tn]) for s, tn, X, _, _ in made]
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            p.str_update_batch([a for _, _, _, a, _ in made], slabs, randomized=True)
        st.synchronize()
        for (_, _, _, _, b), x in zip(made, slabs):
            b.rupdate(x)
    for s, tn, X, a, b in made:
        assert a.time_rows() == b.time_rows()
        for n in (1, 2, 3):
            assert np.array_equal(a.core(n), b.core(n))


def test_batch_matches_the_oracle():
    """Batched updates of uneven order-3 streams (BF16 slabs, FP32 slab
    arithmetic, one sweep), each against the FP64 oracle's STR (Alg. 4) on the
    same BF16 values: cores within the FP32 tolerance 1e-5 after three steps,
    on the default stream and as a captured graph on a side stream."""
    import torch
    from oracle import stream as ost
    p = lib()
    specs = synth.uneven_streams(count=6, steps=3, seed=11, dim_range=(16, 48), rank_range=(2, 5),
                                 tnew_range=(1, 6), t_init=12)
    for on_stream in (False, True):
        made = []
        for i, s in enumerate(specs):
            T = s.t_init + sum(s.t_news)
            G, X = problem(s.dims, T, s.ranks, 500 + i)
            X = synth.to_bf16_values(X)
            init = perturbed_init(G, s.t_init, 600 + i)
            ctx = p.str_init_cores(init, X0=dev(X[..., :s.t_init], torch.bfloat16), compute="f32", t_capacity=T)
            made.append((s, X, ctx, ost.str_init(X[..., :s.t_init], init)))
        t = [s.t_init for s, _, _, _ in made]
        st = torch.cuda.Stream()
        for step in range(3):
            slabs = [dev(X[..., t[i]:t[i] + s.t_news[step]], torch.bfloat16) for i, (s, X, _, _) in enumerate(made)]
            if on_stream:
                torch.cuda.synchronize()
                with torch.cuda.stream(st):
                    p.str_update_batch([c for _, _, c, _ in made], slabs)
                st.synchronize()
            else:
                p.str_update_batch([c for _, _, c, _ in made], slabs)
            for i, (s, X, _, ref) in enumerate(made):
                ost.str_update(ref, X[..., t[i]:t[i] + s.t_news[step]])
                t[i] += s.t_news[step]
        for s, X, ctx, ref in made:
            for n in (1, 2, 3):
                a, b = ctx.core(n), ref.cores[n - 1]
                assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
            ctx.close()


def test_batch_large_rank_products_match_the_oracle():
    """Batched streams whose normal equations have orders R_n R_{n+1} of 132 to
    144 (the solve with an FP64 residual) beside small ones: cores within 1e-5
    of the oracle after two steps, and bit-identical to one update per stream."""
    import torch
    from oracle import stream as ost
    p = lib()
    shapes = [((24, 20), (12, 12, 11), 3), ((20, 28), (11, 12, 12), 2), ((18, 22), (3, 4, 2), 4)]
    made = []
    for i, (dims, ranks, tn) in enumerate(shapes):
        T = 16 + 2 * tn
        G, X = problem(dims, T, ranks, 700 + i)
        init = perturbed_init(G, 16, 710 + i)
        # both initialised through the SIMT MTTKRP (the batch's own path), so the
        # initial P_n, Q_n are the same bytes
        a = p.str_init_cores(init, X0=dev(X[..., :16], torch.float32), compute="f32", t_capacity=T, mttkrp_path=1)
        b = p.str_init_cores(init, X0=dev(X[..., :16], torch.float32), compute="f32", t_capacity=T, mttkrp_path=1)
        made.append((tn, X.astype(np.float32).astype(np.float64), a, b, ost.str_init(
            X.astype(np.float32).astype(np.float64)[..., :16], init)))
    for step in range(2):
        sl = [dev(X[..., 16 + step * tn:16 + (step + 1) * tn], torch.float32) for tn, X, _, _, _ in made]
        p.str_update_batch([a for _, _, a, _, _ in made], sl)
        for (tn, X, a, b, ref), x in zip(made, sl):
            b.update(x)
            ost.str_update(ref, X[..., 16 + step * tn:16 + (step + 1) * tn])
    for tn, X, a, b, ref in made:
        for n in (1, 2, 3):
            assert np.array_equal(a.core(n), b.core(n))
            assert np.linalg.norm(a.core(n) - ref.cores[n - 1]) <= 1e-5 * np.linalg.norm(ref.cores[n - 1])


@pytest.mark.parametrize("sketch", ["none", "leverage", "ksrft"])
def test_checkpoint_resume_is_bit_identical(sketch):
    p = lib()
    G, X = problem((16, 12), 24, (2, 3, 2), 9)
    init = perturbed_init(G, 8, 9)
    a = p.str_init_cores(init, X0=dev(X[..., :8]), sketch=sketch, m=80, seed=4)
    upd = (lambda c, x: c.update(x)) if sketch == "none" else (lambda c, x: c.rupdate(x))
    upd(a, dev(X[..., 8:12]))
    blob = a.save()
    b = p.Stream.load(blob)
    for t0 in (12, 16, 20):
        upd(a, dev(X[..., t0:t0 + 4]))
        upd(b, dev(X[..., t0:t0 + 4]))
    for n in (1, 2, 3):
        assert np.array_equal(a.core(n), b.core(n))
    assert a.time_rows() == b.time_rows() == 24


@pytest.mark.parametrize("compute", ["f64", "f32"])
def test_graph_replay_is_bit_identical(compute):
    """On a non-default stream str_update runs a warm-up step, then captures one
    CUDA graph per buffer parity and replays it; the cores must equal those of
    plain stream launches bit for bit."""
    import torch
    p = lib()
    G, X = problem((16, 24, 8), 40, (3, 2, 4, 3), 13)
    init = perturbed_init(G, 8, 13)
    dt = torch.float64 if compute == "f64" else torch.float32
    a = p.str_init_cores(init, X0=dev(X[..., :8], dt), compute=compute, sweeps=2, graphs=1)
    b = p.str_init_cores(init, X0=dev(X[..., :8], dt), compute=compute, sweeps=2, graphs=0)
    st = torch.cuda.Stream()
    for t0 in range(8, 40, 4):
        xs = dev(X[..., t0:t0 + 4], dt)
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            a.update(xs)
        st.synchronize()
        b.update(xs)
    torch.cuda.synchronize()
    for n in (1, 2, 3, 4):
        assert np.array_equal(a.core(n), b.core(n))
    assert a.time_rows() == b.time_rows() == 40
