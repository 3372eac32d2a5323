"""Pins for the oracle's STR / rSTR steps (CPU only)."""
import itertools

import numpy as np
import pytest

import synth
from oracle import philox, stream, tr
from oracle.loss import closed_form_grad, masked_loss, masked_loss_grad


def _problem(dims, T, ranks, seed, noise=0.0):
    G = synth.gaussian_cores(tuple(dims) + (T,), ranks, seed)
    X = tr.tr_full(G)
    if noise:
        X = synth.add_noise(X, synth.gaussian_tensor(X.shape, seed + 100), noise)
    return G, X


def test_temporal_solve_equals_lstsq():
    """Temporal update (Sec. 3.1) = least squares on the explicit unfolded problem."""
    G, X = _problem((4, 5), 12, (2, 3, 2), 0, noise=0.05)
    st = stream.str_init(X[..., :8], [g if k < 2 else g[:, :8, :] for k, g in enumerate(G)])
    Xnew = X[..., 8:]
    A = tr.subchain_unfold(st.cores, 3)
    ref = np.linalg.lstsq(A, tr.unfold_cyclic(Xnew, 3).T, rcond=None)[0].T
    stream.str_update(st, Xnew)
    got = tr.core_unfold2(st.cores[2][:, 8:, :])
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12)


def test_exact_recovery_fixed_point():
    """Noise-free TR data with the true cores as init: every update is a fixed point."""
    dims, T, ranks = (6, 7), 30, (2, 3, 2)
    G, X = _problem(dims, T, ranks, 1)
    st = stream.str_init(X[..., :10], [G[0], G[1], G[2][:, :10, :]])
    for t0 in range(10, 30, 5):
        stream.str_update(st, X[..., t0:t0 + 5])
    for k in range(3):
        ref = G[k] if k < 2 else G[2]
        assert np.linalg.norm(st.cores[k] - ref) <= 1e-10 * np.linalg.norm(ref)
    assert tr.fit_error(X, st.cores) <= 1e-12


def test_exact_recovery_tensor_train():
    """TT format (R_1 = R_{N+1} = 1, Sec. 2): the TR definitions reduce to the
    train, TR(G)(i) = G_1(i_1) .. G_N(i_N) as a 1 x 1 product, and noise-free
    data with the true cores as init is again a fixed point of every update."""
    dims, T, ranks = (6, 5, 4), 18, (1, 3, 2, 3)
    G, X = _problem(dims, T, ranks, 4)
    i = (2, 4, 1, 7)
    prod = G[0][:, i[0], :] @ G[1][:, i[1], :] @ G[2][:, i[2], :] @ G[3][:, i[3], :]
    assert prod.shape == (1, 1) and abs(X[i] - prod[0, 0]) <= 1e-12 * max(1.0, abs(prod[0, 0]))
    st = stream.str_init(X[..., :6], [G[0], G[1], G[2], G[3][:, :6, :]])
    for t0 in range(6, 18, 4):
        stream.str_update(st, X[..., t0:t0 + 4])
    for k in range(4):
        assert np.linalg.norm(st.cores[k] - G[k]) <= 1e-9 * np.linalg.norm(G[k])


def test_streamed_pq_equal_batch_with_frozen_cores():
    """Eq. partial: with the cores frozen, P_n and Q_n accumulated slab by slab
    equal X_[n] G^{!=n}_[2] and its Gram on the concatenated tensor."""
    dims, T, ranks = (4, 3, 5), 11, (2, 3, 2, 2)
    G = synth.gaussian_cores(dims + (T,), ranks, 2)
    X = synth.gaussian_tensor(dims + (T,), 3)
    splits = [0, 4, 5, 9, 11]
    for n in range(1, 4):
        P = np.zeros((dims[n - 1], ranks[n - 1] * ranks[n % 4]))
        Q = 0
        for a, b in zip(splits[:-1], splits[1:]):
            Gs = G[:3] + [G[3][:, a:b, :]]
            P = P + tr.mttkrp(X[..., a:b], Gs, n)
            Q = Q + tr.gram_explicit(Gs, n)
        np.testing.assert_allclose(P, tr.mttkrp(X, G, n), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(Q, tr.gram_explicit(G, n), rtol=1e-12, atol=1e-12)


def test_one_step_with_empty_history_is_an_als_sweep():
    """P_old = Q_old = 0 and X_new = the whole tensor: one STR step is one ALS
    sweep in the order N, 1, .., N-1, each solve a plain lstsq (Alg. 1)."""
    dims, T, ranks = (4, 5, 3), 6, (2, 2, 3, 2)
    G0 = synth.gaussian_cores(dims + (T,), ranks, 4)
    X = synth.gaussian_tensor(dims + (T,), 5)
    st = stream.State(cores=[g.copy() for g in G0[:3]] + [G0[3][:, :0, :]],
                      P=[np.zeros((d, ranks[n] * ranks[(n + 1) % 4])) for n, d in enumerate(dims)],
                      Q=[np.zeros((ranks[n] * ranks[(n + 1) % 4],) * 2) for n in range(3)])
    stream.str_update(st, X)
    ref = [g.copy() for g in G0]
    for n in [4, 1, 2, 3]:
        A = tr.subchain_unfold(ref, n)
        sol = np.linalg.lstsq(A, tr.unfold_cyclic(X, n).T, rcond=None)[0].T
        ref[n - 1] = tr.core_fold2(sol, ranks[n - 1], ranks[n % 4])
    for k in range(4):
        np.testing.assert_allclose(st.cores[k], ref[k], rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("sweeps", [2, 3])
def test_sweeps_with_empty_history_are_als_sweeps(sweeps):
    """Reading of "s sweeps per update" (P_old, Q_old frozen for the step; every
    sweep recomputes G_N^new, then each P_n = P_n^old + increment with the
    current cores): with P_old = Q_old = 0 and the whole tensor as the slab,
    s sweeps of one STR step are s ALS sweeps (Alg. 1) in the order N, 1, ..,
    N-1, each solve a plain lstsq of the explicit unfolded problem.  A sweep
    that accumulated its increment on top of the previous sweep's P_n (instead
    of the frozen P_n^old) would double-count the slab from the second sweep."""
    dims, T, ranks = (4, 5, 3), 6, (2, 2, 3, 2)
    G0 = synth.gaussian_cores(dims + (T,), ranks, 24)
    X = synth.gaussian_tensor(dims + (T,), 25)
    st = stream.State(cores=[g.copy() for g in G0[:3]] + [G0[3][:, :0, :]],
                      P=[np.zeros((d, ranks[n] * ranks[(n + 1) % 4])) for n, d in enumerate(dims)],
                      Q=[np.zeros((ranks[n] * ranks[(n + 1) % 4],) * 2) for n in range(3)])
    stream.str_update(st, X, sweeps=sweeps)
    ref = [g.copy() for g in G0]
    for _ in range(sweeps):
        for n in [4, 1, 2, 3]:
            A = tr.subchain_unfold(ref, n)
            sol = np.linalg.lstsq(A, tr.unfold_cyclic(X, n).T, rcond=None)[0].T
            ref[n - 1] = tr.core_fold2(sol, ranks[n - 1], ranks[n % 4])
    for k in range(4):
        np.testing.assert_allclose(st.cores[k], ref[k], rtol=1e-8, atol=1e-10)
    # P_n, Q_n after the step hold exactly one slab's worth (the last sweep's)
    for n in range(1, 4):
        before = _cores_before_mode(X, G0, ranks, sweeps, n)
        np.testing.assert_allclose(st.P[n - 1], tr.mttkrp(X, before, n), rtol=1e-8, atol=1e-8)
        np.testing.assert_allclose(st.Q[n - 1], tr.gram_explicit(before, n), rtol=1e-8, atol=1e-8)


def _cores_before_mode(X, G0, ranks, sweeps, n):
    """Cores as they stand when mode n is solved in the last of `sweeps` ALS
    sweeps (order N, 1, .., N-1) from G0 with an empty temporal history."""
    ref = [g.copy() for g in G0]
    for sw in range(sweeps):
        for k in [4, 1, 2, 3]:
            if sw == sweeps - 1 and k == n:
                return ref
            A = tr.subchain_unfold(ref, k)
            sol = np.linalg.lstsq(A, tr.unfold_cyclic(X, k).T, rcond=None)[0].T
            ref[k - 1] = tr.core_fold2(sol, ranks[k - 1], ranks[k % 4])
    return ref


def test_sweeps_reduce_or_keep_error():
    dims, T, ranks = (8, 9), 40, (3, 3, 3)
    G, X = _problem(dims, T, ranks, 16, noise=1e-2)
    init, _, _ = stream.tr_als_ne(X[..., :10], synth.gaussian_cores(dims + (10,), ranks, 216),
                                  tol=1e-10, max_it=60)
    s1 = stream.str_init(X[..., :10], init)
    s5 = stream.str_init(X[..., :10], init)
    for t0 in range(10, 40, 10):
        stream.str_update(s1, X[..., t0:t0 + 10], sweeps=1)
        stream.str_update(s5, X[..., t0:t0 + 10], sweeps=5)
    e1, e5 = tr.fit_error(X, s1.cores), tr.fit_error(X, s5.cores)
    assert e5 <= e1 * 1.05 and e1 < 0.05


def test_tr_als_ne_recovers_exact_tensor():
    dims, ranks = (6, 5, 7), (2, 2, 2)
    G, X = _problem(dims[:2], dims[2], ranks, 7)
    cores, it, err = stream.tr_als_ne(X, synth.gaussian_cores(dims, ranks, 207), tol=1e-14, max_it=300)
    assert err < 1e-6


# ----------------------------------------------------------------------------
# sketches
# ----------------------------------------------------------------------------
def _all_rows(dims, n):
    """idxs (J_n x N) enumerating every combination of the modes k != n, in the
    order of the subchain's row index (i_{n+1} fastest, cyclically)."""
    N = len(dims)
    cyc = [(n + t) % N for t in range(N - 1)]
    rows = []
    for combo in itertools.product(*[range(dims[k]) for k in reversed(cyc)]):
        r = [0] * N
        for k, v in zip(reversed(cyc), combo):
            r[k] = v
        rows.append(r)
    return np.array(rows, dtype=np.int64)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_full_index_set_sketch_is_exact(n):
    """With S = every row once (and no rescale), the sampled subchain (Alg. 3)
    and the gathered fibres are exactly G^{!=n}_[2] and X_[n]."""
    dims, ranks = (3, 4, 2, 3), (2, 3, 2, 3)
    G = synth.gaussian_cores(dims, ranks, 8)
    X = synth.gaussian_tensor(dims, 9)
    idxs = _all_rows(dims, n)
    np.testing.assert_allclose(stream.sampled_subchain(G, idxs, n), tr.subchain_unfold(G, n),
                               rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(stream.sampled_fibres(X, idxs, n), tr.unfold_cyclic(X, n))


def test_dft_mix_is_the_unitary_dft_by_definition():
    dims = (4, 3, 5)
    X = synth.gaussian_tensor(dims, 10)
    D = [philox.signs(3, d, k + 1, 0) for k, d in enumerate(dims)]
    Y = X.astype(complex)
    for k, d in enumerate(dims):
        F = np.array([[np.exp(-2j * np.pi * a * b / d) for b in range(d)] for a in range(d)]) / np.sqrt(d)
        Y = tr.ttm(Y, F @ np.diag(D[k]), k + 1)
    np.testing.assert_allclose(stream.dft_mix(X, D), Y, rtol=1e-12, atol=1e-12)
    assert abs(np.linalg.norm(Y) - np.linalg.norm(X)) <= 1e-12 * np.linalg.norm(X)  # Parseval
    G = synth.gaussian_cores((5,), (3,), 11)[0]
    G = np.random.default_rng(1).standard_normal((2, 5, 3))
    F5 = np.array([[np.exp(-2j * np.pi * a * b / 5) for b in range(5)] for a in range(5)]) / np.sqrt(5)
    np.testing.assert_allclose(stream.dft_mix_core(G, D[2]), tr.ttm(G, F5 @ np.diag(D[2]), 2),
                               rtol=1e-12, atol=1e-12)
    fib = np.random.default_rng(2).standard_normal((5, 7)) + 1j
    np.testing.assert_allclose(stream.dft_unmix(F5 @ np.diag(D[2]) @ fib, D[2]), fib, atol=1e-12)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_ksrft_full_index_set_is_exact(n):
    """KSRFT with every mixed row: (x) F_j D_j is unitary, so the sketched P_n, Q_n
    equal the exact X_[n] G^{!=n}_[2] and Gram (Definition SRFT)."""
    dims, ranks = (3, 4, 5), (2, 3, 2)
    G = synth.gaussian_cores(dims, ranks, 12)
    X = synth.gaussian_tensor(dims, 13)
    D = [philox.signs(4, d, k + 1, 1) for k, d in enumerate(dims)]
    Xh = stream.dft_mix(X, D)
    Gh = [stream.dft_mix_core(g, D[k]) for k, g in enumerate(G)]
    idxs = _all_rows(dims, n)
    Gs = stream.sampled_subchain(Gh, idxs, n)
    Xs = stream.dft_unmix(stream.sampled_fibres(Xh, idxs, n), D[n - 1])
    dP, dQ = stream._pq_increment(Xs, Gs, np.ones(len(idxs)))
    np.testing.assert_allclose(dP, tr.mttkrp(X, G, n), rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(dQ, tr.gram_explicit(G, n), rtol=1e-11, atol=1e-11)


def test_leverage_svd_equals_gram_route_and_sums_to_rank():
    rng = np.random.default_rng(14)
    G = rng.standard_normal((3, 40, 4))
    p = stream.leverage_probs(G)
    A = tr.core_unfold2(G)
    lev_gram = np.einsum("ij,jk,ik->i", A, np.linalg.inv(A.T @ A), A)
    np.testing.assert_allclose(p * 12, lev_gram, rtol=1e-12)
    assert abs(p.sum() - 1) < 1e-12
    # I <= R^2 with full row rank: all leverage scores are 1, p is uniform
    Gs = rng.standard_normal((3, 7, 4))
    np.testing.assert_allclose(stream.leverage_probs(Gs), np.full(7, 1 / 7), rtol=1e-12)


def test_lemma_lev_est_inequality():
    """Lemma lev_est: prod_{m != n} p_m(i_m) >= beta_n p^{!=n}(i) for every row."""
    dims, ranks = (4, 5, 3, 4), (2, 2, 1, 2)
    G = synth.gaussian_cores(dims, ranks, 15)
    N = 4
    for n in range(1, N + 1):
        A = tr.subchain_unfold(G, n)
        U, s, _ = np.linalg.svd(A, full_matrices=False)
        r = int(np.sum(s > 1e-12 * s[0]))
        pex = np.sum(U[:, :r] ** 2, axis=1) / r
        ps = [stream.leverage_probs(g) for g in G]
        idxs = _all_rows(dims, n)
        q = np.ones(len(idxs))
        for k in range(N):
            if k != n - 1:
                q *= ps[k][idxs[:, k]]
        beta = 1.0 / (ranks[n - 1] * ranks[n % N] *
                      np.prod([ranks[k] ** 2 for k in range(N) if k not in (n - 1, n % N)]))
        assert np.all(q >= beta * pex * (1 - 1e-12))


@pytest.mark.parametrize("sketch", ["uniform", "leverage", "ksrft"])
def test_rescaled_sketch_is_unbiased(sketch):
    """E[sketched, rescaled Delta P_n] = exact Delta P_n (Eq. sampDS; for KSRFT the
    scale of the operator in Definition SRFT, with fresh signs per draw): the
    mean over many independent draws lies within 4.5 standard errors."""
    dims, ranks = (4, 3, 3), (2, 2, 2)
    G = synth.gaussian_cores(dims, ranks, 16)
    X = synth.gaussian_tensor(dims, 17)
    n, m, reps = 1, 24, 400
    st = stream.State(cores=G, P=[], Q=[], sketch=sketch, m=m)
    if sketch == "leverage":
        st.p = [stream.leverage_probs(g) for g in G]
    samples = []
    for seed in range(reps):
        st.idxs = np.zeros((m, 3), dtype=np.int64)
        for k in range(1, 4):
            st.seed = seed
            st.idxs[:, k - 1] = stream._draw(st, k, dims[k - 1], 0)
        if sketch == "ksrft":
            D = [philox.signs(seed, d, k + 1, 0) for k, d in enumerate(dims)]
            Gs = stream.sampled_subchain([stream.dft_mix_core(g, D[k]) for k, g in enumerate(G)], st.idxs, n)
            Xs = stream.dft_unmix(stream.sampled_fibres(stream.dft_mix(X, D), st.idxs, n), D[n - 1])
        else:
            Gs = stream.sampled_subchain(G, st.idxs, n)
            Xs = stream.sampled_fibres(X, st.idxs, n)
        dP, _ = stream._pq_increment(Xs, Gs, stream.sketch_weights(st, n, dims))
        samples.append(dP)
    S = np.array(samples)
    mean, se = S.mean(0), S.std(0, ddof=1) / np.sqrt(reps)
    exact = tr.mttkrp(X, G, n)
    assert np.all(np.abs(mean - exact) <= 4.5 * se + 1e-12)


def _cartesian_rows(dims):
    """Every multi-index (i_1, .., i_N) once, i_1 fastest: m = prod(dims) rows."""
    N = len(dims)
    out = np.empty((int(np.prod(dims)), N), dtype=np.int64)
    for s in range(out.shape[0]):
        r = s
        for k in range(N):
            out[s, k] = r % dims[k]
            r //= dims[k]
    return out


@pytest.mark.parametrize("sketch", ["uniform", "ksrft"])
def test_rstr_with_full_index_set_equals_str(sketch, monkeypatch):
    """Full-index-set special case of the sketched updates (Alg. 5 with the
    schedules of Algs. 7 and 9): if every draw returns the whole Cartesian index
    set (m = I_1 .. I_{N-1} t_new rows, so each subchain row of mode n appears
    I_n times and the rescale J_n / m is 1 / I_n), the sketched P_n, Q_n
    increments and the sketched temporal normal equations equal STR's exactly
    (for KSRFT because (x)_j F_j D_j is unitary), so rSTR-U and rSTR-K reproduce
    STR (Alg. 4), step after step, to rounding."""
    dims, T, ranks, t_new = (3, 4), 10, (2, 3, 2), 2
    G, X = _problem(dims, T, ranks, 26, noise=0.05)
    full = _cartesian_rows(dims + (t_new,))

    def draw_all(st, k, size, tau):
        assert size == full[:, k - 1].max() + 1
        return full[:, k - 1].copy()

    monkeypatch.setattr(stream, "_draw", draw_all)
    init = [G[0], G[1], G[2][:, :t_new, :]]
    rs = stream.rstr_init(X[..., :t_new], init, sketch, m=full.shape[0], seed=5)
    ex = stream.str_init(X[..., :t_new], init)
    for n in range(1, 3):
        np.testing.assert_allclose(rs.P[n - 1], ex.P[n - 1], rtol=1e-11, atol=1e-11)
        np.testing.assert_allclose(rs.Q[n - 1], ex.Q[n - 1], rtol=1e-11, atol=1e-11)
    for t0 in range(t_new, T, t_new):
        stream.rstr_update(rs, X[..., t0:t0 + t_new])
        stream.str_update(ex, X[..., t0:t0 + t_new])
        for k in range(3):
            assert np.linalg.norm(rs.cores[k] - ex.cores[k]) <= 1e-10 * np.linalg.norm(ex.cores[k])
    for n in range(1, 3):
        np.testing.assert_allclose(rs.P[n - 1], ex.P[n - 1], rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(rs.Q[n - 1], ex.Q[n - 1], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("sketch", ["uniform", "leverage", "ksrft"])
def test_rstr_tracks_a_noisy_stream(sketch):
    """Qualitative check (Sec. 4): rSTR stays close to STR on a noisy TR stream."""
    dims, T, ranks = (12, 10), 40, (2, 2, 2)
    G, X = _problem(dims, T, ranks, 18, noise=1e-3)
    init, _, _ = stream.tr_als_ne(X[..., :10], synth.gaussian_cores(dims + (10,), ranks, 218),
                                  tol=1e-12, max_it=80)
    st = stream.rstr_init(X[..., :10], init, sketch, m=150, seed=7)
    ex = stream.str_init(X[..., :10], init)
    for t0 in range(10, 40, 5):
        stream.rstr_update(st, X[..., t0:t0 + 5])
        stream.str_update(ex, X[..., t0:t0 + 5])
    e_r, e_s = tr.fit_error(X, st.cores), tr.fit_error(X, ex.cores)
    assert e_s < 1e-2 and e_r < 5e-2
    assert st.cores[2].shape[1] == T


def test_masked_loss_gradient_fd_and_closed_form():
    dims, ranks = (4, 3, 4, 3), (2, 3, 2, 2)
    G = synth.gaussian_cores(dims, ranks, 19)
    X = synth.gaussian_tensor(dims, 20)
    mask = synth.bernoulli_keep_mask(dims, 0.3, 21)
    g = masked_loss_grad(X, G, mask)
    for n in range(4):
        for idx in [(0, 0, 0), (1, 2, 1), (ranks[n] - 1, dims[n] - 1, ranks[(n + 1) % 4] - 1)]:
            h = 1e-6
            Gp = [c.copy() for c in G]
            Gm = [c.copy() for c in G]
            Gp[n][idx] += h
            Gm[n][idx] -= h
            fd = (masked_loss(X, Gp, mask) - masked_loss(X, Gm, mask)) / (2 * h)
            assert abs(fd - g[n][idx]) <= 1e-6 * max(1.0, abs(g[n][idx]))
    g1 = masked_loss_grad(X, G, None)
    cf = closed_form_grad(X, G)
    for a, b in zip(g1, cf):
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-10)
