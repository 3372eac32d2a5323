"""Pins for the oracle's tensor-ring primitives (CPU only).

Each test ties an oracle function to something other than itself: a brute
force loop over the definition, a hand-worked example, an identity of the
paper (Proposition subchain_gram, Eq. prop:ttm) or a library routine.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg

import synth
from oracle import tr

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cores(dims, ranks, seed=0):
    return synth.gaussian_cores(dims, ranks, seed)


def _lin(idx, dims):
    """1-based-paper linear index, i_1 fastest (0-based here)."""
    out, stride = 0, 1
    for i, d in zip(idx, dims):
        out += i * stride
        stride *= d
    return out


def test_tr_full_hand_example():
    """TR format (Sec. 1) against a hand-worked 2x2x2 example."""
    s = {
        1: [np.eye(2), np.array([[0, 1], [1, 0]])],
        2: [np.diag([1.0, 2.0]), np.array([[1, 1], [0, 1]])],
        3: [np.eye(2), np.array([[0, 1], [1, 0]])],
    }
    cores = [np.stack([np.asarray(m, float) for m in s[k]], axis=1) for k in (1, 2, 3)]
    rows = np.loadtxt(os.path.join(GOLDEN, "tr_hand_example.txt"))
    X = tr.tr_full(cores)
    for i1, i2, i3, v in rows:
        assert X[int(i1), int(i2), int(i3)] == v
        assert tr.tr_entry(cores, (int(i1), int(i2), int(i3))) == v


@pytest.mark.parametrize("dims,ranks", [((3, 4, 5, 2), (2, 3, 2, 3)), ((4, 3, 2), (3, 1, 2))])
def test_tr_full_brute_force(dims, ranks):
    G = _cores(dims, ranks)
    X = tr.tr_full(G)
    for idx in itertools.product(*[range(d) for d in dims]):
        m = np.eye(ranks[0])
        for n, i in enumerate(idx):
            m = m @ G[n][:, i, :]
        assert abs(X[idx] - np.trace(m)) <= 1e-12 * (1 + abs(X[idx]))


def test_circular_invariance():
    """Rotating modes and cores by k rotates the tensor (Sec. 1)."""
    dims, ranks = (3, 4, 5, 2), (2, 3, 4, 3)
    G = _cores(dims, ranks, 1)
    X = tr.tr_full(G)
    for k in range(1, 4):
        Gr = G[k:] + G[:k]
        Xr = tr.tr_full(Gr)
        np.testing.assert_allclose(Xr, np.transpose(X, [(k + a) % 4 for a in range(4)]),
                                   rtol=1e-12, atol=1e-12)


def test_unfoldings_by_definition():
    dims = (2, 3, 4, 5)
    X = synth.gaussian_tensor(dims, 3)
    N = len(dims)
    for n in range(1, N + 1):
        Xc, Xk, Xa = tr.unfold_cyclic(X, n), tr.unfold_classical(X, n), tr.unfold_n(X, n)
        for idx in itertools.product(*[range(d) for d in dims]):
            cyc = [(n + t) % N for t in range(N - 1)]
            col_c = _lin([idx[k] for k in cyc], [dims[k] for k in cyc])
            cls = [k for k in range(N) if k != n - 1]
            col_k = _lin([idx[k] for k in cls], [dims[k] for k in cls])
            assert Xc[idx[n - 1], col_c] == X[idx]
            assert Xk[idx[n - 1], col_k] == X[idx]
            row_a = _lin(idx[:n], dims[:n])
            col_a = _lin(idx[n:], dims[n:])
            assert Xa[row_a, col_a] == X[idx]


def test_core_unfold_fold_roundtrip():
    G = _cores((5,), (3,), 2)[0]
    G = np.random.default_rng(0).standard_normal((3, 5, 4))
    M = tr.core_unfold2(G)
    for a, i, b in itertools.product(range(3), range(5), range(4)):
        assert M[i, a + 3 * b] == G[a, i, b]
    np.testing.assert_array_equal(tr.core_fold2(M, 3, 4), G)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_subchain_and_mttkrp_brute_force(n):
    """G^{!=n}_[2] entries and X_[n] G^{!=n}_[2] by nested loops over the definition."""
    dims, ranks = (3, 4, 2, 2), (2, 3, 2, 3)
    G = _cores(dims, ranks, 4)
    N = 4
    X = synth.gaussian_tensor(dims, 5)
    A = tr.subchain_unfold(G, n)
    P = tr.mttkrp(X, G, n)
    Rn, Rn1 = ranks[n - 1], ranks[n % N]
    cyc = [(n + t) % N for t in range(N - 1)]
    Pb = np.zeros((dims[n - 1], Rn * Rn1))
    for idx in itertools.product(*[range(d) for d in dims]):
        m = np.eye(Rn1)
        for k in cyc:
            m = m @ G[k][:, idx[k], :]
        j = _lin([idx[k] for k in cyc], [dims[k] for k in cyc])
        for a in range(Rn):
            for b in range(Rn1):
                assert abs(A[j, a + Rn * b] - m[b, a]) <= 1e-12
                Pb[idx[n - 1], a + Rn * b] += X[idx] * m[b, a]
    np.testing.assert_allclose(P, Pb, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("dims,ranks", [((3, 4, 5, 2), (2, 3, 2, 3)), ((5, 4, 3), (3, 2, 4)),
                                        ((2, 3, 2, 3, 2), (2, 2, 3, 2, 2))])
def test_structured_gram_equals_explicit(dims, ranks):
    """Proposition subchain_gram: the Z-ring Gram equals the explicit Gram."""
    G = _cores(dims, ranks, 6)
    for n in range(1, len(dims) + 1):
        Qe = tr.gram_explicit(G, n)
        Qs = tr.gram_structured(G, n)
        assert np.abs(Qe - Qs).max() <= 1e-13 * np.abs(Qe).max()


def test_unfolding_reproduces_tensor():
    """X_[n] = G_{n(2)} (G^{!=n}_[2])^T (Eq. tr_als) for an exact TR tensor."""
    dims, ranks = (3, 4, 5, 2), (2, 3, 2, 3)
    G = _cores(dims, ranks, 7)
    X = tr.tr_full(G)
    for n in range(1, 5):
        lhs = tr.unfold_cyclic(X, n)
        rhs = tr.core_unfold2(G[n - 1]) @ tr.subchain_unfold(G, n).T
        np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)


def test_multi_ttm_unfolding_identity():
    """Eq. prop:ttm: Y_[n] = U_n X_[n] (U_{n-1} (x) .. (x) U_1 (x) U_N (x) .. (x) U_{n+1})^T."""
    dims = (2, 3, 4)
    X = synth.gaussian_tensor(dims, 8)
    rng = np.random.default_rng(9)
    U = [rng.standard_normal((d + 1, d)) for d in dims]
    Y = X
    for n in range(1, 4):
        Y = tr.ttm(Y, U[n - 1], n)
    for n in range(1, 4):
        order = [(n - 2 - t) % 3 for t in range(2)]   # n-1, .., 1, N, .., n+1
        K = U[order[0]]
        for k in order[1:]:
            K = np.kron(K, U[k])
        np.testing.assert_allclose(tr.unfold_cyclic(Y, n),
                                   U[n - 1] @ tr.unfold_cyclic(X, n) @ K.T, rtol=1e-12, atol=1e-12)


def test_solve_matches_cholesky():
    """Q^dagger by pinv equals the Cholesky solve when Q is well conditioned."""
    rng = np.random.default_rng(10)
    A = rng.standard_normal((200, 16))
    Q = A.T @ A
    P = rng.standard_normal((7, 16))
    G1 = tr.solve_pinv(P, Q)
    G2 = scipy.linalg.cho_solve(scipy.linalg.cho_factor(Q), P.T).T
    np.testing.assert_allclose(G1, G2, rtol=1e-10, atol=1e-12)


def test_fit_error_gram_identity():
    """Direct residual vs ||X||^2 - 2<X, Xh> + ||Xh||^2 on a well-separated case."""
    dims, ranks = (4, 5, 6), (2, 3, 2)
    G = _cores(dims, ranks, 11)
    X = synth.gaussian_tensor(dims, 12)
    Xh = tr.tr_full(G)
    direct = tr.fit_error(X, G)
    gram = np.sqrt(np.sum(X * X) - 2 * np.sum(X * Xh) + np.sum(Xh * Xh)) / np.linalg.norm(X)
    assert abs(direct - gram) <= 1e-12 * gram


def test_rank_one_reduces_to_outer_product():
    """R = 1: TR is the outer product, Q_n = prod_{k!=n} ||g_k||^2 and
    P_n = X x_{k!=n} g_k (rank-one CP / higher-order power iteration)."""
    dims = (3, 4, 5)
    G = _cores(dims, (1, 1, 1), 13)
    g = [Gk[0, :, 0] for Gk in G]
    np.testing.assert_allclose(tr.tr_full(G), np.einsum("i,j,k->ijk", *g), rtol=1e-13)
    X = synth.gaussian_tensor(dims, 14)
    for n in range(1, 4):
        others = [g[k] for k in range(3) if k != n - 1]
        q = np.prod([v @ v for v in others])
        assert abs(tr.gram_explicit(G, n)[0, 0] - q) <= 1e-12 * q
        sub = "ijk"
        spec = f"ijk,{sub[[k for k in range(3) if k != n - 1][0]]},{sub[[k for k in range(3) if k != n - 1][1]]}->{sub[n - 1]}"
        np.testing.assert_allclose(tr.mttkrp(X, G, n)[:, 0], np.einsum(spec, X, *others), rtol=1e-12)
