"""Tensor-ring primitives, written out from their definitions (FP64, CPU).

Test infrastructure only: see the package docstring.

Conventions (Sec. 2 of the paper):
* cores ``G[n]`` have shape (R_n, I_n, R_{n+1}); the lateral slice
  G_n(i_n) = G[n][:, i_n, :] is an R_n x R_{n+1} matrix; R_{N+1} = R_1.
* the linear index of (i_1, ..., i_N) has i_1 fastest (Sec. 2, first
  paragraph); the functions below take the paper's 1-based mode number n.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


# ----------------------------------------------------------------------------
# TR format (Sec. 1, the defining trace formula)
# ----------------------------------------------------------------------------
def tr_entry(cores: Sequence[np.ndarray], idx: Sequence[int]) -> float:
    """X(i_1..i_N) = Trace(G_1(i_1) G_2(i_2) ... G_N(i_N))."""
    m = np.eye(cores[0].shape[0])
    for G, i in zip(cores, idx):
        m = m @ G[:, i, :]
    return float(np.trace(m))


def tr_full(cores: Sequence[np.ndarray]) -> np.ndarray:
    """The full tensor TR({G_n}) as an array indexed X[i_1, ..., i_N].

    Same trace formula as tr_entry, evaluated for all indices at once: the
    slices of G_1..G_{N-1} are multiplied left to right (one library
    contraction per core), then the last core's slice is multiplied in and the
    trace taken in one contraction (R_{N+1} = R_1).
    """
    T = cores[0]                                   # (R_1, I_1, R_2)
    for G in cores[1:-1]:
        T = np.tensordot(T, G, axes=([T.ndim - 1], [0]))   # (R_1, I_1, .., I_k, R_{k+1})
    GN = cores[-1]                                 # (R_N, I_N, R_1)
    R1 = T.shape[0]
    RN = T.shape[-1]
    lead = T.shape[1:-1]
    A = np.moveaxis(T, 0, -1).reshape(int(np.prod(lead)), RN * R1)   # (i_1..i_{N-1}), (r_N, r_1)
    B = GN.transpose(0, 2, 1).reshape(RN * R1, GN.shape[1])          # (r_N, r_1), i_N
    return (A @ B).reshape(tuple(lead) + (GN.shape[1],))


# ----------------------------------------------------------------------------
# Unfoldings (Definition of the three unfoldings, Sec. 2)
# ----------------------------------------------------------------------------
def _fortran_columns(A: np.ndarray, lead: int) -> np.ndarray:
    """Reshape so the first `lead` axes form rows and the rest form columns,
    both with the earliest axis fastest (the paper's linear index)."""
    rows = int(np.prod(A.shape[:lead])) if lead else 1
    return np.reshape(A, (rows, -1), order="F")


def unfold_cyclic(X: np.ndarray, n: int) -> np.ndarray:
    """Mode-n unfolding X_[n]: row i_n, column overline{i_{n+1}..i_N i_1..i_{n-1}}."""
    N = X.ndim
    axes = [(n - 1 + k) % N for k in range(N)]     # n, n+1, .., N, 1, .., n-1
    return _fortran_columns(np.transpose(X, axes), 1)


def unfold_classical(X: np.ndarray, n: int) -> np.ndarray:
    """Classical mode-n unfolding X_(n): column overline{i_1..i_{n-1} i_{n+1}..i_N}."""
    N = X.ndim
    axes = [n - 1] + [k for k in range(N) if k != n - 1]
    return _fortran_columns(np.transpose(X, axes), 1)


def unfold_n(X: np.ndarray, n: int) -> np.ndarray:
    """n-unfolding X_<n>: row overline{i_1..i_n}, column overline{i_{n+1}..i_N}."""
    return _fortran_columns(X, n)


def core_unfold2(G: np.ndarray) -> np.ndarray:
    """G_{n(2)} in R^{I_n x R_n R_{n+1}}: classical mode-2 unfolding of a core,
    column c = r_n + R_n * r_{n+1}."""
    return unfold_classical(G, 2)


def core_fold2(M: np.ndarray, Rn: int, Rn1: int) -> np.ndarray:
    """Inverse of core_unfold2: (I_n, R_n R_{n+1}) -> (R_n, I_n, R_{n+1})."""
    In = M.shape[0]
    G = np.empty((Rn, In, Rn1))
    for b in range(Rn1):
        for a in range(Rn):
            G[a, :, b] = M[:, a + Rn * b]
    return G


# ----------------------------------------------------------------------------
# Subchain tensor (Definition of the subchain tensor, Sec. 2; Eq. subchain_new)
# ----------------------------------------------------------------------------
def subchain_tensor(cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """G^{!=n} in R^{R_{n+1} x J_n x R_n}: slice j = overline{i_{n+1}..i_N i_1..i_{n-1}}
    equals G_{n+1}(i_{n+1}) ... G_N(i_N) G_1(i_1) ... G_{n-1}(i_{n-1}).

    Built as the mode-2 subchain product G_{n+1} [x]_2 ... [x]_2 G_{n-1}
    (Definition of the subchain product: (A [x]_2 B)(overline{j1 j2}) = A(j1) B(j2),
    j1 fastest)."""
    N = len(cores)
    order = [(n + k) % N for k in range(N - 1)]    # 0-based: n+1, .., N, 1, .., n-1
    T = cores[order[0]]
    for k in order[1:]:
        T = subchain_product(T, cores[k])
    return T


def subchain_product(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """A [x]_2 B for A (I1, J1, K) and B (K, J2, I2): slice overline{j1 j2} = A(j1) B(j2)."""
    I1, J1, K = A.shape
    K2, J2, I2 = B.shape
    assert K == K2
    out = np.empty((I1, J1 * J2, I2))
    for j2 in range(J2):
        # columns j1 + J1*j2, j1 fastest
        out[:, j2 * J1:(j2 + 1) * J1, :] = np.einsum("ajk,kb->ajb", A, B[:, j2, :])
    return out


def subchain_unfold(cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """G^{!=n}_[2] in R^{J_n x R_n R_{n+1}}: mode-2 unfolding of the subchain tensor,
    column c = r_n + R_n r_{n+1}, entry G^{!=n}(j)[r_{n+1}, r_n]."""
    return unfold_cyclic(subchain_tensor(cores, n), 2)


# ----------------------------------------------------------------------------
# Gram tensors and the structured Gram (Alg. 2; Proposition subchain_gram)
# ----------------------------------------------------------------------------
def gram_Z(G: np.ndarray) -> np.ndarray:
    """Z = sum_i G(i)^T o G(i)^T, shape (R_{n+1}, R_n, R_{n+1}, R_n) (Alg. 2)."""
    Rn, In, Rn1 = G.shape
    Z = np.zeros((Rn1, Rn, Rn1, Rn))
    for i in range(In):
        Gt = G[:, i, :].T
        Z += np.multiply.outer(Gt, Gt)
    return Z


def contract_2413(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """General contracted tensor product A x_{2,4}^{1,3} B:
    (i1, i2, r1, r2) = sum_{j,k} A(i1, j, r1, k) B(j, i2, k, r2)."""
    return np.einsum("ajrk,jbks->abrs", A, B)


def ring_H(cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """H^{!=n} = Z_{n-1} x Z_{n-2} x .. x Z_1 x Z_N x .. x Z_{n+1} (Alg. 2),
    each x being x_{2,4}^{1,3}; shape (R_n, R_{n+1}, R_n, R_{n+1})."""
    N = len(cores)
    order = [(n - 2 - k) % N for k in range(N - 1)]   # 0-based n-1, .., 1, N, .., n+1
    H = gram_Z(cores[order[0]])
    for k in order[1:]:
        H = contract_2413(H, gram_Z(cores[k]))
    return H


def unfold_2(H: np.ndarray) -> np.ndarray:
    """H_<2>: rows overline{h1 h2}, columns overline{h3 h4}."""
    return unfold_n(H, 2)


def gram_structured(cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """Q_n = (H^{!=n})_<2> via the Gram tensors (Proposition subchain_gram)."""
    return unfold_2(ring_H(cores, n))


def gram_explicit(cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """Q_n = (G^{!=n}_[2])^T G^{!=n}_[2] from the materialised subchain (Eq. partial)."""
    A = subchain_unfold(cores, n)
    return A.T @ A


def mttkrp(X: np.ndarray, cores: Sequence[np.ndarray], n: int) -> np.ndarray:
    """P = X_[n] G^{!=n}_[2] (Eq. partial; Alg. 2)."""
    return unfold_cyclic(X, n) @ subchain_unfold(cores, n)


# ----------------------------------------------------------------------------
# Solve and error
# ----------------------------------------------------------------------------
def solve_pinv(P: np.ndarray, Q: np.ndarray) -> np.ndarray:
    """G_{n(2)} = P Q^dagger with the symmetric pseudo-inverse (Alg. 4);
    default cut-off max(dim) * eps relative to the largest eigenvalue."""
    return P @ np.linalg.pinv(Q, hermitian=True)


def fit_error(X: np.ndarray, cores: Sequence[np.ndarray]) -> float:
    """||X - TR(G)||_F / ||X||_F by the direct residual (Sec. 4, protocol)."""
    return float(np.linalg.norm(X - tr_full(cores)) / np.linalg.norm(X))


def ttm(X: np.ndarray, U: np.ndarray, n: int) -> np.ndarray:
    """(X x_n U)(.., j, ..) = sum_{i_n} X(.., i_n, ..) U(j, i_n) (Definition TTM)."""
    Y = np.tensordot(U, X, axes=([1], [n - 1]))   # j first
    return np.moveaxis(Y, 0, n - 1)
