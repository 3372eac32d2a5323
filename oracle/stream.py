"""Streaming TR decomposition (STR, Alg. 4) and its randomized variants
(rSTR-U / rSTR-L / rSTR-K, Algs. 7-9), step by step in FP64 on the CPU.

Test infrastructure only: see the package docstring.

Every step uses the plain primitives of ``oracle.tr``: the subchain is
materialised, the Gram matrix Q_n is formed explicitly from it, and each
core solve uses the symmetric pseudo-inverse.  Readings of points the paper
leaves open are marked "Reading:".
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence

import numpy as np

from . import philox
from .tr import (core_fold2, core_unfold2, fit_error, gram_explicit, mttkrp,
                 solve_pinv, subchain_unfold, tr_full, unfold_cyclic)

SKETCHES = ("uniform", "leverage", "ksrft")


@dataclasses.dataclass
class State:
    """STR / rSTR state: the cores, the complementary matrices P_n, Q_n
    (n = 1..N-1; Sec. 3.1 calls them complementary matrices) and, for rSTR,
    the current sample indices and leverage distributions."""
    cores: List[np.ndarray]            # G_1..G_N; G_N holds every temporal row so far
    P: List[np.ndarray]                # P_n, I_n x R_n R_{n+1}
    Q: List[np.ndarray]                # Q_n, R_n R_{n+1} x R_n R_{n+1}
    step: int = 0                      # time step tau (0 = after initialisation)
    sketch: Optional[str] = None       # None = STR
    m: int = 0
    seed: int = 0
    stream: int = 0
    rescale: bool = True
    idxs: Optional[np.ndarray] = None  # (m, N) 0-based row indices
    p: Optional[List[np.ndarray]] = None  # leverage distributions p_k (rSTR-L)

    @property
    def N(self) -> int:
        return len(self.cores)

    @property
    def ranks(self) -> List[int]:
        return [G.shape[0] for G in self.cores]


def _rank_pair(st_or_cores, n: int):
    cores = st_or_cores.cores if isinstance(st_or_cores, State) else st_or_cores
    N = len(cores)
    return cores[n - 1].shape[0], cores[n % N].shape[0]


# ----------------------------------------------------------------------------
# Initial decomposition: TR-ALS-NE (Alg. 2)
# ----------------------------------------------------------------------------
def tr_als_ne(X: np.ndarray, cores0: Sequence[np.ndarray], tol: float = 1e-8,
              max_it: int = 100):
    """Alg. 2: for n = 1..N, solve G_{n(2)} H^{!=n}_<2> = X_[n] G^{!=n}_[2].
    Stops when the relative error changes by less than tol between two
    iterations, or after max_it iterations (Sec. 4, init settings).
    Returns (cores, iterations, final relative error)."""
    cores = [np.array(G, dtype=np.float64, copy=True) for G in cores0]
    N = X.ndim
    prev = None
    err = None
    it = 0
    for it in range(1, max_it + 1):
        for n in range(1, N + 1):
            A = subchain_unfold(cores, n)
            H = A.T @ A                       # = (H^{!=n})_<2>, Proposition subchain_gram
            M = unfold_cyclic(X, n) @ A
            Rn, Rn1 = _rank_pair(cores, n)
            cores[n - 1] = core_fold2(solve_pinv(M, H), Rn, Rn1)
        err = fit_error(X, cores)
        if prev is not None and abs(prev - err) < tol:
            break
        prev = err
    return cores, it, err


# ----------------------------------------------------------------------------
# STR (Alg. 4)
# ----------------------------------------------------------------------------
def str_init(X0: np.ndarray, cores: Sequence[np.ndarray]) -> State:
    """Initialisation stage of Alg. 4 with given initial cores:
    P_n = X_[n]^init G^{!=n}_[2], Q_n = Gram of G^{!=n}_[2], n = 1..N-1.
    Reading: Q_n's ring includes Z_N of the initial temporal core."""
    cores = [np.array(G, dtype=np.float64, copy=True) for G in cores]
    N = X0.ndim
    assert cores[N - 1].shape[1] == X0.shape[N - 1]
    P = [mttkrp(X0, cores, n) for n in range(1, N)]
    Q = [gram_explicit(cores, n) for n in range(1, N)]
    return State(cores=cores, P=P, Q=Q)


def str_update(st: State, Xnew: np.ndarray, sweeps: int = 1) -> State:
    """One time step of Alg. 4 (its update stage).

    Temporal mode: G_N^new = X^new_[N] G^{!=N}_[2] (H^{!=N}_<2>)^dagger, rows appended.
    Spatial modes n = 1..N-1 in order (later modes see the updated cores):
    P_n += X^new_[n] (G^{!=n}_new)_[2], Q_n += Gram of (G^{!=n}_new)_[2],
    G_{n(2)} = P_n Q_n^dagger.
    Reading (sweeps > 1): P_n, Q_n from before the step are kept; each sweep
    recomputes G_N^new and then sets P_n = P_n^old + increment from the
    current cores.  sweeps = 1 is exactly Alg. 4."""
    N = st.N
    assert Xnew.ndim == N
    P_old = [p.copy() for p in st.P]
    Q_old = [q.copy() for q in st.Q]
    GN_old = st.cores[N - 1]
    cur = list(st.cores)
    GN_new = None
    for _ in range(max(1, sweeps)):
        # temporal mode first; the subchain uses G_1..G_{N-1} only
        A = subchain_unfold(cur, N)
        M = unfold_cyclic(Xnew, N) @ A
        RN, R1 = _rank_pair(cur, N)
        GN_new = core_fold2(solve_pinv(M, A.T @ A), RN, R1)
        cur[N - 1] = GN_new
        # then the spatial modes in order
        for n in range(1, N):
            A = subchain_unfold(cur, n)
            st.P[n - 1] = P_old[n - 1] + unfold_cyclic(Xnew, n) @ A
            st.Q[n - 1] = Q_old[n - 1] + A.T @ A
            Rn, Rn1 = _rank_pair(cur, n)
            cur[n - 1] = core_fold2(solve_pinv(st.P[n - 1], st.Q[n - 1]), Rn, Rn1)
    cur[N - 1] = np.concatenate([GN_old, GN_new], axis=1)
    st.cores = cur
    st.step += 1
    return st


# ----------------------------------------------------------------------------
# Sketch building blocks (Alg. 3, Eq. sampDS, Lemma lev_est, Definition SRFT)
# ----------------------------------------------------------------------------
def leverage_probs(G: np.ndarray, rcond: float = 1e-12) -> np.ndarray:
    """p(i) = l_i(G_{(2)}) / rank(G_{(2)}) (Lemma lev_est), with the leverage
    scores l_i = ||U(i,:)||^2 of an orthonormal basis U of the column space
    (Definition of leverage scores) from a thin SVD; numerical rank at rcond."""
    A = core_unfold2(G)
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    r = int(np.sum(s > rcond * s[0])) if s.size and s[0] > 0 else 0
    if r == 0:
        return np.full(A.shape[0], 1.0 / A.shape[0])
    lev = np.sum(U[:, :r] ** 2, axis=1)
    return lev / r


def sampled_subchain(cores: Sequence[np.ndarray], idxs: np.ndarray, n: int) -> np.ndarray:
    """Alg. 3: start from identity slices and take the slices-Hadamard
    product with G_k(:, idxs(:,k), :) for k = n+1..N, 1..n-1.  Returns the
    sampled subchain's mode-2 unfolding, m x R_n R_{n+1}, column r_n + R_n r_{n+1}."""
    N = len(cores)
    m = idxs.shape[0]
    Rn, Rn1 = cores[(n - 2) % N].shape[2], cores[n % N].shape[0]   # G_n itself is not used
    dtype = np.result_type(*[G.dtype for k, G in enumerate(cores) if k != n - 1])
    S = np.broadcast_to(np.eye(Rn1, dtype=dtype), (m, Rn1, Rn1)).copy()
    for k0 in [(n + t) % N for t in range(N - 1)]:          # 0-based modes n+1..N,1..n-1
        Gk = cores[k0][:, idxs[:, k0], :]                    # (R_k, m, R_{k+1})
        S = np.einsum("sab,bsc->sac", S, Gk)                 # (A [*]_2 B)(s) = A(s) B(s)
    # S[s] is R_{n+1} x R_n; unfold: column a + R_n * b holds S[s][b, a]
    out = np.empty((m, Rn * Rn1), dtype=dtype)
    for b in range(Rn1):
        for a in range(Rn):
            out[:, a + Rn * b] = S[:, b, a]
    return out


def sampled_fibres(X: np.ndarray, idxs: np.ndarray, n: int) -> np.ndarray:
    """Alg. 3: X_S[n](i_n, s) = X(idxs(s,1), .., i_n, .., idxs(s,N)); I_n x m."""
    N = X.ndim
    m = idxs.shape[0]
    out = np.empty((X.shape[n - 1], m), dtype=X.dtype)
    for s in range(m):
        index = [int(idxs[s, k]) for k in range(N)]
        index[n - 1] = slice(None)
        out[:, s] = X[tuple(index)]
    return out


def sketch_weights(st: State, n: int, dims: Sequence[int], sketch_p=None) -> np.ndarray:
    """Squared diagonal of the rescaling D_n (Eq. sampDS and the KSRFT scale),
    applied to both P_n and Q_n increments.  Reading: rescaling is on by default;
    rescale=False reproduces the paper's "can be ignored" practice."""
    m = st.idxs.shape[0]
    if not st.rescale:
        return np.ones(m)
    N = len(dims)
    if st.sketch in ("uniform", "ksrft"):
        J = 1
        for k in range(N):
            if k != n - 1:
                J *= dims[k]
        return np.full(m, J / m)
    q = np.ones(m)
    for k in range(N):
        if k != n - 1:
            q = q * st.p[k][st.idxs[:, k]]
    return 1.0 / (m * q)


def dft_mix(X: np.ndarray, D: Sequence[np.ndarray]) -> np.ndarray:
    """X x_1 (F_1 D_1) x_2 .. x_N (F_N D_N), F_j the unitary DFT (Definition SRFT)."""
    Y = X.astype(np.complex128)
    for j, d in enumerate(D):
        shape = [1] * Y.ndim
        shape[j] = -1
        Y = np.fft.fft(Y * d.reshape(shape), axis=j, norm="ortho")
    return Y


def dft_mix_core(G: np.ndarray, d: np.ndarray) -> np.ndarray:
    """G x_2 (F D): mix a core along its physical index."""
    return np.fft.fft(G * d[None, :, None], axis=1, norm="ortho")


def dft_unmix(fib: np.ndarray, d: np.ndarray) -> np.ndarray:
    """D F^* applied along the first axis of the sampled fibres (Alg. 6)."""
    return d[:, None] * np.fft.ifft(fib, axis=0, norm="ortho")


def _draw(st: State, k: int, size: int, tau: int) -> np.ndarray:
    if st.sketch == "leverage":
        return philox.weighted_indices(st.seed, st.m, st.p[k - 1], k, tau, st.stream)
    return philox.uniform_indices(st.seed, st.m, size, k, tau, st.stream)


def _pq_increment(Xs: np.ndarray, Gs: np.ndarray, w: np.ndarray):
    """Real parts of X_S diag(w) conj(G_S) and G_S^T diag(w) conj(G_S) (Sec. 3.3
    KSRFT updates; for real sketches conj is the identity)."""
    dP = np.real((Xs * w[None, :]) @ np.conj(Gs))
    dQ = np.real(Gs.T @ (w[:, None] * np.conj(Gs)))
    return dP, dQ


# ----------------------------------------------------------------------------
# rSTR (Alg. 5 with the schedules of Algs. 7, 8, 9)
# ----------------------------------------------------------------------------
def rstr_init(X0: np.ndarray, cores: Sequence[np.ndarray], sketch: str, m: int, seed: int,
              rescale: bool = True, stream: int = 0) -> State:
    """Initialisation stage of Algs. 7-9 with given initial cores: draw idxs(:,k)
    for k = 1..N at tau = 0 (rSTR-L from p_k of every core; rSTR-K after mixing
    the cores and X^init with fresh signs), then P_n, Q_n from the sketch."""
    assert sketch in SKETCHES
    N = X0.ndim
    st = State(cores=[np.array(G, dtype=np.float64, copy=True) for G in cores],
               P=[None] * (N - 1), Q=[None] * (N - 1), sketch=sketch, m=m, seed=seed,
               stream=stream, rescale=rescale)
    dims = X0.shape
    if sketch == "leverage":
        st.p = [leverage_probs(G) for G in st.cores]
    st.idxs = np.zeros((m, N), dtype=np.int64)
    for k in range(1, N + 1):
        st.idxs[:, k - 1] = _draw(st, k, dims[k - 1], 0)
    if sketch == "ksrft":
        D = [philox.signs(seed, dims[j], j + 1, 0, stream) for j in range(N)]
        src = dft_mix(X0, D)
        cs = [dft_mix_core(G, D[j]) for j, G in enumerate(st.cores)]
    else:
        src, cs = X0, st.cores
    for n in range(1, N):
        Gs = sampled_subchain(cs, st.idxs, n)
        Xs = sampled_fibres(src, st.idxs, n)
        if sketch == "ksrft":
            Xs = dft_unmix(Xs, D[n - 1])
        st.P[n - 1], st.Q[n - 1] = _pq_increment(Xs, Gs, sketch_weights(st, n, dims))
    return st


def rstr_update(st: State, Xnew: np.ndarray) -> State:
    """One time step of Alg. 7 (uniform), Alg. 8 (leverage) or Alg. 9 (KSRFT)."""
    N = st.N
    st.step += 1
    tau = st.step
    dims = Xnew.shape
    tn = dims[N - 1]
    ks = st.sketch == "ksrft"
    cur = list(st.cores)
    if ks:
        # Alg. 9: new signs every step, mix the slab and the spatial cores
        D = [philox.signs(st.seed, dims[j], j + 1, tau, st.stream) for j in range(N)]
        src = dft_mix(Xnew, D)
        mixed = [dft_mix_core(cur[j], D[j]) for j in range(N - 1)] + [None]
    else:
        src = Xnew
    # ---- temporal mode ----
    cs = mixed if ks else cur
    Gs = sampled_subchain(cs, st.idxs, N)
    Xs = sampled_fibres(src, st.idxs, N)                # t_new x m
    if ks:
        Xs = dft_unmix(Xs, D[N - 1])
    w = sketch_weights(st, N, dims)
    # Reading (rSTR-K temporal update): the real normal equations
    # Re(X_S conj G_S) Re(G_S^T conj G_S)^dagger; for real sketches this is
    # X_S (G_S^T)^dagger of Algs. 7/8 with the row weights.
    dP, dQ = _pq_increment(Xs, Gs, w)
    RN, R1 = _rank_pair(cur, N)
    GN_new = core_fold2(solve_pinv(dP, dQ), RN, R1)
    cur[N - 1] = GN_new
    if st.sketch == "leverage":
        st.p[N - 1] = leverage_probs(GN_new)
    st.idxs[:, N - 1] = _draw(st, N, tn, tau)
    if ks:
        mixed[N - 1] = dft_mix_core(GN_new, D[N - 1])
    # ---- spatial modes ----
    for n in range(1, N):
        cs = mixed if ks else cur
        Gs = sampled_subchain(cs, st.idxs, n)
        Xs = sampled_fibres(src, st.idxs, n)
        if ks:
            Xs = dft_unmix(Xs, D[n - 1])
        dP, dQ = _pq_increment(Xs, Gs, sketch_weights(st, n, dims))
        st.P[n - 1] = st.P[n - 1] + dP
        st.Q[n - 1] = st.Q[n - 1] + dQ
        Rn, Rn1 = _rank_pair(cur, n)
        cur[n - 1] = core_fold2(solve_pinv(st.P[n - 1], st.Q[n - 1]), Rn, Rn1)
        if st.sketch == "leverage":
            st.p[n - 1] = leverage_probs(cur[n - 1])
        st.idxs[:, n - 1] = _draw(st, n, dims[n - 1], tau)
        if ks:
            mixed[n - 1] = dft_mix_core(cur[n - 1], D[n - 1])
    GN_all = np.concatenate([st.cores[N - 1], GN_new], axis=1)
    cur[N - 1] = GN_all
    st.cores = cur
    return st


def reconstruct(st: State, t0: int = 0, t1: Optional[int] = None) -> np.ndarray:
    """TR(G) over temporal rows [t0, t1) (Sec. 1, TR format)."""
    cores = list(st.cores)
    cores[-1] = cores[-1][:, t0:t1, :]
    return tr_full(cores)
