// FP64 kernels for the structured Gram and the small normal equations.
//
//   core Gram        M = G_{(2)}^T G_{(2)},   transfer form E = sum_i G(i) (x) G(i)
//                    (the Gram tensor Z of Alg. 2, with its indices permuted)
//   ring             W = E_{n+1} E_{n+2} ... E_{n-1}  gives  (H^{!=n})_<2>   (Prop. subchain_gram)
//   solve            G_{n(2)} = P_n Q_n^{-1} (Alg. 4): FP64 LDL^T + substitution, or
//                    (FP32 path) Q_n^{-1} from an FP32 symmetric sweep + FP64-residual refinement
//   leverage         l_i = g_i M^{-1} g_i^T with M = G_{(2)}^T G_{(2)} = L D L^T (Lemma lev_est)
#include <algorithm>

#include "kernels.cuh"
#include "ptx.cuh"

// ---------------------------------------------------------------------------
// core Gram: one (c, c') pair with c <= c' per group of 4 threads (each sums
// every 4th row; the partial sums are added in a fixed order); the rows of G
// are staged in shared memory in chunks (cp.async), so the FMA chains read
// shared memory.  Writes both halves.
// ---------------------------------------------------------------------------
// pairs 64 bx .. 64 bx + 63 of the upper triangle (bx: the block's index)
__device__ __forceinline__ void core_gram_body(const double* __restrict__ G, int64_t I, int Ra, int Rb,
                                               double* __restrict__ M, double* __restrict__ E, int chunk,
                                               int64_t bx) {
  extern __shared__ __align__(16) double sg[];   // chunk x RR
  __shared__ double red[4][64];
  const int RR = Ra * Rb;
  const int64_t npairs = (int64_t)RR * (RR + 1) / 2;
  const int p = threadIdx.x & 63, q = threadIdx.x >> 6;
  const int64_t t = bx * 64 + p;
  int c = 0, cp = 0;
  if (t < npairs) {
    // row c of the upper triangle starts at c RR - c (c - 1) / 2
    const double b2 = 2.0 * RR + 1.0;
    c = (int)floor((b2 - sqrt(b2 * b2 - 8.0 * (double)t)) * 0.5);
    if (c < 0) c = 0;
    while (c > 0 && (int64_t)c * RR - (int64_t)c * (c - 1) / 2 > t) --c;
    while ((int64_t)(c + 1) * RR - (int64_t)(c + 1) * c / 2 <= t) ++c;
    cp = c + (int)(t - ((int64_t)c * RR - (int64_t)c * (c - 1) / 2));
  }
  double s = 0.0;
  const bool vec = ((RR & 1) == 0) && ((((uintptr_t)G) & 15) == 0);
  for (int64_t i0 = 0; i0 < I; i0 += chunk) {
    const int nr = (int)min((int64_t)chunk, I - i0);
    const int64_t cnt = (int64_t)nr * RR;
    if (vec) {
      for (int64_t e = 2 * threadIdx.x; e < cnt; e += 2 * blockDim.x) cp_async16(&sg[e], &G[i0 * RR + e]);
    } else {
      for (int64_t e = threadIdx.x; e < cnt; e += blockDim.x) cp_async8(&sg[e], &G[i0 * RR + e]);
    }
    cp_async_wait_all();
    __syncthreads();
    if (t < npairs) {
      double s0 = 0.0, s1 = 0.0;
      int i = q;
      for (; i + 4 < nr; i += 8) {
        s0 = fma(sg[i * RR + c], sg[i * RR + cp], s0);
        s1 = fma(sg[(i + 4) * RR + c], sg[(i + 4) * RR + cp], s1);
      }
      if (i < nr) s0 = fma(sg[i * RR + c], sg[i * RR + cp], s0);
      s += s0 + s1;
    }
    __syncthreads();
  }
  red[q][p] = s;
  __syncthreads();
  if (q != 0 || t >= npairs) return;
  s = (red[0][p] + red[1][p]) + (red[2][p] + red[3][p]);
  if (M) { M[(int64_t)c * RR + cp] = s; M[(int64_t)cp * RR + c] = s; }
  if (E) {
    // c = a + Ra b, c' = a' + Ra b'  ->  E[(a + Ra a'), (b + Rb b')]
    const int a = c % Ra, b = c / Ra, ap = cp % Ra, bp = cp / Ra;
    const int64_t RR2 = (int64_t)Rb * Rb;
    E[(int64_t)(a + Ra * ap) * RR2 + (b + Rb * bp)] = s;
    E[(int64_t)(ap + Ra * a) * RR2 + (bp + Rb * b)] = s;
  }
}

__global__ void __launch_bounds__(256) core_gram_kernel(const double* __restrict__ G, int64_t I, int Ra,
                                                        int Rb, double* __restrict__ M,
                                                        double* __restrict__ E, int chunk) {
  PDL_ENTRY();
  core_gram_body(G, I, Ra, Rb, M, E, chunk, blockIdx.x);
}

// work list of core Grams: item = (job, pair block)
__global__ void __launch_bounds__(256) core_gram_batch_kernel(const GramJob* __restrict__ jobs,
                                                              const int2* __restrict__ items) {
  PDL_ENTRY();
  const int2 it = items[blockIdx.x];
  const GramJob j = jobs[it.x];
  core_gram_body(j.G, j.I, j.Ra, j.Rb, nullptr, j.E, j.chunk, it.y);
}

cudaError_t launch_core_gram(const double* G, int64_t I, int Ra, int Rb, double* M, double* E,
                             cudaStream_t s) {
  const int RR = Ra * Rb;
  const int64_t npairs = (int64_t)RR * (RR + 1) / 2;
  const int64_t blocks = std::max<int64_t>(1, (npairs + 63) / 64);
  // rows per staged chunk: at most 44 KB of dynamic shared memory (with the
  // kernel's static 2 KB, under the default 48 KB limit)
  const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(I, (44 * 1024) / (8 * (int64_t)RR)));
  const size_t sm = (size_t)chunk * RR * 8;
  launch_k(core_gram_kernel, (unsigned)blocks, 256, sm, s, G, I, Ra, Rb, M, E, chunk);
  return cudaGetLastError();
}

int core_gram_chunk(int64_t I, int RR) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(I, (44 * 1024) / (8 * (int64_t)RR)));
}

int core_gram_blocks(int RR) { return (int)std::max<int64_t>(1, ((int64_t)RR * (RR + 1) / 2 + 63) / 64); }

cudaError_t launch_core_gram_batch(const GramJob* jobs, const int2* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  launch_k(core_gram_batch_kernel, (unsigned)nitems, 256, (size_t)44 * 1024, s, jobs, items);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Inverse of an SPD matrix by the symmetric sweep (in-place Gauss-Jordan without
// pivoting; its pivots are the Schur-complement pivots of the LDL^T / Cholesky
// factorisation).  256 threads as a 16 x 16 grid; thread (ty, tx) keeps the
// entries (ty + 16a, tx + 16b), a, b < B, in registers.  Per pivot k the owners
// of column k publish it to shared memory (double-buffered), then every thread
// updates its entries: one barrier per pivot.  After n sweeps the matrix holds
// -Q^{-1}.
// ---------------------------------------------------------------------------
// orders served by the refined solve with the FP64 fallback (apply_df_kernel)
__host__ __device__ __forceinline__ bool apply_df_supported_d(int n) { return n >= 2 && n <= 128; }

// fast reciprocal for the FP32 inverse (CUDA's approximate division, <= 2 ulp):
// the FP32 inverse only seeds an FP64-residual refinement
__device__ __forceinline__ float recip_fast(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip_fast(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// Q read through ldq (FP64 or FP32 source; the fused form reads an FP32 copy
// written by other CTAs of the same kernel, past L1)
__device__ __forceinline__ float ldq(const float* p, bool cg) { return cg ? __ldcg(p) : *p; }
__device__ __forceinline__ double ldq(const double* p, bool cg) { return cg ? __ldcg(p) : *p; }

// flag_singular: a pivot <= n eps max(diag) sets DEV_ERR_SINGULAR.  When the
// refined solve that follows has the FP64 fallback (orders <= 128) the FP32
// inverse only reports the pivot ratio (0 for such a pivot) and the fallback
// decides singularity in FP64.
template <typename T, int B, typename SRC>
__device__ __forceinline__ void sweep_body(const SRC* __restrict__ Q, int n, T* __restrict__ W, int* status,
                                           double* pivot_ratio, bool cg, bool flag_singular) {
  __shared__ T col[2][16 * B];
  __shared__ T qd[16 * B];
  __shared__ T pivs[16 * B];   // pivot k as met (before any replacement)
  __shared__ T s_tol;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T a[B][B];
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      a[i][j] = (r < n && c < n) ? (T)ldq(Q + (int64_t)r * n + c, cg) : (T)0;
    }
  for (int k = tid; k < n; k += 256) qd[k] = (T)ldq(Q + (int64_t)k * n + k, cg);
  __syncthreads();
  if (tid < 32) {
    T mx = 0;
    for (int k = tid; k < n; k += 32) mx = mx > qd[k] ? mx : qd[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T o = __shfl_xor_sync(0xffffffffu, mx, off);
      mx = mx > o ? mx : o;
    }
    if (tid == 0) s_tol = (T)n * (T)(sizeof(T) == 8 ? 2.220446049250313e-16 : 1.1920928955078125e-07) * mx;
  }
  __syncthreads();
  const T tol = s_tol;
  // the pivot loop is unrolled over the register block index kb only, so that
  // the owners' selections a[.][kb] are static register accesses; the 16
  // pivots inside a block stay a loop (the fully unrolled form does not fit the
  // instruction cache and stalls on instruction fetch)
#pragma unroll
  for (int kb = 0; kb < B; ++kb) {
#pragma unroll 1
    for (int kr = 0; kr < 16; ++kr) {
      const int k = kb * 16 + kr;
      if (k >= n) break;
      const int par = k & 1;
      // padded rows hold zeros, so the owners publish every row of the column
      if (tx == kr) {
#pragma unroll
        for (int i = 0; i < B; ++i) col[par][ty + 16 * i] = a[i][kb];
      }
      __syncthreads();
      T piv = col[par][k];
      if (tid == 0) pivs[k] = piv;
      if (!(piv > tol)) piv = (T)1;   // recorded as singular after the loop
      const T rcp = recip_fast(piv);
      // generic update a_ij -= a_ik a_kj / a_kk for every owned entry, then the
      // owners of row k / column k overwrite theirs (row k and column k scale
      // by 1/a_kk, the pivot becomes -1/a_kk)
      T cir[B], cj[B];
#pragma unroll
      for (int i = 0; i < B; ++i) cir[i] = col[par][ty + 16 * i] * rcp;
#pragma unroll
      for (int j = 0; j < B; ++j) cj[j] = col[par][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) a[i][j] = fma_t(-cir[i], cj[j], a[i][j]);
      if (ty == kr) {
#pragma unroll
        for (int j = 0; j < B; ++j) a[kb][j] = cj[j] * rcp;
      }
      if (tx == kr) {
#pragma unroll
        for (int i = 0; i < B; ++i) a[i][kb] = cir[i];
        if (ty == kr) a[kb][kb] = -rcp;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      if (r < n && c < n) W[(int64_t)r * n + c] = -a[i][j];
    }
  // singular pivots and the smallest pivot / diagonal ratio
  __syncthreads();
  if (tid < 32) {
    int bad = 0;
    T ratio = (T)1;
    for (int k = tid; k < n; k += 32) {
      const T p = pivs[k];
      if (!(p > tol)) { bad = 1; ratio = (T)0; }
      else if (qd[k] > (T)0) {
        const T r = p / qd[k];
        ratio = r < ratio ? r : ratio;
      }
    }
    bad = __any_sync(0xffffffffu, bad);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T o = __shfl_xor_sync(0xffffffffu, ratio, off);
      ratio = o < ratio ? o : ratio;
    }
    if (tid == 0) {
      if (bad && status && flag_singular) atomicOr(status, DEV_ERR_SINGULAR);
      if (pivot_ratio) *pivot_ratio = (double)ratio;
    }
  }
}

// Blocked form of the symmetric sweep: PB pivots K = {k0 .. k0 + PB - 1} per
// barrier.  Sweeping a block of pivots equals sweeping them one after another
// (the sweep operator composes), so with P = A_KK (its LDL^T pivots are the
// Schur-complement pivots of the one-by-one sweep):
//   A_IJ -= A_IK P^{-1} A_KJ,  A_KJ <- P^{-1} A_KJ,  A_IK <- A_IK P^{-1},  A_KK <- -P^{-1}.
// Owners of the PB columns publish them (double-buffered, one barrier per
// block); every thread factors P in registers (LDL^T, PB x PB) and updates its
// B x B entries with a rank-PB product.  Padded pivots (k >= n) act as the
// identity.  After every block the matrix holds -Q^{-1} as in sweep_body.
template <typename T, int B, int PB, typename SRC>
__device__ __forceinline__ void sweep_body_blocked(const SRC* __restrict__ Q, int n, T* __restrict__ W,
                                                   int* status, double* pivot_ratio, bool cg,
                                                   bool flag_singular) {
  __shared__ T colb[2][PB][16 * B];
  __shared__ T qd[16 * B];
  __shared__ T pivs[16 * B];
  __shared__ T s_tol;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T a[B][B];
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      a[i][j] = (r < n && c < n) ? (T)ldq(Q + (int64_t)r * n + c, cg) : (T)0;
    }
  for (int k = tid; k < n; k += 256) qd[k] = (T)ldq(Q + (int64_t)k * n + k, cg);
  __syncthreads();
  if (tid < 32) {
    T mx = 0;
    for (int k = tid; k < n; k += 32) mx = mx > qd[k] ? mx : qd[k];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T o = __shfl_xor_sync(0xffffffffu, mx, off);
      mx = mx > o ? mx : o;
    }
    if (tid == 0) s_tol = (T)n * (T)(sizeof(T) == 8 ? 2.220446049250313e-16 : 1.1920928955078125e-07) * mx;
  }
  __syncthreads();
  const T tol = s_tol;
  int step = 0;
#pragma unroll
  for (int kb = 0; kb < B; ++kb) {
#pragma unroll 1
    for (int kq = 0; kq < 16 / PB; ++kq, ++step) {
      const int k0 = kb * 16 + kq * PB;
      if (k0 >= n) break;
      const int par = step & 1;
      // the block's columns (all rows; padded rows hold zeros)
      if (tx >= kq * PB && tx < kq * PB + PB) {
        const int j = tx - kq * PB;
#pragma unroll
        for (int i = 0; i < B; ++i) colb[par][j][ty + 16 * i] = a[i][kb];
      }
      __syncthreads();
      // LDL^T of the pivot block P (padded pivots: identity)
      T L[PB][PB], d[PB], rdq[PB];
#pragma unroll
      for (int r = 0; r < PB; ++r) {
#pragma unroll
        for (int c = 0; c < PB; ++c) L[r][c] = (T)0;
      }
#pragma unroll
      for (int r = 0; r < PB; ++r) {
        const bool pad = k0 + r >= n;
        T dr = pad ? (T)1 : colb[par][r][k0 + r];
#pragma unroll
        for (int q = 0; q < r; ++q) dr -= L[r][q] * L[r][q] * d[q];
        if (tid == 0 && !pad) pivs[k0 + r] = dr;
        if (!(dr > tol)) dr = (T)1;   // recorded as singular after the loop
        d[r] = dr;
        const T rd = recip_fast(dr);
        rdq[r] = rd;
#pragma unroll
        for (int i = r + 1; i < PB; ++i) {
          T v = (k0 + i >= n) ? (T)0 : colb[par][r][k0 + i];
#pragma unroll
          for (int q = 0; q < r; ++q) v -= L[i][q] * L[r][q] * d[q];
          L[i][r] = v * rd;
        }
      }
      // P^{-1} = L^{-T} D^{-1} L^{-1}: M = L^{-1} (unit lower), Pi = M^T D^{-1} M
      T M[PB][PB];
#pragma unroll
      for (int i = 0; i < PB; ++i) {
#pragma unroll
        for (int j = 0; j < PB; ++j) {
          T v = (i == j) ? (T)1 : (T)0;
          if (j < i) {
#pragma unroll
            for (int q = j; q < i; ++q) v -= L[i][q] * (q == j ? (T)1 : M[q][j]);
          }
          M[i][j] = (j <= i) ? v : (T)0;
        }
      }
      T Pi[PB][PB];
#pragma unroll
      for (int i = 0; i < PB; ++i)
#pragma unroll
        for (int j = 0; j < PB; ++j) {
          T v = (T)0;
#pragma unroll
          for (int q = 0; q < PB; ++q) v += M[q][i] * M[q][j] * rdq[q];
          Pi[i][j] = v;
        }
      // Z = A_IK P^{-1} for the owned rows, A_KJ for the owned columns
      T Z[B][PB], Y[B][PB];
#pragma unroll
      for (int i = 0; i < B; ++i) {
        T aik[PB];
#pragma unroll
        for (int r = 0; r < PB; ++r) aik[r] = colb[par][r][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < PB; ++j) {
          T v = (T)0;
#pragma unroll
          for (int r = 0; r < PB; ++r) v = fma_t(aik[r], Pi[r][j], v);
          Z[i][j] = v;
        }
      }
#pragma unroll
      for (int c = 0; c < B; ++c)
#pragma unroll
        for (int r = 0; r < PB; ++r) Y[c][r] = colb[par][r][tx + 16 * c];   // A_Kc (Q symmetric)
#pragma unroll
      for (int i = 0; i < B; ++i)
#pragma unroll
        for (int c = 0; c < B; ++c) {
          T v = a[i][c];
#pragma unroll
          for (int r = 0; r < PB; ++r) v = fma_t(-Z[i][r], Y[c][r], v);
          a[i][c] = v;
        }
      // the block's rows and columns (selects keep every register index static)
      const bool krow = ty >= kq * PB && ty < kq * PB + PB;
      const bool kcol = tx >= kq * PB && tx < kq * PB + PB;
      const int rr = ty - kq * PB, cc = tx - kq * PB;
      T pir[PB], pic = (T)0;
#pragma unroll
      for (int r = 0; r < PB; ++r) pir[r] = (T)0;
#pragma unroll
      for (int q = 0; q < PB; ++q)
#pragma unroll
        for (int r = 0; r < PB; ++r) {
          if (rr == q) pir[r] = Pi[q][r];
          if (rr == q && cc == r) pic = Pi[q][r];
        }
      if (krow) {
#pragma unroll
        for (int c = 0; c < B; ++c) {
          T v = (T)0;
#pragma unroll
          for (int r = 0; r < PB; ++r) v = fma_t(pir[r], Y[c][r], v);
          a[kb][c] = v;
        }
      }
      if (kcol) {
#pragma unroll
        for (int i = 0; i < B; ++i) {
          T z = (T)0;
#pragma unroll
          for (int r = 0; r < PB; ++r)
            if (cc == r) z = Z[i][r];
          a[i][kb] = z;
        }
        if (krow) a[kb][kb] = -pic;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      if (r < n && c < n) W[(int64_t)r * n + c] = -a[i][j];
    }
  __syncthreads();
  if (tid < 32) {
    int bad = 0;
    T ratio = (T)1;
    for (int k = tid; k < n; k += 32) {
      const T p = pivs[k];
      if (!(p > tol)) { bad = 1; ratio = (T)0; }
      else if (qd[k] > (T)0) {
        const T r = p / qd[k];
        ratio = r < ratio ? r : ratio;
      }
    }
    bad = __any_sync(0xffffffffu, bad);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T o = __shfl_xor_sync(0xffffffffu, ratio, off);
      ratio = o < ratio ? o : ratio;
    }
    if (tid == 0) {
      if (bad && status && flag_singular) atomicOr(status, DEV_ERR_SINGULAR);
      if (pivot_ratio) *pivot_ratio = (double)ratio;
    }
  }
}

// the sweep used by the library: pairs of pivots per barrier up to order 128
// (every thread factors the pivot block itself, so larger blocks trade the
// barriers saved for redundant arithmetic), one by one above
template <typename T, int B, typename SRC>
__device__ __forceinline__ void sweep_any(const SRC* __restrict__ Q, int n, T* __restrict__ W, int* status,
                                          double* pivot_ratio, bool cg, bool flag_singular) {
  if constexpr (B <= 8) sweep_body_blocked<T, B, 2, SRC>(Q, n, W, status, pivot_ratio, cg, flag_singular);
  else sweep_body<T, B, SRC>(Q, n, W, status, pivot_ratio, cg, flag_singular);
}

template <typename T, int B>
__global__ void __launch_bounds__(256) sweep_inverse_kernel(const double* __restrict__ Q, int n,
                                                            T* __restrict__ W, int* status,
                                                            double* pivot_ratio) {
  PDL_ENTRY();
  sweep_any<T, B, double>(Q, n, W, status, pivot_ratio, false, !apply_df_supported_d(n));
}

// work list of FP32 sweep inverses, one CTA per job (orders up to 128: the
// refined solve that follows has the FP64 fallback, so no singular flag there;
// orders 129..160 flag singular pivots as the single-stream sweep does)
__global__ void __launch_bounds__(256) sweep_batch_kernel(const SweepJob* __restrict__ jobs) {
  PDL_ENTRY();
  const SweepJob j = jobs[blockIdx.x];
  if (j.n <= 16) sweep_any<float, 1, double>(j.Q, j.n, j.W, j.status, j.pivot_ratio, false, false);
  else if (j.n <= 32) sweep_any<float, 2, double>(j.Q, j.n, j.W, j.status, j.pivot_ratio, false, false);
  else if (j.n <= 64) sweep_any<float, 4, double>(j.Q, j.n, j.W, j.status, j.pivot_ratio, false, false);
  else if (j.n <= 112) sweep_any<float, 7, double>(j.Q, j.n, j.W, j.status, j.pivot_ratio, false, false);
  else if (j.n <= 128) sweep_any<float, 8, double>(j.Q, j.n, j.W, j.status, j.pivot_ratio, false, false);
  else sweep_any<float, 10, double>(j.Q, j.n, j.W, j.status, j.pivot_ratio, false, true);
}

cudaError_t launch_sweep_batch(const SweepJob* jobs, int njobs, cudaStream_t s) {
  if (njobs <= 0) return cudaSuccess;
  launch_k(sweep_batch_kernel, (unsigned)njobs, 256, 0, s, jobs);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// small FP64 GEMM: 8x8 output tile per CTA, A rows and B columns of the tile
// staged in shared memory (K <= 256); optional ring-permute epilogue.
// SB > 0 (fused factor): the permuted result Q is also written as an FP32 copy
// Qf, and the last CTA to finish (device-scope counter, wrapping to zero)
// runs the FP32 sweep inverse W = Q^{-1} on it -- one kernel boundary less on
// the critical path of a mode update.  The other CTAs exit without waiting.
// ---------------------------------------------------------------------------
struct FuseFactor {
  float* Qf = nullptr;    // Q as an FP32 pair Qf + Qlo (Qlo may be null)
  float* Qlo = nullptr;
  float* W = nullptr;
  unsigned* counter = nullptr;
  int* status = nullptr;
  double* pivot_ratio = nullptr;
};

// the 8 x 8 output tile (by, bx) of C = A B, or of the ring epilogue
__device__ __forceinline__ void gemm64_body(const double* __restrict__ A, const double* __restrict__ B,
                                            double* __restrict__ C, int M, int K, int N, int pRa, int pRb,
                                            const double* __restrict__ base, float* Qf, float* Qlo, int bx,
                                            int by) {
  extern __shared__ double gsm[];
  double* sA = gsm;            // 8 x K
  double* sB = gsm + 8 * K;    // K x 8
  __shared__ double red[4][64];
  const int r0 = by * 8, c0 = bx * 8;
  for (int e = threadIdx.x; e < 8 * K; e += 256) {
    const int r = e / K, k = e % K;
    sA[e] = (r0 + r < M) ? A[(int64_t)(r0 + r) * K + k] : 0.0;
    const int kk = e / 8, c = e % 8;
    sB[e] = (c0 + c < N) ? B[(int64_t)kk * N + c0 + c] : 0.0;
  }
  __syncthreads();
  // 64 outputs x 4 slices of K; slices summed in a fixed order
  const int o = threadIdx.x & 63, q = threadIdx.x >> 6;
  const double* a = sA + (o >> 3) * K;
  const double* b = sB + (o & 7);
  double s0 = 0.0;
  for (int k = q; k < K; k += 4) s0 = fma(a[k], b[k * 8], s0);
  red[q][o] = s0;
  __syncthreads();
  const int col = c0 + (o & 7);
  const int row = r0 + (o >> 3);
  if (q == 0 && row < M && col < N) {
    const double s = (red[0][o] + red[1][o]) + (red[2][o] + red[3][o]);
    if (pRa <= 0) {
      C[(int64_t)row * N + col] = s;
    } else {
      // row = b + Rb b', col = a + Ra a'  ->  Q[a + Ra b][a' + Ra b']
      const int bb = row % pRb, bp = row / pRb, aa = col % pRa, ap = col / pRa;
      const int RR = pRa * pRb;
      const int64_t qi = (int64_t)(aa + pRa * bb) * RR + (ap + pRa * bp);
      const double v = (base ? base[qi] : 0.0) + s;
      C[qi] = v;
      if (Qf) {
        const float hi = (float)v;
        Qf[qi] = hi;
        if (Qlo) Qlo[qi] = (float)(v - (double)hi);
      }
    }
  }
}

template <int SB>
__global__ void __launch_bounds__(256) gemm64_kernel(const double* __restrict__ A,
                                                     const double* __restrict__ B,
                                                     double* __restrict__ C, int M, int K, int N,
                                                     int pRa, int pRb, const double* __restrict__ base,
                                                     FuseFactor ff) {
  PDL_ENTRY();
  __shared__ int s_last;
  gemm64_body(A, B, C, M, K, N, pRa, pRb, base, ff.Qf, ff.Qlo, blockIdx.x, blockIdx.y);
  if constexpr (SB > 0) {
    __threadfence();
    __syncthreads();
    // atomicInc wraps to 0 after the last CTA: the counter is ready for the next launch
    const unsigned total = gridDim.x * gridDim.y;
    if (threadIdx.x == 0) s_last = atomicInc(ff.counter, total - 1) == total - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    sweep_any<float, SB, float>(ff.Qf, pRa * pRb, ff.W, ff.status, ff.pivot_ratio, true,
                                !apply_df_supported_d(pRa * pRb));
  }
}

cudaError_t launch_gemm64(const double* A, const double* B, double* C, int M, int K, int N,
                          int perm_Ra, int perm_Rb, const double* base, cudaStream_t s, float* Qhi, float* Qlo) {
  dim3 grid((unsigned)ceil_div_i(N, 8), (unsigned)ceil_div_i(M, 8));
  const size_t sm = (size_t)16 * K * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gemm64_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  FuseFactor ff;
  if (perm_Ra > 0) { ff.Qf = Qhi; ff.Qlo = Qlo; }
  launch_k(gemm64_kernel<0>, grid, 256, sm, s, A, B, C, M, K, N, perm_Ra, perm_Rb, base, ff);
  return cudaGetLastError();
}

// work list of small GEMMs / ring products: item = (job, column tile, row tile)
__global__ void __launch_bounds__(256) gemm64_batch_kernel(const GemmJob* __restrict__ jobs,
                                                           const int4* __restrict__ items) {
  PDL_ENTRY();
  const int4 it = items[blockIdx.x];
  const GemmJob j = jobs[it.x];
  gemm64_body(j.A, j.B, j.C, j.M, j.K, j.N, j.pRa, j.pRb, j.base, j.Qf, j.Qlo, it.y, it.z);
}

cudaError_t launch_gemm64_batch(const GemmJob* jobs, const int4* items, int nitems, int Kmax, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  const size_t sm = (size_t)16 * Kmax * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(gemm64_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  launch_k(gemm64_batch_kernel, (unsigned)nitems, 256, sm, s, jobs, items);
  return cudaGetLastError();
}

cudaError_t launch_gemm64_factor(const double* A, const double* B, double* Qout, int M, int K, int N, int Ra,
                                 int Rb, const double* base, float* Qf, float* Qlo, float* W32, unsigned* counter,
                                 int* status, double* pivot_ratio, cudaStream_t s) {
  const int n = Ra * Rb;
  void (*k)(const double*, const double*, double*, int, int, int, int, int, const double*, FuseFactor) = nullptr;
  if (n <= 16) k = gemm64_kernel<1>;
  else if (n <= 32) k = gemm64_kernel<2>;
  else if (n <= 64) k = gemm64_kernel<4>;
  else if (n <= 112) k = gemm64_kernel<7>;
  else if (n <= 160) k = gemm64_kernel<10>;
  else return cudaErrorInvalidValue;
  dim3 grid((unsigned)ceil_div_i(N, 8), (unsigned)ceil_div_i(M, 8));
  const size_t sm = (size_t)16 * K * sizeof(double);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  FuseFactor ff;
  ff.Qf = Qf;
  ff.Qlo = Qlo;
  ff.W = W32;
  ff.counter = counter;
  ff.status = status;
  ff.pivot_ratio = pivot_ratio;
  launch_k(k, grid, 256, sm, s, A, B, Qout, M, K, N, Ra, Rb, base, ff);
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_sweep(const double* Q, int n, T* W, int* status, double* pivot_ratio, cudaStream_t s) {
  void (*k)(const double*, int, T*, int*, double*) = nullptr;
  if (n <= 16) k = sweep_inverse_kernel<T, 1>;
  else if (n <= 32) k = sweep_inverse_kernel<T, 2>;
  else if (n <= 64) k = sweep_inverse_kernel<T, 4>;
  else if (n <= 112) k = sweep_inverse_kernel<T, 7>;
  else if (n <= 160) k = sweep_inverse_kernel<T, 10>;
  else return cudaErrorInvalidValue;
  launch_k(k, 1, 256, 0, s, Q, n, W, status, pivot_ratio);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 LDL^T, register-blocked like the sweep: thread (ty, tx) keeps entries
// (ty + 16a, tx + 16b).  Per pivot k the owners of column k publish it (double
// buffered) and the owner of (k, k) publishes 1/d_k: one barrier per pivot and
// one FP64 division per pivot.  Only the lower triangle is updated (n^3/6 FMA).
// Output: unit lower L (row-major) and invdiag = 1/d.
// ---------------------------------------------------------------------------
template <int B>
__global__ void __launch_bounds__(256) ldlt64_kernel(const double* __restrict__ Q, int n,
                                                     double* __restrict__ L, double* __restrict__ invdiag,
                                                     int* status, double* pivot_ratio) {
  PDL_ENTRY();
  __shared__ double col[2][16 * B];
  __shared__ double rb[2];
  __shared__ double sinv[16 * B];
  __shared__ double qd[16 * B];
  __shared__ double s_tol, s_ratio;
  __shared__ int s_bad;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  double a[B][B];
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      a[i][j] = (r < n && c < n && c <= r) ? Q[(int64_t)r * n + c] : 0.0;
    }
  for (int k = tid; k < n; k += 256) qd[k] = Q[(int64_t)k * n + k];
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int k = 0; k < n; ++k) mx = fmax(mx, qd[k]);
    s_tol = (double)n * 2.220446049250313e-16 * mx;
    s_bad = 0;
    s_ratio = 1.0;
  }
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    const int par = k & 1, kb = k >> 4, kr = k & 15;
    if (tx == kr) {
#pragma unroll
      for (int i = 0; i < B; ++i) {
        const int r = ty + 16 * i;
#pragma unroll
        for (int j = 0; j < B; ++j)
          if (j == kb && r < n && r >= k) {
            col[par][r] = a[i][j];
            if (r == k) {   // pivot owner
              double d = a[i][j];
              if (!(d > s_tol)) { s_bad = 1; d = 1.0; }
              else if (qd[k] > 0) s_ratio = fmin(s_ratio, d / qd[k]);
              const double rc = 1.0 / d;
              rb[par] = rc;
              sinv[k] = rc;
            }
          }
      }
    }
    __syncthreads();
    const double rc = rb[par];
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int r = ty + 16 * i;
      if (r <= k || r >= n) continue;
      const double li = col[par][r] * rc;
#pragma unroll
      for (int j = 0; j < B; ++j) {
        const int c = tx + 16 * j;
        if (c > k && c <= r) a[i][j] = fma(-li, col[par][c], a[i][j]);
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < B; ++i)
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      if (r < n && c < n) L[(int64_t)r * n + c] = (c < r) ? a[i][j] * sinv[c] : (c == r ? 1.0 : 0.0);
    }
  for (int k = tid; k < n; k += 256) invdiag[k] = sinv[k];
  if (tid == 0) {
    if (s_bad && status) atomicOr(status, DEV_ERR_SINGULAR);
    if (pivot_ratio) *pivot_ratio = s_ratio;
  }
}

cudaError_t launch_chol_factor(const double* Q, int n, double* L, double* invdiag, int* status,
                               double* pivot_ratio, cudaStream_t s) {
  if (n <= 16) launch_k(ldlt64_kernel<1>, 1, 256, 0, s, Q, n, L, invdiag, status, pivot_ratio);
  else if (n <= 32) launch_k(ldlt64_kernel<2>, 1, 256, 0, s, Q, n, L, invdiag, status, pivot_ratio);
  else if (n <= 64) launch_k(ldlt64_kernel<4>, 1, 256, 0, s, Q, n, L, invdiag, status, pivot_ratio);
  else if (n <= 112) launch_k(ldlt64_kernel<7>, 1, 256, 0, s, Q, n, L, invdiag, status, pivot_ratio);
  else if (n <= 160) launch_k(ldlt64_kernel<10>, 1, 256, 0, s, Q, n, L, invdiag, status, pivot_ratio);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// row solves x = p Q^{-1} = p L^{-T} D^{-1} L^{-1} with L (unit) in shared
// memory (padded rows); one warp per right-hand side row, 4 warps per CTA.
// leverage mode: lev[r] = ||D^{-1/2} L^{-1} p||^2 / n.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) chol_solve_kernel(const double* __restrict__ Lg,
                                                         const double* __restrict__ invdiag, int n,
                                                         const double* __restrict__ P, int64_t rows,
                                                         double* out64, float* out32, double* lev) {
  PDL_ENTRY();
  extern __shared__ double sm[];
  const int ld = n + 1;
  double* L = sm;                       // n x ld
  double* inv = L + n * ld;             // n
  double* ys = inv + n;                 // 4 warps x n
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < n * n; e += blockDim.x) cp_async8(&L[(e / n) * ld + (e % n)], &Lg[e]);
  for (int e = tid; e < n; e += blockDim.x) cp_async8(&inv[e], &invdiag[e]);
  cp_async_wait_all();
  __syncthreads();
  double* y = ys + warp * n;
  for (int64_t r = (int64_t)blockIdx.x * 4 + warp; r < rows; r += (int64_t)gridDim.x * 4) {
    for (int j = lane; j < n; j += 32) y[j] = P[r * n + j];
    __syncwarp();
    for (int k = 0; k < n - 1; ++k) {
      const double yk = y[k];
      for (int j = k + 1 + lane; j < n; j += 32) y[j] = fma(-L[j * ld + k], yk, y[j]);
      __syncwarp();
    }
    if (lev) {
      double sum = 0.0;
      for (int j = lane; j < n; j += 32) sum = fma(y[j] * inv[j], y[j], sum);
      for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) lev[r] = sum / n;
      __syncwarp();
      continue;
    }
    for (int j = lane; j < n; j += 32) y[j] *= inv[j];
    __syncwarp();
    for (int k = n - 1; k > 0; --k) {
      const double xk = y[k];
      for (int j = lane; j < k; j += 32) y[j] = fma(-L[k * ld + j], xk, y[j]);
      __syncwarp();
    }
    for (int j = lane; j < n; j += 32) {
      if (out64) out64[r * n + j] = y[j];
      if (out32) out32[r * n + j] = (float)y[j];
    }
    __syncwarp();
  }
}

cudaError_t launch_chol_solve(const double* L, const double* invdiag, int n, const double* P,
                              int64_t rows, double* out64, float* out32, double* lev,
                              cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  const size_t sm = ((size_t)n * (n + 1) + n + 4 * (size_t)n) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(chol_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((rows + 3) / 4, 152 * 2));
  launch_k(chol_solve_kernel, (unsigned)blocks, 128, sm, s, L, invdiag, n, P, rows, out64, out32, lev);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Mixed precision (FP32 slab arithmetic): W32 = Q^{-1} by the FP32 sweep, then
// per row g = p W32 followed by `iters` refinement steps
// r = p - g Q (FP64, Q symmetric), g += r W32.
// ---------------------------------------------------------------------------
// rows bx, bx + nbx, ...
__device__ __forceinline__ void solve_refine_body(const float* __restrict__ Wg, const double* __restrict__ Qg,
                                                  int n, const double* __restrict__ P, int64_t rows, int iters,
                                                  int q_in_smem, double* out64, float* out32, const PartialSum& ps,
                                                  int64_t bx, int64_t nbx) {
  // one row of P per CTA at a time, one thread per column of the solution
  extern __shared__ unsigned char smr[];
  float* Wm = (float*)smr;                                                    // n x n
  double* Qs = (double*)(((uintptr_t)(Wm + n * n) + 15) & ~(uintptr_t)15);    // n x n (optional)
  double* gs = Qs + (q_in_smem ? n * n : 0);                                  // n: current solution
  float* vf = (float*)(gs + n);                                               // n: right-hand side (FP32)
  const int tid = threadIdx.x;
  // stage W32 and Q (16-byte copies when the sizes allow); completion is awaited
  // only before the first use, so it overlaps the first right-hand side's loads
  if ((n & 3) == 0 && (((uintptr_t)Wg | (uintptr_t)Qg) & 15) == 0) {
    for (int e = 4 * tid; e < n * n; e += 4 * blockDim.x) cp_async16(&Wm[e], &Wg[e]);
    if (q_in_smem)
      for (int e = 2 * tid; e < n * n; e += 2 * blockDim.x) cp_async16(&Qs[e], &Qg[e]);
  } else {
    for (int e = tid; e < n * n; e += blockDim.x) cp_async4(&Wm[e], &Wg[e]);
    if (q_in_smem)
      for (int e = tid; e < n * n; e += blockDim.x) cp_async8(&Qs[e], &Qg[e]);
  }
  cp_async_commit();
  const double* Q = q_in_smem ? Qs : Qg;
  const int c = tid;
  for (int64_t r = bx; r < rows; r += nbx) {
    double pc = 0.0;
    if (c < n) {
      if (ps.part) {
        // P = base + sum of the split partials, in split order; stored, then solved.
        // Loads are issued eight at a time ahead of the (ordered) additions.
        pc = ps.base ? ps.base[r * n + c] : 0.0;
        double acc = 0.0;
        const float* pp = ps.part + r * n + c;
        const int64_t st = rows * n;
        for (int k0 = 0; k0 < ps.splits; k0 += 8) {
          float v[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) v[u] = (k0 + u < ps.splits) ? pp[(int64_t)(k0 + u) * st] : 0.f;
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (k0 + u < ps.splits) acc += (double)v[u];
        }
        pc += acc;
        ps.pout[r * n + c] = pc;
      } else {
        pc = P[r * n + c];
      }
    }
    cp_async_wait_all();
    if (c < n) vf[c] = (float)pc;
    double g = 0.0;
    __syncthreads();
    for (int it = 0; it <= iters; ++it) {
      // g += v W32   (v = p on the first pass, then the FP64 residual)
      if (c < n) {
        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
        int k = 0;
        for (; k + 3 < n; k += 4) {
          a0 = fmaf(vf[k], Wm[k * n + c], a0);
          a1 = fmaf(vf[k + 1], Wm[(k + 1) * n + c], a1);
          a2 = fmaf(vf[k + 2], Wm[(k + 2) * n + c], a2);
          a3 = fmaf(vf[k + 3], Wm[(k + 3) * n + c], a3);
        }
        for (; k < n; ++k) a0 = fmaf(vf[k], Wm[k * n + c], a0);
        g += (double)((a0 + a1) + (a2 + a3));
        gs[c] = g;
      }
      __syncthreads();
      if (it == iters) break;
      // v = p - g Q in FP64 (Q symmetric)
      if (c < n) {
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int k = 0;
        for (; k + 3 < n; k += 4) {
          a0 = fma(-gs[k], Q[(int64_t)k * n + c], a0);
          a1 = fma(-gs[k + 1], Q[(int64_t)(k + 1) * n + c], a1);
          a2 = fma(-gs[k + 2], Q[(int64_t)(k + 2) * n + c], a2);
          a3 = fma(-gs[k + 3], Q[(int64_t)(k + 3) * n + c], a3);
        }
        for (; k < n; ++k) a0 = fma(-gs[k], Q[(int64_t)k * n + c], a0);
        vf[c] = (float)(pc + ((a0 + a1) + (a2 + a3)));
      }
      __syncthreads();
    }
    if (c < n) {
      if (out64) out64[r * n + c] = g;
      if (out32) out32[r * n + c] = (float)g;
    }
  }
}

__global__ void __launch_bounds__(160) solve_refine_kernel(const float* __restrict__ Wg,
                                                           const double* __restrict__ Qg, int n,
                                                           const double* __restrict__ P, int64_t rows,
                                                           int iters, int q_in_smem, double* out64,
                                                           float* out32, PartialSum ps) {
  PDL_ENTRY();
  solve_refine_body(Wg, Qg, n, P, rows, iters, q_in_smem, out64, out32, ps, blockIdx.x, gridDim.x);
}

// work list of refined solves of orders 129..160 (FP64 residual): item = (job, block, blocks of the job)
__global__ void __launch_bounds__(160) solve_refine_batch_kernel(const RefineJob* __restrict__ jobs,
                                                                 const int4* __restrict__ items) {
  PDL_ENTRY();
  const int4 it = items[blockIdx.x];
  const RefineJob j = jobs[it.x];
  solve_refine_body(j.W, j.Q, j.n, j.P, j.rows, j.iters, j.q_in_smem, j.out64, j.out32, j.ps, it.y, it.z);
}

// ---------------------------------------------------------------------------
// Refined solve for n <= 128, one row of P per CTA at a time, 256
// threads: thread (c, part) owns column c (and c + 64) and the quarter part of
// every inner sum.  W32 and Q = Qh + Ql (an FP32 pair carrying Q to about 2^-48) are
// staged by bulk copies (plain loads for odd n); the right-hand side is formed from the split
// partials as in solve_refine_kernel.
//   g  = p W32                           (FP32)
//   r  = p - g Q                         (double-FP32 arithmetic: exact products
//                                         and error-free sums, Dekker / Knuth)
//   g += r W32                           (FP32), result rounded to FP64 / FP32
// The FP64 pipe is not used in the inner loops.
// ---------------------------------------------------------------------------

// FP64 fallback of the refined solve, for a Q whose FP32 inverse cannot seed a
// converging refinement (cond(Q) u_32 not small; see apply_df_kernel): the CTA
// inverts Q in FP64 by the symmetric sweep in shared memory (two barriers per
// pivot), then each of its rows takes g = p Q^{-1} and one FP64 refinement
// step g += (p - g Q) Q^{-1}.  The right-hand side is formed from the split
// partials in split order (and stored) as in the FP32 path.
constexpr double kFallbackPivotRatio = 1.0 / 8192.0;   // smallest FP32 pivot / diagonal kept
constexpr float kFallbackCorrection = 1e-3f;           // largest first correction kept, |dg| / |g|
constexpr int kRowMaskBits = 256;                      // rows of a CTA tracked one by one

// Rows bx, bx + nbx, ...; with `mask`, only the rows whose local index (0 for
// bx, 1 for bx + nbx, ...) has its bit set.
__device__ __noinline__ void apply_fp64_rows(const ApplyDF& a, double* sm, int64_t bx, int64_t nbx,
                                             const unsigned* mask) {
  const int n = a.n, tid = threadIdx.x, nt = blockDim.x;
  double* W = sm;           // n x n: Q, then -Q^{-1}
  double* cb = W + n * n;   // pivot column
  double* pv = cb + n;      // right-hand side
  double* gv = pv + n;      // solution
  double* rv = gv + n;      // residual
  __shared__ double s_tol;
  __shared__ int s_bad;
  for (int e = tid; e < n * n; e += nt) W[e] = a.Q64[e];
  __syncthreads();
  if (tid == 0) {
    double mx = 0.0;
    for (int k = 0; k < n; ++k) mx = fmax(mx, W[k * n + k]);
    s_tol = (double)n * 2.220446049250313e-16 * mx;
    s_bad = 0;
  }
  __syncthreads();
  const double tol = s_tol;
  for (int k = 0; k < n; ++k) {
    for (int i = tid; i < n; i += nt) cb[i] = W[i * n + k];
    __syncthreads();
    double piv = cb[k];
    if (!(piv > tol)) {
      piv = 1.0;
      if (tid == 0) s_bad = 1;
    }
    const double rcp = 1.0 / piv;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e - i * n;
      double v;
      if (i == k) v = (j == k) ? -rcp : cb[j] * rcp;
      else if (j == k) v = cb[i] * rcp;
      else v = fma(-cb[i] * rcp, cb[j], W[e]);
      W[e] = v;
    }
    __syncthreads();
  }
  if (tid == 0 && s_bad && a.status) atomicOr(a.status, DEV_ERR_SINGULAR);
  int64_t lr = 0;
  for (int64_t r = bx; r < a.rows; r += nbx, ++lr) {
    if (mask && lr < kRowMaskBits && !((mask[lr >> 5] >> (lr & 31)) & 1u)) continue;
    for (int c = tid; c < n; c += nt) {
      double pc;
      if (a.ps.part) {
        pc = a.ps.base ? a.ps.base[r * n + c] : 0.0;
        double acc = 0.0;
        const float* pp = a.ps.part + r * n + c;
        const int64_t st = a.rows * n;
        for (int k = 0; k < a.ps.splits; ++k) acc += (double)pp[(int64_t)k * st];
        pc += acc;
        a.ps.pout[r * n + c] = pc;
      } else {
        pc = a.P[r * n + c];
      }
      pv[c] = pc;
    }
    __syncthreads();
    for (int c = tid; c < n; c += nt) {          // g = p Q^{-1}  (W = -Q^{-1})
      double g = 0.0;
      for (int k = 0; k < n; ++k) g = fma(-pv[k], W[k * n + c], g);
      gv[c] = g;
    }
    __syncthreads();
    for (int c = tid; c < n; c += nt) {          // residual p - g Q  (Q symmetric)
      double t = pv[c];
      for (int k = 0; k < n; ++k) t = fma(-gv[k], a.Q64[(int64_t)k * n + c], t);
      rv[c] = t;
    }
    __syncthreads();
    for (int c = tid; c < n; c += nt) {
      double g = gv[c];
      for (int k = 0; k < n; ++k) g = fma(-rv[k], W[k * n + c], g);
      if (a.out64) a.out64[r * n + c] = g;
      if (a.out32) a.out32[r * n + c] = (float)g;
    }
    __syncthreads();
  }
  if (tid == 0 && a.fallbacks) atomicAdd(a.fallbacks, 1u);
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// rows bx, bx + nbx, ... of one refined solve (bx: the block's index, nbx: the
// blocks sharing the solve)
template <int CPT>
__device__ __forceinline__ void apply_df_body(const ApplyDF& a, int64_t bx, int64_t nbx) {
  // CPT columns per thread: c = (tid & 63) + 64 u, u < CPT (n <= 64 CPT)
  extern __shared__ __align__(16) unsigned char sma[];
  const int n = a.n, nn = n * n, nns = (nn + 3) & ~3;
  float* Wm = (float*)sma;                  // n x n
  float* Qh = Wm + nns;                     // n x n
  float* Ql = Qh + nns;                     // n x n
  double* pd = (double*)(Ql + nns);         // n: right-hand side (FP64)
  double* pd4 = pd + n;                     // 4 x n: per-part sums of the split partials
  float* vf = (float*)(pd4 + 4 * n);        // n: FP32 vector of the current product
  float* red = vf + n;                      // 4 x n partial sums (x2 for pairs)
  __shared__ __align__(8) uint64_t bar;
  __shared__ float s_dn[2], s_gn[2];
  __shared__ int s_redo;
  __shared__ unsigned s_rows[kRowMaskBits / 32];   // rows to redo in FP64, by local index
  const int tid = threadIdx.x, c0 = tid & 63, part = tid >> 6;
  if (tid == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_redo = 0;
  }
  if (tid < kRowMaskBits / 32) s_rows[tid] = 0u;
  __syncthreads();
  // even n: bulk copies (sizes in 16-byte units); odd n: plain loads
  const bool bulk = (n & 1) == 0;
  if (bulk && tid == 0) {
    mbar_expect_tx(&bar, 3u * nn * 4u);
    bulk_g2s(Wm, a.W, nn * 4, &bar);
    bulk_g2s(Qh, a.Qh, nn * 4, &bar);
    bulk_g2s(Ql, a.Ql, nn * 4, &bar);
  }
  // a tiny FP32 pivot (or none recorded as usable): the FP32 inverse cannot seed
  // the refinement, go straight to the FP64 fallback (read while the copies run;
  // the fallback reuses the staging area once they have landed)
  if (a.Q64 && a.pivot_ratio && !(*a.pivot_ratio >= kFallbackPivotRatio)) {
    const bool ok = !bulk || mbar_wait(&bar, 0, 2000000000ull);
    if (__syncthreads_or(!ok)) {
      if (tid == 0 && a.status) atomicOr(a.status, DEV_ERR_TIMEOUT);
      return;
    }
    apply_fp64_rows(a, (double*)sma, bx, nbx, nullptr);
    return;
  }
  bool staged = !bulk;
  if (!bulk) {
    for (int e = tid; e < nn; e += 256) {
      Wm[e] = a.W[e];
      Qh[e] = a.Qh[e];
      Ql[e] = a.Ql[e];
    }
    __syncthreads();
  }
  const int k0 = part * ((n + 3) / 4), k1 = min(n, k0 + (n + 3) / 4);
  // sum_{k in this part} v[k] W[k][c]
  auto part_dot = [&](int c) {
    float s0 = 0.f, s1 = 0.f;
    int k = k0;
    for (; k + 1 < k1; k += 2) {
      s0 = fmaf(vf[k], Wm[k * n + c], s0);
      s1 = fmaf(vf[k + 1], Wm[(k + 1) * n + c], s1);
    }
    if (k < k1) s0 = fmaf(vf[k], Wm[k * n + c], s0);
    return s0 + s1;
  };
  int64_t lr = 0;
  for (int64_t r = bx; r < a.rows; r += nbx, ++lr) {
    // right-hand side: base + split partials (or P).  Part q sums the splits
    // q, q + 4, ... in order; the four sums are added in part order.
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = c0 + 64 * u;
      if (c >= n) continue;
      if (a.ps.part) {
        double acc = 0.0;
        const float* pp = a.ps.part + r * n + c;
        const int64_t st = a.rows * n;
        for (int s0 = part; s0 < a.ps.splits; s0 += 32) {
          float v[8];
#pragma unroll
          for (int w = 0; w < 8; ++w) v[w] = (s0 + 4 * w < a.ps.splits) ? pp[(int64_t)(s0 + 4 * w) * st] : 0.f;
#pragma unroll
          for (int w = 0; w < 8; ++w)
            if (s0 + 4 * w < a.ps.splits) acc += (double)v[w];
        }
        pd4[part * n + c] = acc;
      } else if (part == 0) {
        pd4[c] = a.P[r * n + c];
      }
    }
    __syncthreads();
    if (part == 0) {
#pragma unroll
      for (int u = 0; u < CPT; ++u) {
        const int c = c0 + 64 * u;
        if (c >= n) continue;
        double pc;
        if (a.ps.part) {
          pc = a.ps.base ? a.ps.base[r * n + c] : 0.0;
          pc += ((pd4[c] + pd4[n + c]) + pd4[2 * n + c]) + pd4[3 * n + c];
          a.ps.pout[r * n + c] = pc;
        } else {
          pc = pd4[c];
        }
        pd[c] = pc;
        vf[c] = (float)pc;
      }
    }
    if (!staged) {
      const bool ok = mbar_wait(&bar, 0, 2000000000ull);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(a.status, DEV_ERR_TIMEOUT);
        return;
      }
      staged = true;
    } else {
      __syncthreads();
    }
    // g = p W32
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = c0 + 64 * u;
      if (c < n) red[part * n + c] = part_dot(c);
    }
    __syncthreads();
    float g[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = c0 + 64 * u;
      g[u] = 0.f;
      if (part == 0 && c < n) {
        g[u] = (red[c] + red[n + c]) + (red[2 * n + c] + red[3 * n + c]);
        vf[c] = g[u];            // g, read by every part below
      }
    }
    __syncthreads();
    // s = g Q in pair arithmetic over this part's k
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = c0 + 64 * u;
      if (c >= n) continue;
      float sh = 0.f, sl = 0.f;
      for (int k = k0; k < k1; ++k) {
        const float gk = vf[k], qh = Qh[k * n + c], ql = Ql[k * n + c];
        const float ph = gk * qh;
        float pl = fmaf(gk, qh, -ph);     // exact: gk qh = ph + pl
        pl = fmaf(gk, ql, pl);
        float t, e;
        two_sum(sh, ph, t, e);
        sh = t;
        sl += e + pl;
      }
      red[part * n + c] = sh;
      red[4 * n + part * n + c] = sl;
    }
    __syncthreads();
    float rfl[CPT];
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = c0 + 64 * u;
      rfl[u] = 0.f;
      if (part == 0 && c < n) {
        double sm = 0.0;
#pragma unroll
        for (int q = 0; q < 4; ++q) sm += (double)red[q * n + c] + (double)red[4 * n + q * n + c];
        rfl[u] = (float)(pd[c] - sm);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = c0 + 64 * u;
      if (part == 0 && c < n) vf[c] = rfl[u];
    }
    __syncthreads();
    // g += r W32
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      const int c = c0 + 64 * u;
      if (c < n) red[part * n + c] = part_dot(c);
    }
    __syncthreads();
    if (part == 0) {
      // the first correction's size estimates the FP32 inverse's error on this
      // row (the refined error is about its square): too large = fallback
      float dn = 0.f, gn = 0.f;
#pragma unroll
      for (int u = 0; u < CPT; ++u) {
        const int c = c0 + 64 * u;
        if (c >= n) continue;
        const float d = (red[c] + red[n + c]) + (red[2 * n + c] + red[3 * n + c]);
        const double gv = (double)g[u] + (double)d;
        if (a.out64) a.out64[r * n + c] = gv;
        if (a.out32) a.out32[r * n + c] = (float)gv;
        dn = fmaf(d, d, dn);
        gn = fmaf(g[u], g[u], gn);
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        dn += __shfl_xor_sync(0xffffffffu, dn, off);
        gn += __shfl_xor_sync(0xffffffffu, gn, off);
      }
      if ((tid & 31) == 0) { s_dn[tid >> 5] = dn; s_gn[tid >> 5] = gn; }
    }
    __syncthreads();
    if (tid == 0) {
      const float dn = s_dn[0] + s_dn[1], gn = s_gn[0] + s_gn[1];
      if (!(dn <= kFallbackCorrection * kFallbackCorrection * gn)) {
        s_redo = 1;
        if (lr < kRowMaskBits) s_rows[lr >> 5] |= 1u << (lr & 31);
        else s_redo = 2;   // beyond the tracked rows: redo every row of the block
      }
    }
  }
  if (!staged) {   // no row: the bulk copies still complete before exit
    mbar_wait(&bar, 0, 2000000000ull);
  }
  if (a.Q64 && __syncthreads_or(s_redo)) apply_fp64_rows(a, (double*)sma, bx, nbx, s_redo == 2 ? nullptr : s_rows);
}

template <int CPT>
__global__ void __launch_bounds__(256) apply_df_kernel(ApplyDF a) {
  PDL_ENTRY();
  apply_df_body<CPT>(a, blockIdx.x, gridDim.x);
}

// work list of refined solves: item = (job, block, blocks of the job)
template <int CPT>
__global__ void __launch_bounds__(256) apply_df_batch_kernel(const ApplyDF* __restrict__ jobs,
                                                             const int4* __restrict__ items) {
  PDL_ENTRY();
  __shared__ ApplyDF sj;
  const int4 it = items[blockIdx.x];
  {
    const int* src = (const int*)&jobs[it.x];
    int* dst = (int*)&sj;
    for (int e = threadIdx.x; e < (int)(sizeof(ApplyDF) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
  }
  __syncthreads();
  apply_df_body<CPT>(sj, it.y, it.z);
}

size_t apply_df_smem(int n) {
  return (size_t)3 * ((n * n + 3) & ~3) * 4 + (size_t)5 * n * 8 + (size_t)n * 4 + (size_t)8 * n * 4;
}

// Q (FP64) -> FP32 pair (hi, lo)
__global__ void split_pair_kernel(const double* __restrict__ Q, int64_t count, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  PDL_ENTRY();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
    const double v = Q[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

cudaError_t launch_split_pair(const double* Q, int64_t count, float* hi, float* lo, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152));
  launch_k(split_pair_kernel, blocks, 256, 0, s, Q, count, hi, lo);
  return cudaGetLastError();
}

bool apply_df_supported(int n) { return apply_df_supported_d(n); }

cudaError_t launch_apply_df_batch(const ApplyDF* jobs, const int4* items, int nitems, int nmax, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (!apply_df_supported(nmax)) return cudaErrorInvalidValue;
  const size_t sm = apply_df_smem(nmax);
  auto kern = nmax <= 64 ? apply_df_batch_kernel<1> : apply_df_batch_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  launch_k(kern, (unsigned)nitems, 256, sm, s, jobs, items);
  return cudaGetLastError();
}

cudaError_t launch_apply_df(const float* W32, const float* Qh, const float* Ql, int n, const double* P, int64_t rows,
                            double* out64, float* out32, const PartialSum* ps, int* status, cudaStream_t s,
                            const double* Q64, const double* pivot_ratio, unsigned* fallbacks) {
  if (rows <= 0) return cudaSuccess;
  if (!apply_df_supported(n)) return cudaErrorInvalidValue;
  const size_t sm = apply_df_smem(n);
  auto kern = n <= 64 ? apply_df_kernel<1> : apply_df_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  ApplyDF a;
  a.W = W32; a.Qh = Qh; a.Ql = Ql; a.n = n; a.rows = rows; a.P = P;
  if (ps) a.ps = *ps;
  a.out64 = out64; a.out32 = out32; a.status = status;
  a.Q64 = Q64; a.pivot_ratio = pivot_ratio; a.fallbacks = fallbacks;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(rows, 152 * 4));
  launch_k(kern, (unsigned)blocks, 256, sm, s, a);
  return cudaGetLastError();
}

// leverage scores from the solved rows: p_i = (g_i . x_i) / n with x_i = g_i M^{-1}
// (FP64 dot per row, one warp per row)
__global__ void leverage_dot_kernel(const double* __restrict__ G, const double* __restrict__ Xs, int64_t rows,
                                    int n, double* __restrict__ p) {
  PDL_ENTRY();
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double sum = 0.0;
    for (int c = lane; c < n; c += 32) sum = fma(G[r * n + c], Xs[r * n + c], sum);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) p[r] = sum / n;
  }
}

cudaError_t launch_leverage_dot(const double* G, const double* X, int64_t rows, int n, double* p, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows * 32 + 255) / 256, 152 * 8));
  launch_k(leverage_dot_kernel, blocks, 256, 0, s, G, X, rows, n, p);
  return cudaGetLastError();
}

cudaError_t launch_factor_mixed(const double* Q, int n, float* W32, int* status, double* pivot_ratio,
                                cudaStream_t s) {
  return launch_sweep<float>(Q, n, W32, status, pivot_ratio, s);
}

int refine_q_in_smem(int n) {
  const size_t base = (size_t)n * n * sizeof(float) + 16 + (size_t)n * (sizeof(double) + sizeof(float));
  return base + (size_t)n * n * sizeof(double) <= 200 * 1024 ? 1 : 0;
}

size_t refine_smem(int n, int q_in_smem) {
  const size_t base = (size_t)n * n * sizeof(float) + 16 + (size_t)n * (sizeof(double) + sizeof(float));
  return base + (q_in_smem ? (size_t)n * n * sizeof(double) : 0);
}

cudaError_t launch_refine_batch(const RefineJob* jobs, const int4* items, int nitems, int nmax, size_t smem,
                                cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(solve_refine_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  launch_k(solve_refine_batch_kernel, (unsigned)nitems, ((nmax + 31) / 32) * 32, smem, s, jobs, items);
  return cudaGetLastError();
}

cudaError_t launch_apply_mixed(const float* W32, const double* Q, int n, const double* P, int64_t rows,
                               int iters, double* out64, float* out32, const PartialSum* ps, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  if (n < 1 || n > 160) return cudaErrorInvalidValue;
  const size_t base = (size_t)n * n * sizeof(float) + 16 + (size_t)n * (sizeof(double) + sizeof(float));
  const int q_in_smem = base + (size_t)n * n * sizeof(double) <= 200 * 1024 ? 1 : 0;
  const size_t sms = base + (q_in_smem ? (size_t)n * n * sizeof(double) : 0);
  cudaError_t e = cudaFuncSetAttribute(solve_refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sms);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(rows, 152 * 4));
  const int threads = ((n + 31) / 32) * 32;
  PartialSum none;
  launch_k(solve_refine_kernel, (unsigned)blocks, threads, sms, s, W32, Q, n, P, rows, iters, q_in_smem, out64, out32,
                                                            ps ? *ps : none);
  return cudaGetLastError();
}

cudaError_t launch_solve_mixed(const double* Q, int n, const double* P, int64_t rows, int iters,
                               float* W32, float* /*unused*/, double* out64, float* out32, int* status,
                               double* pivot_ratio, cudaStream_t s) {
  cudaError_t e = launch_factor_mixed(Q, n, W32, status, pivot_ratio, s);
  if (e != cudaSuccess) return e;
  return launch_apply_mixed(W32, Q, n, P, rows, iters, out64, out32, nullptr, s);
}

__global__ void fill_kernel(double* p, int64_t count, double v) {
  PDL_ENTRY();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

cudaError_t launch_fill(double* p, int64_t count, double v, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 1024));
  launch_k(fill_kernel, (unsigned)blocks, 256, 0, s, p, count, v);
  return cudaGetLastError();
}
