// FP64 kernels for the structured Gram and the small normal equations.
//
//   core Gram        M = G_{(2)}^T G_{(2)},   transfer form E = sum_i G(i) (x) G(i)
//                    (the Gram tensor Z of Alg. 2 line 2, with its indices permuted)
//   ring             W = E_{n+1} E_{n+2} ... E_{n-1}  gives  (H^{!=n})_<2>   (Prop. subchain_gram)
//   solve            G_{n(2)} = P_n Q_n^{-1} by Cholesky (Alg. 4 line 17)
//   leverage         l_i = ||L^{-1} g_i||^2 with M = L L^T (Lemma lev_est)
#include <algorithm>

#include "kernels.cuh"

// ---------------------------------------------------------------------------
// core Gram: one thread per (c, c') pair with c <= c'; writes both halves
// ---------------------------------------------------------------------------
__global__ void core_gram_kernel(const double* __restrict__ G, int64_t I, int Ra, int Rb,
                                 double* __restrict__ M, double* __restrict__ E) {
  const int RR = Ra * Rb;
  const int64_t npairs = (int64_t)RR * (RR + 1) / 2;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < npairs;
       t += (int64_t)gridDim.x * blockDim.x) {
    // decode t -> (c, c') with c <= c'  (row-wise over the upper triangle)
    int c = 0;
    int64_t rem = t;
    while (rem >= RR - c) { rem -= RR - c; ++c; }
    const int cp = c + (int)rem;
    double s = 0.0;
    for (int64_t i = 0; i < I; ++i) s = fma(G[i * RR + c], G[i * RR + cp], s);
    if (M) { M[(int64_t)c * RR + cp] = s; M[(int64_t)cp * RR + c] = s; }
    if (E) {
      // c = a + Ra b, c' = a' + Ra b'  ->  E[(a + Ra a'), (b + Rb b')]
      const int a = c % Ra, b = c / Ra, ap = cp % Ra, bp = cp / Ra;
      const int64_t RR2 = (int64_t)Rb * Rb;
      E[(int64_t)(a + Ra * ap) * RR2 + (b + Rb * bp)] = s;
      E[(int64_t)(ap + Ra * a) * RR2 + (bp + Rb * b)] = s;
    }
  }
}

cudaError_t launch_core_gram(const double* G, int64_t I, int Ra, int Rb, double* M, double* E,
                             cudaStream_t s) {
  const int RR = Ra * Rb;
  const int64_t npairs = (int64_t)RR * (RR + 1) / 2;
  const int threads = 128;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((npairs + threads - 1) / threads, 2048));
  core_gram_kernel<<<(unsigned)blocks, threads, 0, s>>>(G, I, Ra, Rb, M, E);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// small FP64 GEMM, one output per thread; optional ring-permute epilogue
// ---------------------------------------------------------------------------
__global__ void gemm64_kernel(const double* __restrict__ A, const double* __restrict__ B,
                              double* __restrict__ C, int M, int K, int N, int pRa, int pRb,
                              const double* __restrict__ base) {
  const int col = blockIdx.x * 8 + (threadIdx.x & 7);
  const int row = blockIdx.y * 8 + (threadIdx.x >> 3);
  if (row >= M || col >= N) return;
  double s = 0.0;
  for (int k = 0; k < K; ++k) s = fma(A[(int64_t)row * K + k], B[(int64_t)k * N + col], s);
  if (pRa <= 0) {
    C[(int64_t)row * N + col] = s;
  } else {
    // row = b + Rb b', col = a + Ra a'  ->  Q[a + Ra b][a' + Ra b']
    const int b = row % pRb, bp = row / pRb, a = col % pRa, ap = col / pRa;
    const int RR = pRa * pRb;
    const int64_t q = (int64_t)(a + pRa * b) * RR + (ap + pRa * bp);
    C[q] = (base ? base[q] : 0.0) + s;
  }
}

cudaError_t launch_gemm64(const double* A, const double* B, double* C, int M, int K, int N,
                          int perm_Ra, int perm_Rb, const double* base, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div_i(N, 8), (unsigned)ceil_div_i(M, 8));
  gemm64_kernel<<<grid, 64, 0, s>>>(A, B, C, M, K, N, perm_Ra, perm_Rb, base);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cholesky factorisation in shared memory (right-looking, one CTA)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) chol_factor_kernel(const double* __restrict__ Q, int n,
                                                          double* __restrict__ L,
                                                          double* __restrict__ invdiag,
                                                          int* status, double* pivot_ratio) {
  extern __shared__ double A[];   // n x n, row-major, lower triangle used
  __shared__ double s_tol, s_ratio;
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  for (int e = tid; e < n * n; e += blockDim.x) A[e] = Q[e];
  if (tid == 0) {
    double mx = 0.0;
    for (int k = 0; k < n; ++k) mx = fmax(mx, Q[(int64_t)k * n + k]);
    s_tol = (double)n * 2.220446049250313e-16 * mx;
    s_ratio = 1.0;
    s_bad = 0;
  }
  __syncthreads();
  const int tx = tid & 31, ty = tid >> 5, nty = blockDim.x >> 5;
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double d = A[k * n + k];
      const double q = Q[(int64_t)k * n + k];
      if (!(d > s_tol)) { s_bad = 1; d = 1.0; }
      else if (q > 0) s_ratio = fmin(s_ratio, d / q);
      const double r = sqrt(d);
      A[k * n + k] = r;
      invdiag[k] = 1.0 / r;
    }
    __syncthreads();
    const double inv = 1.0 / A[k * n + k];
    for (int i = k + 1 + tid; i < n; i += blockDim.x) A[i * n + k] *= inv;
    __syncthreads();
    for (int i = k + 1 + ty; i < n; i += nty) {
      const double lik = A[i * n + k];
      for (int j = k + 1 + tx; j <= i; j += 32) A[i * n + j] = fma(-lik, A[j * n + k], A[i * n + j]);
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    L[e] = (j <= i) ? A[e] : 0.0;
  }
  if (tid == 0) {
    if (s_bad && status) atomicOr(status, DEV_ERR_SINGULAR);
    if (pivot_ratio) *pivot_ratio = s_ratio;
  }
}

cudaError_t launch_chol_factor(const double* Q, int n, double* L, double* invdiag, int* status,
                               double* pivot_ratio, cudaStream_t s) {
  const size_t sm = (size_t)n * n * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(chol_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  chol_factor_kernel<<<1, 256, sm, s>>>(Q, n, L, invdiag, status, pivot_ratio);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// row solves with L in shared memory; one warp per right-hand side row
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) chol_solve_kernel(const double* __restrict__ Lg,
                                                         const double* __restrict__ invdiag, int n,
                                                         const double* __restrict__ P, int64_t rows,
                                                         double* out64, float* out32, double* lev) {
  extern __shared__ double sm[];
  double* L = sm;                       // n x n
  double* inv = L + n * n;              // n
  double* ys = inv + n;                 // 8 warps x n
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < n * n; e += blockDim.x) L[e] = Lg[e];
  for (int e = tid; e < n; e += blockDim.x) inv[e] = invdiag[e];
  __syncthreads();
  double* y = ys + warp * n;
  for (int64_t r = (int64_t)blockIdx.x * 8 + warp; r < rows; r += (int64_t)gridDim.x * 8) {
    for (int j = lane; j < n; j += 32) y[j] = P[r * n + j];
    __syncwarp();
    // forward: L y = p
    for (int k = 0; k < n; ++k) {
      const double yk = y[k] * inv[k];
      __syncwarp();
      if (lane == 0) y[k] = yk;
      for (int j = k + 1 + lane; j < n; j += 32) y[j] = fma(-L[j * n + k], yk, y[j]);
      __syncwarp();
    }
    if (lev) {
      double s = 0.0;
      for (int j = lane; j < n; j += 32) s = fma(y[j], y[j], s);
      for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) lev[r] = s / n;
      __syncwarp();
      continue;
    }
    // backward: L^T x = y
    for (int k = n - 1; k >= 0; --k) {
      const double xk = y[k] * inv[k];
      __syncwarp();
      if (lane == 0) y[k] = xk;
      for (int j = lane; j < k; j += 32) y[j] = fma(-L[k * n + j], xk, y[j]);
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
  const size_t sm = ((size_t)n * n + n + 8 * (size_t)n) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(chol_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, 152 * 2));
  chol_solve_kernel<<<(unsigned)blocks, 256, sm, s>>>(L, invdiag, n, P, rows, out64, out32, lev);
  return cudaGetLastError();
}

__global__ void fill_kernel(double* p, int64_t count, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

cudaError_t launch_fill(double* p, int64_t count, double v, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 1024));
  fill_kernel<<<(unsigned)blocks, 256, 0, s>>>(p, count, v);
  return cudaGetLastError();
}
