// Reconstruction, relative fit error and masked loss of the TR format
// (Sec. 1: X(i) = Trace(G_1(i_1) ... G_N(i_N))).
//
// The modes are split into a prefix 1..k and a suffix k+1..N.  With the
// prefix products L(row) = G_1 ... G_k and suffix products S(col) =
// G_{k+1} ... G_N, X(row, col) = Trace(L S) = sum_c Lm[row][c] Rm[col][c], a
// GEMM with K = R_1 R_{k+1} over row = linear index of (i_1..i_k) and col =
// linear index of (i_{k+1}..i_N) -- exactly the tensor's own memory order.
#include <algorithm>

#include "kernels.cuh"

static __device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
static __device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }

// one thread per (j, r): row r of the chain product, kept in registers
struct ChainArgs {
  const void* core[STR_MAXN];
  int64_t dim[STR_MAXN];
  int R[STR_MAXN + 1];
};

// RM: a bound on every rank of the chain (the register rows and the unrolled
// loops are RM long; the sums run over the true ranks in the same order for any
// RM, so the result does not depend on it)
template <typename T, int RM>
__global__ void chain_table_kernel(ChainArgs ca, int k0, int k1, int transpose, int64_t J,
                                   T* __restrict__ table) {
  PDL_ENTRY();
  const int Rf = ca.R[k0], Rl = ca.R[k1 + 1];
  const int64_t total = J * Rf;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / Rf;
    const int r = (int)(e % Rf);
    T v[RM], w[RM];
    int64_t rem = j;
    // first factor: row r of G_{k0}(i_{k0})
    int cols = ca.R[k0 + 1];
    {
      const int64_t i = rem % ca.dim[k0];
      rem /= ca.dim[k0];
      const T* g = (const T*)ca.core[k0] + i * (int64_t)Rf * cols;
#pragma unroll
      for (int c = 0; c < RM; ++c) v[c] = (c < cols) ? g[r + Rf * c] : (T)0;
    }
    for (int k = k0 + 1; k <= k1; ++k) {
      const int64_t i = rem % ca.dim[k];
      rem /= ca.dim[k];
      const int Rk = ca.R[k], Rk1 = ca.R[k + 1];
      const T* g = (const T*)ca.core[k] + i * (int64_t)Rk * Rk1;
#pragma unroll
      for (int c = 0; c < RM; ++c) {
        T s = 0;
        if (c < Rk1) {
#pragma unroll
          for (int x = 0; x < RM; ++x)
            if (x < Rk) s += v[x] * g[x + Rk * c];
        }
        w[c] = s;
      }
#pragma unroll
      for (int c = 0; c < RM; ++c) v[c] = w[c];
      cols = Rk1;
    }
    T* out = table + j * (int64_t)Rf * Rl;
    for (int c = 0; c < Rl; ++c) {
      if (!transpose) out[r + Rf * c] = v[c];      // P(r, c) at r + Rf c
      else out[c + Rl * r] = v[c];                 // P(r, c) at c + Rl r
    }
  }
}

// Two-core chain table: T[i_a + I_a i_b] = G_a(i_a) G_b(i_b), (r, c) at r + Rf c.
// CTA per (tile of 16 i_a, i_b): both operands staged in shared memory, each
// thread forms four entries.
template <typename T>
__global__ void __launch_bounds__(256) chain2_kernel(const T* __restrict__ Ga, const T* __restrict__ Gb, int Ia,
                                                    int Rf, int Rm, int Rl, T* __restrict__ table) {
  PDL_ENTRY();
  __shared__ T sa[16 * STR_MAXRR];
  __shared__ T sb[STR_MAXRR];
  const int ib = blockIdx.y, ia0 = blockIdx.x * 16;
  const int na = min(16, Ia - ia0);
  const int sza = Rf * Rm, szb = Rm * Rl, szo = Rf * Rl;
  for (int e = threadIdx.x; e < na * sza; e += 256) sa[e] = Ga[(int64_t)ia0 * sza + e];
  for (int e = threadIdx.x; e < szb; e += 256) sb[e] = Gb[(int64_t)ib * szb + e];
  __syncthreads();
  for (int e = threadIdx.x; e < na * szo; e += 256) {
    const int t = e / szo, o = e - t * szo;
    const int r = o % Rf, c = o / Rf;
    const T* ga = sa + t * sza;
    T v = 0;
    for (int x = 0; x < Rm; ++x) v += ga[r + Rf * x] * sb[x + Rm * c];
    table[((int64_t)ib * Ia + ia0 + t) * szo + o] = v;
  }
}

cudaError_t launch_chain_table(const void* const* cores, int compute, const int* R, int N,
                               const int64_t* dims, int k0, int k1, int64_t /*row_off_last*/,
                               int transpose, void* table, cudaStream_t s) {
  int64_t J = 1;
  for (int k = k0; k <= k1; ++k) J *= dims[k];
  const int64_t total = J * R[k0];
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 127) / 128, 152 * 16));
  if (k1 == k0 + 1 && !transpose && R[k0] * R[k0 + 1] <= STR_MAXRR && R[k0 + 1] * R[k1 + 1] <= STR_MAXRR &&
      dims[k1] <= 65535) {
    dim3 grid((unsigned)((dims[k0] + 15) / 16), (unsigned)dims[k1]);
    if (compute == 2)
      launch_k(chain2_kernel<double>, grid, 256, 0, s, (const double*)cores[k0], (const double*)cores[k1],
               (int)dims[k0], R[k0], R[k0 + 1], R[k1 + 1], (double*)table);
    else
      launch_k(chain2_kernel<float>, grid, 256, 0, s, (const float*)cores[k0], (const float*)cores[k1],
               (int)dims[k0], R[k0], R[k0 + 1], R[k1 + 1], (float*)table);
    return cudaGetLastError();
  }
  ChainArgs ca;
  for (int k = 0; k < STR_MAXN; ++k) { ca.core[k] = k < N ? cores[k] : nullptr; ca.dim[k] = k < N ? dims[k] : 1; }
  for (int k = 0; k <= STR_MAXN; ++k) ca.R[k] = k <= N ? R[k] : 1;
  int rmax = 1;
  for (int k = k0; k <= k1 + 1; ++k) rmax = std::max(rmax, R[k]);
  if (rmax <= 8) {
    if (compute == 2) launch_k(chain_table_kernel<double, 8>, blocks, 128, 0, s, ca, k0, k1, transpose, J, (double*)table);
    else launch_k(chain_table_kernel<float, 8>, blocks, 128, 0, s, ca, k0, k1, transpose, J, (float*)table);
  } else {
    if (compute == 2)
      launch_k(chain_table_kernel<double, STR_MAXR>, blocks, 128, 0, s, ca, k0, k1, transpose, J, (double*)table);
    else launch_k(chain_table_kernel<float, STR_MAXR>, blocks, 128, 0, s, ca, k0, k1, transpose, J, (float*)table);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 64 x 64 output tile per CTA; K staged in chunks of 32.
// ---------------------------------------------------------------------------
template <typename T, int MODE>
__global__ void __launch_bounds__(256) recon_kernel(const T* __restrict__ Lm, const T* __restrict__ Rm,
                                                    int64_t rows, int64_t cols, int K,
                                                    const void* __restrict__ X, int xtype,
                                                    const uint32_t* __restrict__ mask, void* out,
                                                    int out_type, double* __restrict__ block_sums) {
  PDL_ENTRY();
  constexpr int KC = 32;
  __shared__ T sL[KC][64 + 1], sR[KC][64 + 1];
  __shared__ double red[2][256];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t row0 = (int64_t)blockIdx.x * 64, col0 = (int64_t)blockIdx.y * 64;
  T acc[4][4];
#pragma unroll
  for (int p = 0; p < 4; ++p)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[p][q] = 0;
  for (int k0 = 0; k0 < K; k0 += KC) {
    for (int e = tid; e < KC * 64; e += 256) {
      const int kk = e % KC, rr = e / KC;
      const int k = k0 + kk;
      sL[kk][rr] = (k < K && row0 + rr < rows) ? Lm[(row0 + rr) * K + k] : (T)0;
      sR[kk][rr] = (k < K && col0 + rr < cols) ? Rm[(col0 + rr) * K + k] : (T)0;
    }
    __syncthreads();
    const int kn = min(KC, K - k0);
    for (int kk = 0; kk < kn; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) a[p] = sL[kk][tx + 16 * p];
#pragma unroll
      for (int q = 0; q < 4; ++q) b[q] = sR[kk][ty + 16 * q];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] += a[p] * b[q];
    }
    __syncthreads();
  }
  double d2 = 0.0, n2 = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t col = col0 + ty + 16 * q;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t row = row0 + tx + 16 * p;
      if (row >= rows || col >= cols) continue;
      const int64_t lin = row + rows * col;
      const double xh = (double)acc[p][q];
      if (MODE == RM_WRITE) {
        if (out_type == XT_F64) ((double*)out)[lin] = xh;
        else ((float*)out)[lin] = (float)xh;
        continue;
      }
      double x;
      switch (xtype) {
        case XT_F64: x = ((const double*)X)[lin]; break;
        case XT_F32: x = (double)((const float*)X)[lin]; break;
        default: x = (double)__bfloat162float(((const __nv_bfloat16*)X)[lin]); break;
      }
      const bool keep = !mask || ((mask[lin >> 5] >> (lin & 31)) & 1u);
      const double r = x - xh;
      if (MODE == RM_FIT) { d2 = fma(r, r, d2); n2 = fma(x, x, n2); }
      else if (MODE == RM_LOSS) { if (keep) d2 = fma(r, r, d2); }
      else {
        const double v = keep ? r : 0.0;
        if (out_type == XT_F64) ((double*)out)[lin] = v;
        else ((float*)out)[lin] = (float)v;
      }
    }
  }
  if (MODE == RM_FIT || MODE == RM_LOSS) {
    red[0][tid] = d2;
    red[1][tid] = n2;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
      if (tid < o) { red[0][tid] += red[0][tid + o]; red[1][tid] += red[1][tid + o]; }
      __syncthreads();
    }
    if (tid == 0) {
      const int64_t b = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
      block_sums[2 * b] = red[0][0];
      block_sums[2 * b + 1] = red[1][0];
    }
  }
}

int recon_blocks(int64_t rows, int64_t cols) {
  return ceil_div_i(rows, 64) * ceil_div_i(cols, 64);
}

cudaError_t launch_recon(const void* Lm, const void* Rm, int compute, int64_t rows, int64_t cols,
                         int K, int mode, const void* X, int xtype, const uint32_t* mask, void* out,
                         int out_type, double* block_sums, int64_t* nblocks, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div_i(rows, 64), (unsigned)ceil_div_i(cols, 64));
  if (grid.y > 65535) return cudaErrorInvalidValue;
  if (nblocks) *nblocks = (int64_t)grid.x * grid.y;
#define STR_RECON_CASE(T, M)                                                                 \
  launch_k(recon_kernel<T, M>, grid, 256, 0, s, (const T*)Lm, (const T*)Rm, rows, cols, K, X, xtype, \
                                          mask, out, out_type, block_sums)
  if (compute == 2) {
    switch (mode) {
      case RM_WRITE: STR_RECON_CASE(double, RM_WRITE); break;
      case RM_FIT: STR_RECON_CASE(double, RM_FIT); break;
      case RM_LOSS: STR_RECON_CASE(double, RM_LOSS); break;
      default: STR_RECON_CASE(double, RM_RESID); break;
    }
  } else {
    switch (mode) {
      case RM_WRITE: STR_RECON_CASE(float, RM_WRITE); break;
      case RM_FIT: STR_RECON_CASE(float, RM_FIT); break;
      case RM_LOSS: STR_RECON_CASE(float, RM_LOSS); break;
      default: STR_RECON_CASE(float, RM_RESID); break;
    }
  }
#undef STR_RECON_CASE
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused masked-loss pass.  With the residual r = M .* (X - Lm Rm^T) over
// (row, col) = (prefix index, suffix index), one read of X gives
//   loss partials      sum r^2,
//   Z[row][c] = sum_col r Rm[col][c]   (partial per column group),
//   W[col][c] = sum_row r Lm[row][c]   (partial per row group),
// from which the core gradients follow as small MTTKRPs (the gradient of the
// trace with respect to the prefix product is -Z, to the suffix product -W).
// CTA (column group, row group): Lm^T of its rows and Z^T stay in shared
// memory; the 64 x 64 tiles of X (and their mask words) stream through an
// S-stage cp.async ring; per 64-column block, Rm^T is staged from registers
// loaded one block ahead and W accumulates in registers over the row blocks.
// ---------------------------------------------------------------------------
template <typename T> struct Vec4;
template <> struct Vec4<float> {
  static __device__ __forceinline__ void ld(const float* p, float* v) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  static __device__ __forceinline__ void st(float* p, const float* v) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Vec4<double> {
  static __device__ __forceinline__ void ld(const double* p, double* v) {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  static __device__ __forceinline__ void st(double* p, const double* v) {
    *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
  }
};
__device__ __forceinline__ void cp_async_elem(float* d, const float* g) { cp_async4(d, g); }
__device__ __forceinline__ void cp_async_elem(double* d, const double* g) { cp_async8(d, g); }

constexpr int LP_SB = 68;   // row stride of the 64-wide staged tiles (Rm^T, residual)

template <typename T, bool BWD, int S, int NJ>
__global__ void __launch_bounds__(256, 1) loss_pass_kernel(const T* __restrict__ Lm, const T* __restrict__ Rm,
                                                          int64_t rows, int64_t cols, int K,
                                                          const T* __restrict__ X,
                                                          const uint32_t* __restrict__ mask, int64_t nwords,
                                                          int RG, int64_t cb_per, int vec,
                                                          double* __restrict__ loss_part,
                                                          T* __restrict__ Zpart, T* __restrict__ Wpart) {
  PDL_ENTRY();
  extern __shared__ __align__(16) unsigned char smem_lp[];
  __shared__ double red[8];
  const int RGP = RG + 4;
  T* sA = (T*)smem_lp;                          // [K][RGP]     Lm^T of the row group
  T* sB = sA + (size_t)K * RGP;                 // [64][LP_SB]  Rm^T of the column block, rows k >= K zero
  T* sX = sB + 64 * LP_SB;                      // [S][64 cols][64 rows]
  uint32_t* sM = (uint32_t*)(sX + S * 4096);    // [S][64 cols][4 words]
  T* sZ = (T*)(sM + S * 256);                   // [K][RGP]     Z^T of the row group (BWD)
  T* sR = sZ + (size_t)K * RGP;                 // [64 cols][LP_SB]  residual tile (BWD)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t rg0 = (int64_t)blockIdx.y * RG;
  const int nr = (int)min((int64_t)RG, rows - rg0);
  const int nrb = (nr + 63) / 64;
  const int64_t ncb = (cols + 63) / 64;
  const int64_t cb0 = (int64_t)blockIdx.x * cb_per, cb1 = min(ncb, cb0 + cb_per);
  const int ntiles = (int)(cb1 - cb0) * nrb;
  for (int e = tid; e < nrb * 64 * K; e += 256) {
    const int r = e / K, k = e - r * K;
    sA[k * RGP + r] = r < nr ? Lm[(rg0 + r) * K + k] : (T)0;
  }
  for (int e = K * LP_SB + tid; e < 64 * LP_SB; e += 256) sB[e] = (T)0;
  if (BWD)
    for (int e = tid; e < K * RGP; e += 256) sZ[e] = (T)0;

  // X tile t (and its mask words) into ring slot t % S; one commit group per call
  auto issue = [&](int t) {
    if (t < ntiles) {
      const int64_t col0 = (cb0 + t / nrb) * 64;
      const int rb = (t % nrb) * 64;
      const int ncol = (int)min((int64_t)64, cols - col0), nrow = min(64, nr - rb);
      T* dx = sX + (t % S) * 4096;
      const T* gx = X + (rg0 + rb) + rows * col0;
      if (vec) {
        constexpr int VE = 16 / sizeof(T), CPC = 64 / VE;
        for (int e = tid; e < 64 * CPC; e += 256) {
          const int c = e / CPC, r = (e - c * CPC) * VE;
          if (c < ncol && r < nrow) cp_async16(dx + c * 64 + r, gx + r + rows * c);
        }
      } else {
        for (int e = tid; e < 4096; e += 256) {
          const int c = e >> 6, r = e & 63;
          if (c < ncol && r < nrow) cp_async_elem(dx + c * 64 + r, gx + r + rows * c);
        }
      }
      if (mask && tid < 192) {
        const int c = tid / 3, w = tid - 3 * c;
        const int64_t wi = ((rg0 + rb + rows * (col0 + c)) >> 5) + w;
        if (c < ncol && wi < nwords) cp_async4(sM + (t % S) * 256 + c * 4 + w, mask + wi);
      }
    }
    cp_async_commit();
  };
  // Rm^T of a column block: the thread's share in registers
  T breg[16];
  auto load_b = [&](int64_t cb) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u;
      breg[u] = (T)0;
      if (cb < cb1 && e < 64 * K) {
        const int c = e / K;
        if (cb * 64 + c < cols) breg[u] = Rm[cb * 64 * K + e];
      }
    }
  };
  auto store_b = [&]() {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
      const int e = tid + 256 * u;
      if (e < 64 * K) {
        const int c = e / K, k = e - c * K;
        sB[k * LP_SB + c] = breg[u];
      }
    }
  };
  T wacc[4][NJ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NJ; ++j) wacc[i][j] = (T)0;
  // W of a finished column block through shared memory, written contiguously
  auto flush_w = [&](int64_t cb) {
    const int64_t col0 = cb * 64;
    const int ncol = (int)min((int64_t)64, cols - col0);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int k = ty + 16 * j;
        if (k < K) sR[(tx + 16 * i) * K + k] = wacc[i][j];
        wacc[i][j] = (T)0;
      }
    __syncthreads();
    T* Wout = Wpart + ((int64_t)blockIdx.y * cols + col0) * K;
    for (int e = tid; e < ncol * K; e += 256) Wout[e] = sR[e];
    __syncthreads();
  };

  load_b(cb0);
  store_b();
  load_b(cb0 + 1);
  for (int t = 0; t < S - 1; ++t) issue(t);
  double lsum = 0.0;
  for (int t = 0; t < ntiles; ++t) {
    const int64_t cb = cb0 + t / nrb;
    const int rb = (t % nrb) * 64;
    const int64_t col0 = cb * 64;
    const int ncol = (int)min((int64_t)64, cols - col0);
    if (rb == 0 && t > 0) {
      __syncthreads();              // every thread is done with the previous block's sB / sR
      if (BWD) flush_w(cb - 1);
      store_b();
      load_b(cb + 1);
    }
    cp_async_wait_n<S - 2>();
    __syncthreads();
    issue(t + S - 1);
    const T* xs = sX + (t % S) * 4096;
    const uint32_t* ms = sM + (t % S) * 256;
    T acc[4][4];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[p][q] = (T)0;
    for (int k = 0; k < K; ++k) {
      T av[4], bv[4];
      Vec4<T>::ld(sA + k * RGP + rb + 4 * tx, av);
      Vec4<T>::ld(sB + k * LP_SB + 4 * ty, bv);
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = fma_t(av[p], bv[q], acc[p][q]);
    }
    T ts = (T)0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = 4 * ty + q;
      T xv[4], rv[4];
      Vec4<T>::ld(xs + c * 64 + 4 * tx, xv);
      const int sh = (int)((rg0 + rb + rows * (col0 + c)) & 31);
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int r = 4 * tx + p;
        bool keep = rb + r < nr && c < ncol;
        if (mask && keep) {
          const int pos = sh + r;
          keep = (ms[c * 4 + (pos >> 5)] >> (pos & 31)) & 1u;
        }
        const T v = keep ? xv[p] - acc[p][q] : (T)0;
        rv[p] = v;
        ts = fma_t(v, v, ts);
      }
      if (BWD) Vec4<T>::st(sR + c * LP_SB + 4 * tx, rv);
    }
    lsum += (double)ts;
    if (BWD) {
      __syncthreads();
      // Z rows rb + 4tx .. +3, k = ty + 16j: sum over the block's 64 columns
      T z[4][NJ];
#pragma unroll
      for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int j = 0; j < NJ; ++j) z[p][j] = (T)0;
      for (int c = 0; c < 64; ++c) {
        T rv[4], bv[NJ];
        Vec4<T>::ld(sR + c * LP_SB + 4 * tx, rv);
#pragma unroll
        for (int j = 0; j < NJ; ++j) bv[j] = sB[(ty + 16 * j) * LP_SB + c];
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int j = 0; j < NJ; ++j) z[p][j] = fma_t(rv[p], bv[j], z[p][j]);
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const int k = ty + 16 * j;
        if (k < K) {
          T zz[4];
          T* zp = sZ + k * RGP + rb + 4 * tx;
          Vec4<T>::ld(zp, zz);
#pragma unroll
          for (int p = 0; p < 4; ++p) zz[p] += z[p][j];
          Vec4<T>::st(zp, zz);
        }
      }
      // W columns tx + 16i, k = ty + 16j: sum over the tile's 64 rows, four at a time
      for (int rq = 0; rq < 16; ++rq) {
        T rv[4][4], av[NJ][4];
#pragma unroll
        for (int i = 0; i < 4; ++i) Vec4<T>::ld(sR + (tx + 16 * i) * LP_SB + 4 * rq, rv[i]);
#pragma unroll
        for (int j = 0; j < NJ; ++j) {
          const int k = ty + 16 * j;
          if (k < K) Vec4<T>::ld(sA + k * RGP + rb + 4 * rq, av[j]);
          else av[j][0] = av[j][1] = av[j][2] = av[j][3] = (T)0;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < NJ; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) wacc[i][j] = fma_t(rv[i][e], av[j][e], wacc[i][j]);
      }
    }
  }
  cp_async_wait_n<0>();
  if (BWD) {
    __syncthreads();
    if (ntiles > 0) flush_w(cb1 - 1);
    T* Zo = Zpart + ((int64_t)blockIdx.x * rows + rg0) * K;
    for (int e = tid; e < nr * K; e += 256) {
      const int r = e / K, k = e - r * K;
      Zo[e] = sZ[k * RGP + r];
    }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((tid & 31) == 0) red[tid >> 5] = lsum;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    loss_part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
  }
}

static int lp_stages(int esize, bool bwd) { return esize == 8 ? 2 : (bwd ? 3 : 4); }

size_t loss_pass_smem(int esize, int RG, int K, bool bwd) {
  const int S = lp_stages(esize, bwd);
  const size_t m = bwd ? 2 : 1;
  return (size_t)esize * (m * K * (size_t)(RG + 4) + m * 64 * LP_SB + (size_t)S * 4096) + 4 * (size_t)S * 256;
}

bool loss_pass_plan(int compute, int64_t rows, int64_t cols, int K, bool bwd, LossPlan* pl) {
  if (K < 1 || K > 64 || rows < 1 || cols < 1) return false;
  const int es = compute == 2 ? 8 : 4;
  const size_t cap = 220 * 1024;
  const int64_t rows64 = (rows + 63) / 64 * 64;
  int RGmax = (int)std::min<int64_t>(rows64, 4096);
  while (RGmax > 64 && loss_pass_smem(es, RGmax, K, bwd) > cap) RGmax -= 64;
  if (loss_pass_smem(es, RGmax, K, bwd) > cap) return false;
  const int64_t ncb = (cols + 63) / 64;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // one resident CTA per SM: minimise the tiles of the busiest SM (waves x (tiles
  // per CTA + about two tiles of staging and ring fill per CTA)), plus the
  // partial sums written (row groups x cols + column groups x rows)
  double best = 1e300;
  bool found = false;
  for (int rg = RGmax; rg >= 64; rg -= 64) {
    const int64_t nrg = (rows + rg - 1) / rg;
    const int RG = (int)(((rows + nrg - 1) / nrg + 63) / 64 * 64);
    if (RG != rg) continue;                   // each row-group count once, at its equalised size
    for (int64_t ncg = 1; ncg <= std::min<int64_t>(ncb, 4 * sms); ++ncg) {
      const int64_t cb_per = (ncb + ncg - 1) / ncg;
      const int64_t ncg2 = (ncb + cb_per - 1) / cb_per;
      if (ncg2 != ncg || nrg * ncg2 > 65535) continue;
      const int64_t waves = (nrg * ncg2 + sms - 1) / sms;
      const double tiles = (double)waves * ((RG / 64) * cb_per + 2.0);
      const double part = bwd ? (double)(nrg * cols + ncg2 * rows) * K / (4096.0 * sms) : 0.0;
      const double cost = tiles + part + 0.5 * (double)(RG / 64);
      if (cost < best) {
        best = cost;
        found = true;
        pl->RG = RG;
        pl->nrg = (int)nrg;
        pl->ncg = (int)ncg2;
        pl->cb_per = cb_per;
      }
    }
  }
  if (!found) return false;
  pl->smem = loss_pass_smem(es, pl->RG, K, bwd);
  return true;
}

cudaError_t launch_loss_pass(const void* Lm, const void* Rm, int compute, int64_t rows, int64_t cols, int K,
                             const void* X, const uint32_t* mask, const LossPlan& pl, bool bwd,
                             double* loss_part, void* Zpart, void* Wpart, cudaStream_t s) {
  dim3 grid((unsigned)pl.ncg, (unsigned)pl.nrg);
  const int es = compute == 2 ? 8 : 4;
  const int vec = (rows % (16 / es) == 0 && ((uintptr_t)X & 15) == 0) ? 1 : 0;
  const int64_t nwords = (rows * cols + 31) / 32;
#define STR_LP_CASE(T, B, S, J)                                                                     \
  do {                                                                                              \
    cudaError_t e = cudaFuncSetAttribute(loss_pass_kernel<T, B, S, J>,                              \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem); \
    if (e != cudaSuccess) return e;                                                                 \
    launch_k(loss_pass_kernel<T, B, S, J>, grid, 256, pl.smem, s, (const T*)Lm, (const T*)Rm, rows, cols, K, \
             (const T*)X, mask, nwords, pl.RG, pl.cb_per, vec, loss_part, (T*)Zpart, (T*)Wpart);    \
  } while (0)
  // k slots per thread in the Z and W products: ceil(K / 16)
  const int nj = (K + 15) / 16;
  if (compute == 2) {
    if (!bwd) STR_LP_CASE(double, false, 2, 1);
    else if (nj == 1) STR_LP_CASE(double, true, 2, 1);
    else if (nj == 2) STR_LP_CASE(double, true, 2, 2);
    else if (nj == 3) STR_LP_CASE(double, true, 2, 3);
    else STR_LP_CASE(double, true, 2, 4);
  } else {
    if (!bwd) STR_LP_CASE(float, false, 4, 1);
    else if (nj == 1) STR_LP_CASE(float, true, 3, 1);
    else if (nj == 2) STR_LP_CASE(float, true, 3, 2);
    else if (nj == 3) STR_LP_CASE(float, true, 3, 3);
    else STR_LP_CASE(float, true, 3, 4);
  }
#undef STR_LP_CASE
  return cudaGetLastError();
}

// Zt[c * rows + row] = sum_g Zpart[g][row][c] (fixed order over the column groups)
template <typename T>
__global__ void loss_zsum_kernel(const T* __restrict__ Zpart, int ng, int64_t rows, int K, T* __restrict__ Zt) {
  PDL_ENTRY();
  const int64_t total = rows * K;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int g = 0; g < ng; ++g) acc += (double)Zpart[(int64_t)g * total + e];
    const int64_t row = e / K;
    const int c = (int)(e - row * K);
    Zt[(int64_t)c * rows + row] = (T)acc;
  }
}

// W[e] = sum_g Wpart[g][e] (fixed order over the row groups)
template <typename T>
__global__ void loss_wsum_kernel(const T* __restrict__ Wpart, int ng, int64_t count, T* __restrict__ W) {
  PDL_ENTRY();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int g = 0; g < ng; ++g) acc += (double)Wpart[(int64_t)g * count + e];
    W[e] = (T)acc;
  }
}

// unit cores of the two reduced trace problems (K = R_1 R_{k+1}):
//   U(c) (R_{k+1} x R_1) with Trace(L U(c)) = Lm[c]:  U(c)[c / R_1, c % R_1] = 1
//   V(c) (R_1 x R_{k+1}) with Trace(V(c) S) = Rm[c]: V(c)[c % R_1, c / R_1] = 1
template <typename T>
__global__ void unit_cores_kernel(int R1, int Rk, T* __restrict__ U, T* __restrict__ V) {
  PDL_ENTRY();
  const int K = R1 * Rk;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += gridDim.x * blockDim.x) {
    const int c = e / K, o = e - c * K;
    U[e] = o == (c % R1) * Rk + c / R1 ? (T)1 : (T)0;
    V[e] = o == c ? (T)1 : (T)0;
  }
}

// gradient of the first core when the prefix is that core alone:
// grad[i][c] = -scale Zt[c][i]
template <typename T>
__global__ void prefix1_grad_kernel(const T* __restrict__ Zt, int64_t I, int K, double scale, T* __restrict__ grad) {
  PDL_ENTRY();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < I * K; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / K;
    const int c = (int)(e - i * K);
    grad[e] = (T)(-scale * (double)Zt[(int64_t)c * I + i]);
  }
}

cudaError_t launch_loss_reduce(const void* Zpart, int ncg, int64_t rows, const void* Wpart, int nrg, int64_t cols,
                               int K, int compute, void* Zt, void* W, cudaStream_t s) {
  const int64_t zc = rows * K, wc = cols * K;
  const unsigned bz = (unsigned)std::max<int64_t>(1, std::min<int64_t>((zc + 255) / 256, 152 * 8));
  const unsigned bw = (unsigned)std::max<int64_t>(1, std::min<int64_t>((wc + 255) / 256, 152 * 8));
  if (compute == 2) {
    launch_k(loss_zsum_kernel<double>, bz, 256, 0, s, (const double*)Zpart, ncg, rows, K, (double*)Zt);
    if (nrg > 1) launch_k(loss_wsum_kernel<double>, bw, 256, 0, s, (const double*)Wpart, nrg, wc, (double*)W);
  } else {
    launch_k(loss_zsum_kernel<float>, bz, 256, 0, s, (const float*)Zpart, ncg, rows, K, (float*)Zt);
    if (nrg > 1) launch_k(loss_wsum_kernel<float>, bw, 256, 0, s, (const float*)Wpart, nrg, wc, (float*)W);
  }
  return cudaGetLastError();
}

cudaError_t launch_unit_cores(int R1, int Rk, int compute, void* U, void* V, cudaStream_t s) {
  const int K = R1 * Rk;
  const unsigned b = (unsigned)std::max(1, std::min((K * K + 255) / 256, 64));
  if (compute == 2) launch_k(unit_cores_kernel<double>, b, 256, 0, s, R1, Rk, (double*)U, (double*)V);
  else launch_k(unit_cores_kernel<float>, b, 256, 0, s, R1, Rk, (float*)U, (float*)V);
  return cudaGetLastError();
}

cudaError_t launch_prefix1_grad(const void* Zt, int64_t I, int K, double scale, int compute, void* grad,
                                cudaStream_t s) {
  const unsigned b = (unsigned)std::max<int64_t>(1, std::min<int64_t>((I * K + 255) / 256, 152 * 8));
  if (compute == 2) launch_k(prefix1_grad_kernel<double>, b, 256, 0, s, (const double*)Zt, I, K, scale, (double*)grad);
  else launch_k(prefix1_grad_kernel<float>, b, 256, 0, s, (const float*)Zt, I, K, scale, (float*)grad);
  return cudaGetLastError();
}

// fixed-order sum of per-block pairs: out[0] = sum of column 0, out[1] = column 1
__global__ void sum_blocks_kernel(const double* __restrict__ bs, int64_t nb, int width,
                                  double* __restrict__ out, double scale) {
  PDL_ENTRY();
  __shared__ double red[256];
  for (int c = 0; c < width; ++c) {
    double s = 0.0;
    for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) s += bs[b * width + c];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = scale * red[0];
    __syncthreads();
  }
}

cudaError_t launch_sum_blocks(const double* block_sums, int64_t nblocks, int width, double* out,
                              double scale, cudaStream_t s) {
  launch_k(sum_blocks_kernel, 1, 256, 0, s, block_sums, nblocks, width, out, scale);
  return cudaGetLastError();
}
