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

// one thread per (j, r): row r of the chain product, kept in registers
struct ChainArgs {
  const void* core[STR_MAXN];
  int64_t dim[STR_MAXN];
  int R[STR_MAXN + 1];
};

template <typename T>
__global__ void chain_table_kernel(ChainArgs ca, int k0, int k1, int transpose, int64_t J,
                                   T* __restrict__ table) {
  PDL_ENTRY();
  const int Rf = ca.R[k0], Rl = ca.R[k1 + 1];
  const int64_t total = J * Rf;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / Rf;
    const int r = (int)(e % Rf);
    T v[STR_MAXR], w[STR_MAXR];
    int64_t rem = j;
    // first factor: row r of G_{k0}(i_{k0})
    int cols = ca.R[k0 + 1];
    {
      const int64_t i = rem % ca.dim[k0];
      rem /= ca.dim[k0];
      const T* g = (const T*)ca.core[k0] + i * (int64_t)Rf * cols;
#pragma unroll
      for (int c = 0; c < STR_MAXR; ++c) v[c] = (c < cols) ? g[r + Rf * c] : (T)0;
    }
    for (int k = k0 + 1; k <= k1; ++k) {
      const int64_t i = rem % ca.dim[k];
      rem /= ca.dim[k];
      const int Rk = ca.R[k], Rk1 = ca.R[k + 1];
      const T* g = (const T*)ca.core[k] + i * (int64_t)Rk * Rk1;
#pragma unroll
      for (int c = 0; c < STR_MAXR; ++c) {
        T s = 0;
        if (c < Rk1) {
#pragma unroll
          for (int x = 0; x < STR_MAXR; ++x)
            if (x < Rk) s += v[x] * g[x + Rk * c];
        }
        w[c] = s;
      }
#pragma unroll
      for (int c = 0; c < STR_MAXR; ++c) v[c] = w[c];
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
  if (k1 == k0 + 1 && !transpose && R[k0] * R[k0 + 1] <= STR_MAXRR && R[k0 + 1] * R[k1 + 1] <= STR_MAXRR) {
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
  if (compute == 2) launch_k(chain_table_kernel<double>, blocks, 128, 0, s, ca, k0, k1, transpose, J, (double*)table);
  else launch_k(chain_table_kernel<float>, blocks, 128, 0, s, ca, k0, k1, transpose, J, (float*)table);
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
