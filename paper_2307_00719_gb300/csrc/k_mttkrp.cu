// Slab MTTKRP with the TR subchain generated on the fly (never materialised).
//
//   P_n increment = X^new_[n] (G^{!=n}_new)_[2]            (Eq. partial, Alg. 4)
//   temporal      = X^new_[N] G^{!=N}_[2]                   (Alg. 4)
//   sampled       = X_S[n] diag(w) G^{!=n}_S[2]             (Alg. 3, Alg. 5)
//
// Each CTA owns BM rows of mode n and a contiguous range of fibres (split-K).
// Per chunk of BK fibres it (1) decodes the fibre multi-indices, (2) forms the
// subchain slices S_f = G_{n+1}(i_{n+1}) ... G_{n-1}(i_{n-1}) in shared memory
// as a chain of small matrix products, (3) stages the X tile, (4) accumulates
// the outer products into registers.  Partials go to a per-split buffer that a
// second kernel sums in a fixed order (deterministic, no atomics).
#include <algorithm>

#include "kernels.cuh"

namespace {

template <typename T, bool C> struct ElemT { typedef T type; };
template <typename T> struct ElemT<T, true> { typedef cplx<T> type; };

template <typename E> __device__ __forceinline__ E ezero();
template <> __device__ __forceinline__ float ezero<float>() { return 0.f; }
template <> __device__ __forceinline__ double ezero<double>() { return 0.0; }
template <> __device__ __forceinline__ cplx<float> ezero<cplx<float>>() { return {0.f, 0.f}; }
template <> __device__ __forceinline__ cplx<double> ezero<cplx<double>>() { return {0.0, 0.0}; }

// acc += x * conj(s)   (conj is the identity for real types)
__device__ __forceinline__ void mac(float& acc, float x, float s) { acc = fmaf(x, s, acc); }
__device__ __forceinline__ void mac(double& acc, double x, double s) { acc = fma(x, s, acc); }
template <typename T> __device__ __forceinline__ void mac(cplx<T>& acc, cplx<T> x, cplx<T> s) {
  acc.re += x.re * s.re + x.im * s.im;
  acc.im += x.im * s.re - x.re * s.im;
}
// acc += a * b  (true product, used for the subchain)
__device__ __forceinline__ void mulacc(float& acc, float a, float b) { acc = fmaf(a, b, acc); }
__device__ __forceinline__ void mulacc(double& acc, double a, double b) { acc = fma(a, b, acc); }
template <typename T> __device__ __forceinline__ void mulacc(cplx<T>& acc, cplx<T> a, cplx<T> b) {
  acc.re += a.re * b.re - a.im * b.im;
  acc.im += a.re * b.im + a.im * b.re;
}
template <typename T> __device__ __forceinline__ T scal(T x, T w) { return x * w; }
template <typename T> __device__ __forceinline__ cplx<T> scal(cplx<T> x, T w) { return {x.re * w, x.im * w}; }

template <typename E, typename XS> struct LoadX;
template <typename T> struct LoadX<T, __nv_bfloat16> {
  static __device__ __forceinline__ T ld(const void* X, int64_t o) {
    return (T)__bfloat162float(((const __nv_bfloat16*)X)[o]);
  }
};
template <typename T> struct LoadX<T, float> {
  static __device__ __forceinline__ T ld(const void* X, int64_t o) { return (T)((const float*)X)[o]; }
};
template <typename T> struct LoadX<T, double> {
  static __device__ __forceinline__ T ld(const void* X, int64_t o) { return (T)((const double*)X)[o]; }
};
template <typename T, typename S> struct LoadX<cplx<T>, cplx<S>> {
  static __device__ __forceinline__ cplx<T> ld(const void* X, int64_t o) {
    const S* p = (const S*)X + 2 * o;
    return {(T)p[0], (T)p[1]};
  }
};

struct SmemPlan {
  int BK;
  size_t bytes;
  int Rmid;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~(size_t)15; }

__host__ __device__ inline void smem_offsets(int BK, int BM, int RR, int Rb, int Rmid, int esize,
                                             int tsize, int slice_elems, size_t* o) {
  size_t off = 0;
  o[0] = off; off = align16(off + (size_t)BK * STR_MAXN * 4);   // sIdx
  o[1] = off; off = align16(off + (size_t)BK * 8);              // sBase
  o[2] = off; off = align16(off + (size_t)BK * tsize);          // sW
  o[3] = off; off = align16(off + (size_t)BK * BM * esize);     // sX
  o[4] = off; off = align16(off + (size_t)BK * RR * esize);     // sS
  o[5] = off; off = align16(off + (size_t)BK * Rb * Rmid * esize);  // sT0
  o[6] = off; off = align16(off + (size_t)BK * Rb * Rmid * esize);  // sT1
  o[7] = off; off = align16(off + (size_t)BK * slice_elems * esize); // staged core slices
  o[8] = off;
}

// row block bx and fibre split by of one MTTKRP
template <typename T, bool C, typename XS, int RPT, int CPT>
__device__ __forceinline__ void mttkrp_body(const MttkrpArgs& a, int BK, int64_t bx, int64_t by) {
  typedef typename ElemT<T, C>::type E;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int N = a.N, n = a.n;
  const int Ra = a.R[n], Rb = a.R[n + 1];
  const int RR = Ra * Rb;
  const int64_t In = a.dim[n];
  constexpr int BM = 16 * RPT;

  int order[STR_MAXN];
  int64_t stride[STR_MAXN];
  int64_t st = 1;
  for (int k = 0; k < N; ++k) { stride[k] = st; st *= a.dim[k]; }
  for (int t = 0; t < N - 1; ++t) order[t] = (n + 1 + t) % N;
  int Rmid = 1;
  for (int t = 1; t < N - 2; ++t) Rmid = max(Rmid, a.R[order[t] + 1]);
  int slice_elems = 0;
  for (int t = 0; t < N - 1; ++t) slice_elems += a.R[order[t]] * a.R[order[t] + 1];

  size_t o[9];
  smem_offsets(BK, BM, RR, Rb, Rmid, (int)sizeof(E), (int)sizeof(T), slice_elems, o);
  int32_t* sIdx = (int32_t*)(smem + o[0]);
  int64_t* sBase = (int64_t*)(smem + o[1]);
  T* sW = (T*)(smem + o[2]);
  E* sX = (E*)(smem + o[3]);
  E* sS = (E*)(smem + o[4]);
  E* sT[2] = {(E*)(smem + o[5]), (E*)(smem + o[6])};
  E* sG = (E*)(smem + o[7]);   // slices of the chain cores: [t][jj][R_k R_{k+1}]

  const int64_t f_begin = by * a.fib_per_split;
  const int64_t f_end = min(a.nfib, f_begin + a.fib_per_split);
  const int64_t row0 = bx * BM;
  const int tx = tid & 15, ty = tid >> 4;

  E acc[RPT][CPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q)
#pragma unroll
    for (int p = 0; p < CPT; ++p) acc[q][p] = ezero<E>();

  for (int64_t f0 = f_begin; f0 < f_end; f0 += BK) {
    const int nf = (int)min((int64_t)BK, f_end - f0);
    // (1) decode fibre multi-indices and base offsets
    if (tid < nf) {
      const int64_t f = f0 + tid;
      int64_t off = 0;
      double w = a.wscale;
      if (a.idxs) {
        for (int k = 0; k < N; ++k) {
          if (k == n) continue;
          const int i = a.idxs[(int64_t)k * a.m + f];
          sIdx[tid * STR_MAXN + k] = i;
          off += (int64_t)i * stride[k];
          if (a.leverage) w /= a.p[k][i];
        }
      } else {
        int64_t rem = f;
        for (int k = 0; k < N; ++k) {
          if (k == n) continue;
          const int64_t i = rem % a.dim[k];
          rem /= a.dim[k];
          sIdx[tid * STR_MAXN + k] = (int32_t)i;
          off += i * stride[k];
        }
      }
      sBase[tid] = off;
      sW[tid] = (T)w;
      if (a.ws_out && bx == 0) a.ws_out[f] = w;
    }
    __syncthreads();

    // (2a) stage the chain cores' slices G_k(i_k) of this chunk (each slice is
    //      contiguous in global memory: coalesced copies)
    {
      int soff = 0;
      for (int t = 0; t < N - 1; ++t) {
        const int k = order[t];
        const int sz = a.R[k] * a.R[k + 1];
        const E* Gk = (const E*)a.core[k];
        E* dst = sG + (size_t)BK * soff;
        for (int e = tid; e < nf * sz; e += blockDim.x) {
          const int jj = e / sz, x = e - jj * sz;
          dst[e] = Gk[(int64_t)sIdx[jj * STR_MAXN + k] * sz + x];
        }
        soff += sz;
      }
    }
    __syncthreads();
    // (2b) subchain slices S_f = F_0 F_1 ... F_{N-2},  F_t = G_{order[t]}(i_{order[t]})
    {
      const int k0 = order[0], k1 = order[1];
      const int R0 = a.R[k0], R1 = a.R[k1], R2 = a.R[k1 + 1];
      const int sz0 = R0 * R1, sz1 = R1 * R2;
      const E* g0s = sG;
      const E* g1s = sG + (size_t)BK * sz0;
      const bool last = (N == 3);
      E* dst = last ? sS : sT[0];
      const int cols = R2;
      const int total = nf * Rb * cols;
      for (int e = tid; e < total; e += blockDim.x) {
        const int jj = e / (Rb * cols);
        const int rc = e - jj * Rb * cols;
        const int r = rc / cols, c = rc - r * cols;
        const E* g0 = g0s + jj * sz0;
        const E* g1 = g1s + jj * sz1;
        E v = ezero<E>();
        for (int x = 0; x < R1; ++x) mulacc(v, g0[r + R0 * x], g1[x + R1 * c]);
        if (last) dst[jj * RR + c + Ra * r] = v;      // S(b=r, a=c) -> column a + Ra b
        else dst[jj * Rb * Rmid + r * Rmid + c] = v;
      }
      int cur = 0;
      int cur_cols = R2;
      int soff = sz0 + sz1;
      for (int t = 2; t < N - 1; ++t) {
        __syncthreads();
        const int k = order[t];
        const int Rk = a.R[k], Rk1 = a.R[k + 1];
        const int szk = Rk * Rk1;
        const E* gks = sG + (size_t)BK * soff;
        soff += szk;
        const bool fin = (t == N - 2);
        E* src = sT[cur];
        E* out = fin ? sS : sT[cur ^ 1];
        const int tot = nf * Rb * Rk1;
        for (int e = tid; e < tot; e += blockDim.x) {
          const int jj = e / (Rb * Rk1);
          const int rc = e - jj * Rb * Rk1;
          const int r = rc / Rk1, c = rc - r * Rk1;
          const E* gk = gks + jj * szk;
          const E* srow = src + jj * Rb * Rmid + r * Rmid;
          E v = ezero<E>();
          for (int x = 0; x < cur_cols; ++x) mulacc(v, srow[x], gk[x + Rk * c]);
          if (fin) out[jj * RR + c + Ra * r] = v;
          else out[jj * Rb * Rmid + r * Rmid + c] = v;
        }
        cur ^= 1;
        cur_cols = Rk1;
      }
    }
    // (3) X tile: sX[jj][r] = w_f * X_[n](row0 + r, f)
    for (int e = tid; e < BK * BM; e += blockDim.x) {
      int jj, r;
      if (n == 0) { r = e % BM; jj = e / BM; } else { jj = e % BK; r = e / BK; }
      E v = ezero<E>();
      const int64_t row = row0 + r;
      if (jj < nf && row < In) v = scal(LoadX<E, XS>::ld(a.X, sBase[jj] + row * stride[n]), sW[jj]);
      sX[jj * BM + r] = v;
    }
    __syncthreads();
    if (a.gs_out && bx == 0) {
      E* g = (E*)a.gs_out;
      for (int e = tid; e < nf * RR; e += blockDim.x) g[(f0 + e / RR) * RR + (e % RR)] = sS[e];
    }
    // (4) outer-product accumulation
    for (int jj = 0; jj < nf; ++jj) {
      E xv[RPT], sv[CPT];
#pragma unroll
      for (int q = 0; q < RPT; ++q) xv[q] = sX[jj * BM + ty + 16 * q];
#pragma unroll
      for (int p = 0; p < CPT; ++p) {
        const int c = tx + 16 * p;
        sv[p] = (c < RR) ? sS[jj * RR + c] : ezero<E>();
      }
#pragma unroll
      for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int p = 0; p < CPT; ++p) mac(acc[q][p], xv[q], sv[p]);
    }
    __syncthreads();
  }
  E* out = (E*)a.partial + (size_t)by * In * RR;
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int64_t row = row0 + ty + 16 * q;
#pragma unroll
    for (int p = 0; p < CPT; ++p) {
      const int c = tx + 16 * p;
      if (row < In && c < RR) out[row * RR + c] = acc[q][p];
    }
  }
}

template <typename T, bool C, typename XS, int RPT, int CPT>
__global__ void __launch_bounds__(256) mttkrp_kernel(MttkrpArgs a, int BK) {
  PDL_ENTRY();
  mttkrp_body<T, C, XS, RPT, CPT>(a, BK, blockIdx.x, blockIdx.y);
}

// work list of MTTKRPs of one register-block class: item = (job, row block, split)
template <typename T, bool C, typename XS, int RPT, int CPT>
__global__ void __launch_bounds__(256) mttkrp_batch_kernel(const MttkrpArgs* __restrict__ jobs,
                                                           const int4* __restrict__ items,
                                                           const void* const* __restrict__ xptrs, int BK) {
  PDL_ENTRY();
  __shared__ MttkrpArgs sj;
  const int4 it = items[blockIdx.x];
  {
    const int* src = (const int*)&jobs[it.x];
    int* dst = (int*)&sj;
    for (int e = threadIdx.x; e < (int)(sizeof(MttkrpArgs) / sizeof(int)); e += blockDim.x) dst[e] = src[e];
  }
  __syncthreads();
  if (threadIdx.x == 0 && xptrs) sj.X = xptrs[it.w];   // this step's slab of stream it.w
  __syncthreads();
  mttkrp_body<T, C, XS, RPT, CPT>(sj, BK, it.y, it.z);
}

int plan_rmid(const MttkrpArgs& a) {
  int order[STR_MAXN];
  for (int t = 0; t < a.N - 1; ++t) order[t] = (a.n + 1 + t) % a.N;
  int Rmid = 1;
  for (int t = 1; t < a.N - 2; ++t) Rmid = std::max(Rmid, a.R[order[t] + 1]);
  return Rmid;
}

size_t smem_bytes(const MttkrpArgs& a, int BK, int BM) {
  const int esize = (a.compute == 2 ? 8 : 4) * (a.cplx ? 2 : 1);
  const int tsize = a.compute == 2 ? 8 : 4;
  int slice_elems = 0;
  for (int t = 0; t < a.N - 1; ++t) {
    const int k = (a.n + 1 + t) % a.N;
    slice_elems += a.R[k] * a.R[k + 1];
  }
  size_t o[9];
  smem_offsets(BK, BM, a.R[a.n] * a.R[a.n + 1], a.R[a.n + 1], plan_rmid(a), esize, tsize, slice_elems, o);
  return o[8];
}

template <typename T, bool C, typename XS, int RPT, int CPT>
cudaError_t launch_t(const MttkrpArgs& a, cudaStream_t s) {
  constexpr int BM = 16 * RPT;
  int BK = 32;
  while (BK > 4 && smem_bytes(a, BK, BM) > 96 * 1024) BK /= 2;
  const size_t sm = smem_bytes(a, BK, BM);
  auto kern = mttkrp_kernel<T, C, XS, RPT, CPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)ceil_div_i(a.dim[a.n], BM), (unsigned)a.splits);
  launch_k(kern, grid, 256, sm, s, a, BK);
  return cudaGetLastError();
}

template <typename T, bool C, typename XS>
cudaError_t launch_rc(const MttkrpArgs& a, cudaStream_t s) {
  const int RR = a.R[a.n] * a.R[a.n + 1];
  const bool small_rows = a.dim[a.n] <= 16;
  if (RR <= 16) return small_rows ? launch_t<T, C, XS, 1, 1>(a, s) : launch_t<T, C, XS, 4, 1>(a, s);
  if (RR <= 64) return small_rows ? launch_t<T, C, XS, 1, 4>(a, s) : launch_t<T, C, XS, 4, 4>(a, s);
  return small_rows ? launch_t<T, C, XS, 1, 10>(a, s) : launch_t<T, C, XS, 4, 10>(a, s);
}

template <typename XS, int RPT, int CPT>
cudaError_t launch_batch_t(const MttkrpArgs* jobs, const int4* items, const void* const* xptrs, int nitems, int BK,
                           size_t smem, cudaStream_t s) {
  auto kern = mttkrp_batch_kernel<float, false, XS, RPT, CPT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  launch_k(kern, (unsigned)nitems, 256, smem, s, jobs, items, xptrs, BK);
  return cudaGetLastError();
}

template <typename XS>
cudaError_t launch_batch_x(const MttkrpArgs* jobs, const int4* items, const void* const* xptrs, int nitems, int cls,
                           int BK, size_t smem, cudaStream_t s) {
  switch (cls) {
    case 0: return launch_batch_t<XS, 1, 1>(jobs, items, xptrs, nitems, BK, smem, s);
    case 1: return launch_batch_t<XS, 4, 1>(jobs, items, xptrs, nitems, BK, smem, s);
    case 2: return launch_batch_t<XS, 1, 4>(jobs, items, xptrs, nitems, BK, smem, s);
    case 3: return launch_batch_t<XS, 4, 4>(jobs, items, xptrs, nitems, BK, smem, s);
    case 4: return launch_batch_t<XS, 1, 10>(jobs, items, xptrs, nitems, BK, smem, s);
    default: return launch_batch_t<XS, 4, 10>(jobs, items, xptrs, nitems, BK, smem, s);
  }
}

}  // namespace

// register-block class of launch_rc: 0..5 = (RPT, CPT) in (1,1) (4,1) (1,4) (4,4) (1,10) (4,10)
int mttkrp_class(const MttkrpArgs& a) {
  const int RR = a.R[a.n] * a.R[a.n + 1];
  const bool small_rows = a.dim[a.n] <= 16;
  const int c = RR <= 16 ? 0 : (RR <= 64 ? 2 : 4);
  return c + (small_rows ? 0 : 1);
}

int mttkrp_rows_per_block(const MttkrpArgs& a) { return (mttkrp_class(a) & 1) ? 64 : 16; }

size_t mttkrp_smem_bytes(const MttkrpArgs& a, int BK) { return smem_bytes(a, BK, mttkrp_rows_per_block(a)); }

// FP32 dense (real) jobs only: the batched path of FP32 slab arithmetic
cudaError_t launch_mttkrp_batch(const MttkrpArgs* jobs, const int4* items, const void* const* xptrs, int nitems,
                                int cls, int xtype, int BK, size_t smem, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  switch (xtype) {
    case XT_F64: return launch_batch_x<double>(jobs, items, xptrs, nitems, cls, BK, smem, s);
    case XT_F32: return launch_batch_x<float>(jobs, items, xptrs, nitems, cls, BK, smem, s);
    default: return launch_batch_x<__nv_bfloat16>(jobs, items, xptrs, nitems, cls, BK, smem, s);
  }
}

int mttkrp_plan_splits(const MttkrpArgs& a, int64_t* fib_per_split) {
  const int BM = a.dim[a.n] <= 16 ? 16 : 64;
  const int gx = ceil_div_i(a.dim[a.n], BM);
  const int target = 2 * 152;
  // sampled problems have few fibres (the sketch size): smaller chunks keep the SMs busy
  int64_t min_chunk = a.idxs ? 32 : 256;
  int64_t splits = std::max<int64_t>(1, target / std::max(1, gx));
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, (a.nfib + min_chunk - 1) / min_chunk));
  int64_t per = (a.nfib + splits - 1) / splits;
  per = std::max<int64_t>(per, 1);
  splits = (a.nfib + per - 1) / per;
  if (splits < 1) splits = 1;
  *fib_per_split = per;
  return (int)splits;
}

cudaError_t launch_mttkrp(const MttkrpArgs& a, cudaStream_t s) {
  if (a.cplx) {
    if (a.compute == 2) return launch_rc<double, true, cplx<double>>(a, s);
    return launch_rc<float, true, cplx<float>>(a, s);
  }
  if (a.compute == 2) {
    switch (a.xtype) {
      case XT_F64: return launch_rc<double, false, double>(a, s);
      case XT_F32: return launch_rc<double, false, float>(a, s);
      default: return launch_rc<double, false, __nv_bfloat16>(a, s);
    }
  }
  switch (a.xtype) {
    case XT_F64: return launch_rc<float, false, double>(a, s);
    case XT_F32: return launch_rc<float, false, float>(a, s);
    default: return launch_rc<float, false, __nv_bfloat16>(a, s);
  }
}

// ---------------------------------------------------------------------------
// fixed-order reduction of split partials: a CTA owns 16 outputs; its 16 lane
// groups each sum the splits g, g+16, g+32, ... and the 16 group sums are then
// added in group order -- the same order on every run (no atomics).
// ---------------------------------------------------------------------------
// outputs 16 bx .. 16 bx + 15
template <typename T, bool CPLX>
__device__ __forceinline__ void reduce_body(const T* __restrict__ partial, int splits, int64_t count,
                                            const double* __restrict__ base, double scale,
                                            double* __restrict__ out, int64_t bx) {
  constexpr int W = CPLX ? 2 : 1;
  __shared__ double red[16][16 * W];
  const int o = threadIdx.x & 15, g = threadIdx.x >> 4;
  const int64_t i = bx * 16 + o;
  double acc[W];
#pragma unroll
  for (int w = 0; w < W; ++w) acc[w] = 0.0;
  if (i < count) {
    for (int k = g; k < splits; k += 16) {
#pragma unroll
      for (int w = 0; w < W; ++w) acc[w] += (double)partial[((int64_t)k * count + i) * W + w];
    }
  }
#pragma unroll
  for (int w = 0; w < W; ++w) red[g][o * W + w] = acc[w];
  __syncthreads();
  if (g == 0 && i < count) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      double sum = 0.0;
      for (int q = 0; q < 16; ++q) sum += red[q][o * W + w];
      if (CPLX) out[2 * i + w] = scale * sum;
      else out[i] = (base ? base[i] : 0.0) + scale * sum;
    }
  }
}

template <typename T, bool CPLX>
__global__ void __launch_bounds__(256) reduce_kernel(const T* __restrict__ partial, int splits,
                                                     int64_t count, const double* __restrict__ base,
                                                     double scale, double* __restrict__ out) {
  PDL_ENTRY();
  reduce_body<T, CPLX>(partial, splits, count, base, scale, out, blockIdx.x);
}

// work list of split reductions: item = (job, block of 256 outputs), one thread
// per output.  The thread forms reduce_body's sum in reduce_body's order: group
// g sums the splits g, g + 16, ... in FP64, then the 16 group sums are added in
// group order (the same FP64 operations, so the same result)
__global__ void __launch_bounds__(256) reduce_batch_kernel(const ReduceJob* __restrict__ jobs,
                                                           const int2* __restrict__ items) {
  PDL_ENTRY();
  const int2 it = items[blockIdx.x];
  const ReduceJob j = jobs[it.x];
  const int64_t i = (int64_t)it.y * 256 + threadIdx.x;
  if (i >= j.count) return;
  double sum = 0.0;
  for (int g = 0; g < 16; ++g) {
    double acc = 0.0;
    for (int k = g; k < j.splits; k += 16) acc += (double)j.partial[(int64_t)k * j.count + i];
    sum += acc;
  }
  j.out[i] = (j.base ? j.base[i] : 0.0) + 1.0 * sum;
}

// work list of copies: item = (job, 16 KB chunk)
__global__ void __launch_bounds__(256) copy_batch_kernel(const CopyJob* __restrict__ jobs,
                                                         const int2* __restrict__ items) {
  PDL_ENTRY();
  const int2 it = items[blockIdx.x];
  const CopyJob j = jobs[it.x];
  const int64_t b0 = (int64_t)it.y * 16384, b1 = min(j.bytes, b0 + 16384);
  const bool v16 = ((((uintptr_t)j.src) | ((uintptr_t)j.dst)) & 15) == 0 && (j.bytes & 15) == 0;
  if (v16) {
    const uint4* s4 = (const uint4*)j.src;
    uint4* d4 = (uint4*)j.dst;
    for (int64_t e = (b0 >> 4) + threadIdx.x; e < (b1 >> 4); e += blockDim.x) d4[e] = s4[e];
  } else {
    const unsigned char* s1 = (const unsigned char*)j.src;
    unsigned char* d1 = (unsigned char*)j.dst;
    for (int64_t e = b0 + threadIdx.x; e < b1; e += blockDim.x) d1[e] = s1[e];
  }
}

// out[i] = *ptrs[i]: the status words of many contexts in one array
__global__ void gather_ints_kernel(const int* const* __restrict__ ptrs, int n, int* __restrict__ out) {
  PDL_ENTRY();
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = *ptrs[i];
}

cudaError_t launch_gather_ints(const int* const* ptrs, int n, int* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  launch_k(gather_ints_kernel, (unsigned)std::min(64, (n + 255) / 256), 256, 0, s, ptrs, n, out);
  return cudaGetLastError();
}

cudaError_t launch_reduce_batch(const ReduceJob* jobs, const int2* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  launch_k(reduce_batch_kernel, (unsigned)nitems, 256, 0, s, jobs, items);
  return cudaGetLastError();
}

cudaError_t launch_copy_batch(const CopyJob* jobs, const int2* items, int nitems, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  launch_k(copy_batch_kernel, (unsigned)nitems, 256, 0, s, jobs, items);
  return cudaGetLastError();
}

static unsigned grid_for(int64_t count) {
  int64_t g = (count + 255) / 256;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, 4096));
}

cudaError_t launch_reduce_partials(const void* partial, int compute, int cplx, int splits,
                                   int64_t count, const double* base, double scale, double* out,
                                   cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((count + 15) / 16);
  if (cplx) {
    if (compute == 2) launch_k(reduce_kernel<double, true>, blocks, 256, 0, s, (const double*)partial, splits, count, nullptr, scale, out);
    else launch_k(reduce_kernel<float, true>, blocks, 256, 0, s, (const float*)partial, splits, count, nullptr, scale, out);
  } else {
    if (compute == 2) launch_k(reduce_kernel<double, false>, blocks, 256, 0, s, (const double*)partial, splits, count, base, scale, out);
    else launch_k(reduce_kernel<float, false>, blocks, 256, 0, s, (const float*)partial, splits, count, base, scale, out);
  }
  return cudaGetLastError();
}

template <typename T, typename O>
__global__ void reduce_to_kernel(const T* partial, int splits, int64_t count, double scale, O* out) {
  PDL_ENTRY();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += (double)partial[(int64_t)k * count + i];
    out[i] = (O)(scale * s);
  }
}

// many splits: one warp per output, lane l sums the splits l, l + 32, ... and the
// 32 lane sums are combined by a fixed butterfly (same order on every run)
template <typename T, typename O>
__global__ void reduce_to_warp_kernel(const T* partial, int splits, int64_t count, double scale, O* out) {
  PDL_ENTRY();
  const int lane = threadIdx.x & 31;
  for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < count;
       i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    double s = 0.0;
    for (int k = lane; k < splits; k += 32) s += (double)partial[(int64_t)k * count + i];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = (O)(scale * s);
  }
}

cudaError_t launch_reduce_partials_to(const void* partial, int compute, int splits, int64_t count,
                                      double scale, void* out, int out_type, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (splits >= 64) {
    const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count * 32 + 255) / 256, 152 * 16));
#define STR_RW(T, O) launch_k(reduce_to_warp_kernel<T, O>, g, 256, 0, s, (const T*)partial, splits, count, scale, (O*)out)
    if (compute == 2) {
      if (out_type == XT_F64) STR_RW(double, double); else STR_RW(double, float);
    } else {
      if (out_type == XT_F64) STR_RW(float, double); else STR_RW(float, float);
    }
#undef STR_RW
    return cudaGetLastError();
  }
  if (compute == 2) {
    if (out_type == XT_F64) launch_k(reduce_to_kernel<double, double>, grid_for(count), 256, 0, s, (const double*)partial, splits, count, scale, (double*)out);
    else launch_k(reduce_to_kernel<double, float>, grid_for(count), 256, 0, s, (const double*)partial, splits, count, scale, (float*)out);
  } else {
    if (out_type == XT_F64) launch_k(reduce_to_kernel<float, double>, grid_for(count), 256, 0, s, (const float*)partial, splits, count, scale, (double*)out);
    else launch_k(reduce_to_kernel<float, float>, grid_for(count), 256, 0, s, (const float*)partial, splits, count, scale, (float*)out);
  }
  return cudaGetLastError();
}
