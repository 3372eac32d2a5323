// Sketch kernels for rSTR: Philox row draws (Eq. sampDS; Lemma lev_est),
// random sign flips and unitary DFT mixing (Definition of the KSRFT), the
// weighted Gram of the sampled subchain (Alg. 5), and small utilities.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "kernels.cuh"

// ---------------------------------------------------------------------------
// row draws: uniform floor(u I / 2^64), or weighted from the sequential CDF of p
// ---------------------------------------------------------------------------
__global__ void draw_indices_kernel(int32_t* __restrict__ out, int64_t m, int64_t I, uint64_t seed,
                                    int k, uint64_t tau, uint32_t sid, const double* __restrict__ p) {
  PDL_ENTRY();
  extern __shared__ double cdf[];
  __shared__ int s_last;
  if (p) {
    if (threadIdx.x == 0) {
      double c = 0.0;
      int last = (int)I - 1;
      for (int64_t i = 0; i < I; ++i) {
        c = c + p[i];     // sequential left-to-right prefix sums
        cdf[i] = c;
      }
      for (int64_t i = I - 1; i >= 0; --i)
        if (p[i] > 0.0) { last = (int)i; break; }
      s_last = last;
    }
    __syncthreads();
  }
  for (int64_t sidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sidx < m;
       sidx += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = draw_u64(seed, (uint64_t)sidx, (uint64_t)k, tau, 0u, sid);
    int64_t idx;
    if (p) {
      const double v = (double)(u >> 11) * 0x1.0p-53;
      const double target = v * cdf[I - 1];
      // first i with cdf[i] > target
      int64_t lo = 0, hi = I;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cdf[mid] > target) hi = mid; else lo = mid + 1;
      }
      idx = (lo < I) ? lo : s_last;
    } else {
      idx = (int64_t)__umul64hi(u, (uint64_t)I);
    }
    out[sidx] = (int32_t)idx;
  }
}

cudaError_t launch_draw_indices(int32_t* out, int64_t m, int64_t I, uint64_t seed, int k,
                                uint64_t tau, uint32_t stream_id, const double* p, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  size_t sm = p ? (size_t)I * sizeof(double) : 0;
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(draw_indices_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((m + 511) / 512, 152));
  launch_k(draw_indices_kernel, (unsigned)blocks, 512, sm, s, out, m, I, seed, k, tau, stream_id, p);
  return cudaGetLastError();
}

__global__ void signs_kernel(double* d, int64_t I, uint64_t seed, int k, uint64_t tau, uint32_t sid) {
  PDL_ENTRY();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < I;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t u = draw_u64(seed, (uint64_t)i, (uint64_t)k, tau, 1u, sid);
    d[i] = (u & 1ull) ? -1.0 : 1.0;
  }
}

cudaError_t launch_signs(double* d, int64_t I, uint64_t seed, int k, uint64_t tau,
                         uint32_t stream_id, cudaStream_t s) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((I + 255) / 256, 256));
  launch_k(signs_kernel, (unsigned)blocks, 256, 0, s, d, I, seed, k, tau, stream_id);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// weighted Gram of sampled rows: out = base + sum_s w_s Re(g_s g_s^H), FP64
// 16x16 output tile per CTA, sample chunks staged in shared memory.
// ---------------------------------------------------------------------------
template <typename T, bool C>
__global__ void __launch_bounds__(256) wgram_kernel(const T* __restrict__ g, const double* __restrict__ w,
                                                    int64_t m, int64_t per, int RR, double* __restrict__ part) {
  PDL_ENTRY();
  constexpr int CH = 32;
  constexpr int W = C ? 2 : 1;
  __shared__ double sa[CH][16 * W], sb[CH][16 * W];
  __shared__ double sw[CH];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.y * 16, c0 = blockIdx.x * 16;
  const int64_t sbeg = (int64_t)blockIdx.z * per, send = min(m, sbeg + per);
  double acc = 0.0;
  for (int64_t s0 = sbeg; s0 < send; s0 += CH) {
    const int ns = (send - s0 < CH) ? (int)(send - s0) : CH;
    for (int e = threadIdx.x; e < CH * 16 * W; e += 256) {
      const int ss = e / (16 * W), x = e % (16 * W);
      const int cc = x / W, part = x % W;
      double va = 0.0, vb = 0.0;
      if (ss < ns) {
        if (r0 + cc < RR) va = (double)g[((s0 + ss) * RR + r0 + cc) * W + part];
        if (c0 + cc < RR) vb = (double)g[((s0 + ss) * RR + c0 + cc) * W + part];
      }
      sa[ss][x] = va;
      sb[ss][x] = vb;
    }
    for (int e = threadIdx.x; e < CH; e += 256) sw[e] = (e < ns) ? (w ? w[s0 + e] : 1.0) : 0.0;
    __syncthreads();
    for (int ss = 0; ss < ns; ++ss) {
      double v;
      if (C) v = sa[ss][2 * ty] * sb[ss][2 * tx] + sa[ss][2 * ty + 1] * sb[ss][2 * tx + 1];
      else v = sa[ss][ty] * sb[ss][tx];
      acc = fma(sw[ss], v, acc);
    }
    __syncthreads();
  }
  const int r = r0 + ty, c = c0 + tx;
  if (r < RR && c < RR) part[((int64_t)blockIdx.z * RR + r) * RR + c] = acc;
}

// Same weighted Gram for FP32 samples (real or complex) without the FP64 pipe: every term
// w_s g_a g_b is formed as an FP32 pair (g_a g_b exactly by FMA, times the
// weight carried as an FP32 pair) and summed with error-free transformations
// (Dekker / Knuth), so the split sum carries about 44 significant bits.
__device__ __forceinline__ void pair_add(float& sh, float& sl, float ph, float pl) {
  const float t = sh + ph;
  const float bb = t - sh;
  const float e = (sh - (t - bb)) + (ph - bb);
  sh = t;
  sl += e + pl;
}

// C: complex samples, term w_s Re(g_a conj(g_b)) = w_s (re_a re_b + im_a im_b),
// both products exact pairs, summed error-free before the weight
template <bool C>
__global__ void __launch_bounds__(256) wgram_pair_kernel(const float* __restrict__ g, const double* __restrict__ w,
                                                         int64_t m, int64_t per, int RR, double* __restrict__ part) {
  PDL_ENTRY();
  constexpr int CH = 64;
  constexpr int W = C ? 2 : 1;
  __shared__ float sa[CH][16 * W], sb[CH][16 * W];
  __shared__ float swh[CH], swl[CH];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.y * 16, c0 = blockIdx.x * 16;
  const int64_t sbeg = (int64_t)blockIdx.z * per, send = min(m, sbeg + per);
  float sh = 0.f, sl = 0.f;
  for (int64_t s0 = sbeg; s0 < send; s0 += CH) {
    const int ns = (send - s0 < CH) ? (int)(send - s0) : CH;
    for (int e = threadIdx.x; e < CH * 16 * W; e += 256) {
      const int ss = e / (16 * W), x = e % (16 * W);
      const int cc = x / W, q = x % W;
      float va = 0.f, vb = 0.f;
      if (ss < ns) {
        if (r0 + cc < RR) va = g[((s0 + ss) * RR + r0 + cc) * W + q];
        if (c0 + cc < RR) vb = g[((s0 + ss) * RR + c0 + cc) * W + q];
      }
      sa[ss][x] = va;
      sb[ss][x] = vb;
    }
    for (int e = threadIdx.x; e < CH; e += 256) {
      const double wv = (e < ns) ? (w ? w[s0 + e] : 1.0) : 0.0;
      const float wh = (float)wv;
      swh[e] = wh;
      swl[e] = (float)(wv - (double)wh);
    }
    __syncthreads();
    for (int ss = 0; ss < ns; ++ss) {
      float ph, pl;
      if (C) {
        const float ar = sa[ss][2 * ty], ai = sa[ss][2 * ty + 1], br = sb[ss][2 * tx], bi = sb[ss][2 * tx + 1];
        const float h1 = ar * br, l1 = fmaf(ar, br, -h1);   // exact products
        const float h2 = ai * bi, l2 = fmaf(ai, bi, -h2);
        ph = h1 + h2;                                       // two-sum of the high parts
        const float bb = ph - h1;
        pl = ((h1 - (ph - bb)) + (h2 - bb)) + (l1 + l2);
      } else {
        const float a = sa[ss][ty], b = sb[ss][tx];
        ph = a * b;
        pl = fmaf(a, b, -ph);                     // a b = ph + pl exactly
      }
      const float wh = swh[ss], wl = swl[ss];
      const float th = wh * ph;
      float tl = fmaf(wh, ph, -th);              // wh ph = th + tl exactly
      tl = fmaf(wh, pl, fmaf(wl, ph, tl));       // + wh pl + wl ph
      pair_add(sh, sl, th, tl);
    }
    __syncthreads();
  }
  const int r = r0 + ty, c = c0 + tx;
  if (r < RR && c < RR) part[((int64_t)blockIdx.z * RR + r) * RR + c] = (double)sh + (double)sl;
}

// out = base + sum over sample splits (fixed order), FP64
cudaError_t launch_weighted_gram(const void* gs, int compute, int cplx, const double* w, int64_t m, int RR,
                                 const double* base, double* out, double* part, cudaStream_t s) {
  const int tiles = ceil_div_i(RR, 16) * ceil_div_i(RR, 16);
  int64_t splits = std::max<int64_t>(1, (4 * 152 + tiles - 1) / tiles);
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, m / 64));
  splits = std::min<int64_t>(splits, 64);
  const int64_t per = (m + splits - 1) / splits;
  splits = (m + per - 1) / per;
  dim3 grid((unsigned)ceil_div_i(RR, 16), (unsigned)ceil_div_i(RR, 16), (unsigned)splits);
  if (compute == 2) {
    if (cplx) launch_k(wgram_kernel<double, true>, grid, 256, 0, s, (const double*)gs, w, m, per, RR, part);
    else launch_k(wgram_kernel<double, false>, grid, 256, 0, s, (const double*)gs, w, m, per, RR, part);
  } else {
    if (cplx) launch_k(wgram_pair_kernel<true>, grid, 256, 0, s, (const float*)gs, w, m, per, RR, part);
    else launch_k(wgram_pair_kernel<false>, grid, 256, 0, s, (const float*)gs, w, m, per, RR, part);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_reduce_partials(part, 2, 0, (int)splits, (int64_t)RR * RR, base, 1.0, out, s);
}

// ---------------------------------------------------------------------------
// unitary DFT along one mode with a sign pre-multiply (X x_j F_j D_j).
// A CTA takes FB fibres that are adjacent in memory and stages them [L][FB].
// Twiddles: cos/sin(2 pi j / L) for j < L, computed once on the host side of
// the launch in FP64 and indexed by (k * i) mod L.
// ---------------------------------------------------------------------------
template <typename T, int FB>
__global__ void dft_mode_kernel(const void* __restrict__ in, int in_type, T* __restrict__ out,
                                int L, int64_t inner, int64_t nfib, const double* __restrict__ d,
                                const double* __restrict__ tw) {
  PDL_ENTRY();
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sre = (T*)smraw;                 // L * FB
  T* sim = sre + L * FB;              // L * FB
  T* cs = sim + L * FB;               // L
  T* sn = cs + L;                     // L
  __shared__ int64_t fbase[FB];       // offset of element 0 of each staged fibre
  for (int j = threadIdx.x; j < L; j += blockDim.x) { cs[j] = (T)tw[2 * j]; sn[j] = (T)tw[2 * j + 1]; }
  const T scale = (T)(1.0 / sqrt((double)L));
  for (int64_t fb0 = (int64_t)blockIdx.x * FB; fb0 < nfib; fb0 += (int64_t)gridDim.x * FB) {
    // fibre f: inner index = f % inner, outer = f / inner; element i at
    // outer * L * inner + i * inner + inner_idx
    if (threadIdx.x < FB) {
      const int64_t f = fb0 + threadIdx.x;
      fbase[threadIdx.x] = f < nfib ? (f / inner) * (int64_t)L * inner + (f % inner) : -1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < L * FB; e += blockDim.x) {
      const int ff = e % FB, i = e / FB;
      const int64_t fo = fbase[ff];
      T re = 0, im = 0;
      if (fo >= 0) {
        const int64_t o = fo + (int64_t)i * inner;
        switch (in_type) {
          case XT_BF16: re = (T)__bfloat162float(((const __nv_bfloat16*)in)[o]); break;
          case XT_F32: re = (T)((const float*)in)[o]; break;
          case XT_F64: re = (T)((const double*)in)[o]; break;
          case XT_C32: re = (T)((const float*)in)[2 * o]; im = (T)((const float*)in)[2 * o + 1]; break;
          default: re = (T)((const double*)in)[2 * o]; im = (T)((const double*)in)[2 * o + 1]; break;
        }
        if (d) { re *= (T)d[i]; im *= (T)d[i]; }
      }
      sre[i * FB + ff] = re;
      sim[i * FB + ff] = im;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < L * FB; e += blockDim.x) {
      const int ff = e % FB, kk = e / FB;
      const int64_t fo = fbase[ff];
      T are = 0, aim = 0;
      int ph = 0;   // (kk * i) mod L
      for (int i = 0; i < L; ++i) {
        const T c = cs[ph], sv = sn[ph];     // F(k,i) = c - i s
        const T xr = sre[i * FB + ff], xi = sim[i * FB + ff];
        are += c * xr + sv * xi;
        aim += c * xi - sv * xr;
        ph += kk;
        if (ph >= L) ph -= L;
      }
      if (fo >= 0) {
        const int64_t o = fo + (int64_t)kk * inner;
        out[2 * o] = are * scale;
        out[2 * o + 1] = aim * scale;
      }
    }
    __syncthreads();
  }
}

// twiddle tables cached per length (host-computed cos/sin in FP64)
static std::mutex g_tw_mu;
static std::map<std::pair<int, int64_t>, double*> g_tw;

static const double* twiddles(int64_t L) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_tw_mu);
  auto key = std::make_pair(dev, L);
  auto it = g_tw.find(key);
  if (it != g_tw.end()) return it->second;
  std::vector<double> h(2 * L);
  for (int64_t j = 0; j < L; ++j) {
    const double th = 2.0 * 3.14159265358979323846 * (double)j / (double)L;
    h[2 * j] = cos(th);
    h[2 * j + 1] = sin(th);
  }
  double* dptr = nullptr;
  if (cudaMalloc(&dptr, 2 * L * sizeof(double)) != cudaSuccess) return nullptr;
  // a copy from pageable memory may still be in flight when cudaMemcpy returns, and
  // the legacy stream does not order the non-blocking streams that read the table
  if (cudaMemcpy(dptr, h.data(), 2 * L * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dptr);
    return nullptr;
  }
  g_tw[key] = dptr;
  return dptr;
}

// ---------------------------------------------------------------------------
// radix-2 FFT along one mode (power-of-two length L <= 4096), in shared memory:
// bit-reversed load (with the sign pre-multiply), log2(L) in-place butterfly
// stages (decimation in time), then either the unitary transform written as
// complex values, or (inverse, unmixing) base + d_k * Re(result) as FP64.
// ---------------------------------------------------------------------------
template <typename T, int FB>
__global__ void fft_mode_kernel(const void* __restrict__ in, int in_type, void* __restrict__ out,
                                int out_real, const double* __restrict__ base, int L, int logL,
                                int64_t inner, int64_t nfib, const double* __restrict__ dpre,
                                const double* __restrict__ dpost, int inverse,
                                const double* __restrict__ tw) {
  PDL_ENTRY();
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int FS = FB + 1;           // odd row stride: natural-order rows are conflict-free
  T* sre = (T*)smraw;                 // L * FS
  T* sim = sre + L * FS;              // L * FS
  T* cs = sim + L * FS;               // L
  T* sn = cs + L;                     // L
  __shared__ int64_t fbase[FB];       // offset of element 0 of each staged fibre
  for (int j = threadIdx.x; j < L; j += blockDim.x) { cs[j] = (T)tw[2 * j]; sn[j] = (T)tw[2 * j + 1]; }
  const T scale = (T)(1.0 / sqrt((double)L));
  const T sgn = inverse ? (T)1 : (T)-1;   // exp(sgn * 2 pi i t / L) = cos + sgn * i sin
  // inner == 1: a fibre is L contiguous elements, threads run along it (coalesced);
  // otherwise adjacent fibres are adjacent in memory, threads run across them
  const bool along = inner == 1;
  for (int64_t fb0 = (int64_t)blockIdx.x * FB; fb0 < nfib; fb0 += (int64_t)gridDim.x * FB) {
    if (threadIdx.x < FB) {
      const int64_t f = fb0 + threadIdx.x;
      fbase[threadIdx.x] = f < nfib ? (f / inner) * (int64_t)L * inner + (f % inner) : -1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < L * FB; e += blockDim.x) {
      const int ff = along ? e >> logL : e % FB;
      const int i = along ? e & (L - 1) : e / FB;
      const int64_t fo = fbase[ff];
      T re = 0, im = 0;
      if (fo >= 0) {
        const int64_t o = fo + (int64_t)i * inner;
        switch (in_type) {
          case XT_BF16: re = (T)__bfloat162float(((const __nv_bfloat16*)in)[o]); break;
          case XT_F32: re = (T)((const float*)in)[o]; break;
          case XT_F64: re = (T)((const double*)in)[o]; break;
          case XT_C32: re = (T)((const float*)in)[2 * o]; im = (T)((const float*)in)[2 * o + 1]; break;
          default: re = (T)((const double*)in)[2 * o]; im = (T)((const double*)in)[2 * o + 1]; break;
        }
        if (dpre) { re *= (T)dpre[i]; im *= (T)dpre[i]; }
      }
      const int br = (int)(__brev((unsigned)i) >> (32 - logL));
      sre[br * FS + ff] = re;
      sim[br * FS + ff] = im;
    }
    __syncthreads();
    for (int st = 0; st < logL; ++st) {
      const int half = 1 << st;
      const int tstep = L >> (st + 1);     // twiddle index stride = L / len
      for (int e = threadIdx.x; e < (L / 2) * FB; e += blockDim.x) {
        const int ff = e % FB;
        const int b = e / FB;
        const int g = b >> st, j = b & (half - 1);
        const int i0 = g * 2 * half + j, i1 = i0 + half;
        const int t = j * tstep;
        const T wr = cs[t], wi = sgn * sn[t];
        const T xr = sre[i1 * FS + ff], xi = sim[i1 * FS + ff];
        const T vr = xr * wr - xi * wi, vi = xr * wi + xi * wr;
        const T ur = sre[i0 * FS + ff], ui = sim[i0 * FS + ff];
        sre[i0 * FS + ff] = ur + vr;
        sim[i0 * FS + ff] = ui + vi;
        sre[i1 * FS + ff] = ur - vr;
        sim[i1 * FS + ff] = ui - vi;
      }
      __syncthreads();
    }
    for (int e = threadIdx.x; e < L * FB; e += blockDim.x) {
      const int ff = along ? e >> logL : e % FB;
      const int kk = along ? e & (L - 1) : e / FB;
      const int64_t fo = fbase[ff];
      if (fo >= 0) {
        const int64_t o = fo + (int64_t)kk * inner;
        T yr = sre[kk * FS + ff] * scale, yi = sim[kk * FS + ff] * scale;
        if (dpost) { yr *= (T)dpost[kk]; yi *= (T)dpost[kk]; }
        if (out_real) ((double*)out)[o] = (base ? base[o] : 0.0) + (double)yr;
        else { ((T*)out)[2 * o] = yr; ((T*)out)[2 * o + 1] = yi; }
      }
    }
    __syncthreads();
  }
}

static int log2_exact(int64_t L) {
  if (L < 2 || L > 4096 || (L & (L - 1))) return -1;
  int lg = 0;
  while (((int64_t)1 << lg) < L) ++lg;
  return lg;
}

template <typename T>
static cudaError_t launch_fft(const void* in, int in_type, void* out, int out_real, const double* base,
                              int64_t L, int logL, int64_t inner, int64_t nfib, const double* dpre,
                              const double* dpost, int inverse, const double* tw, cudaStream_t s) {
  const int tsize = sizeof(T);
  // fibres per CTA: up to 16, fewer when there are few fibres (two CTAs per SM at least)
  int FB = 16;
  while (FB > 1 && (size_t)(2 * L * (FB + 1) + 2 * L) * tsize > 96 * 1024) FB /= 2;
  while (FB > 1 && (nfib + FB - 1) / FB < 2 * 152) FB /= 2;
  const size_t sm = (size_t)(2 * L * (FB + 1) + 2 * L) * tsize;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((nfib + FB - 1) / FB, 152 * 8));
#define STR_FFT_CASE(F)                                                                                   \
  do {                                                                                                    \
    cudaError_t e = cudaFuncSetAttribute(fft_mode_kernel<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)sm);                                                        \
    if (e != cudaSuccess) return e;                                                                       \
    launch_k(fft_mode_kernel<T, F>, (unsigned)blocks, 256, sm, s, in, in_type, out, out_real, base, (int)L, \
             logL, inner, nfib, dpre, dpost, inverse, tw);                                                \
  } while (0)
  switch (FB) {
    case 16: STR_FFT_CASE(16); break;
    case 8: STR_FFT_CASE(8); break;
    case 4: STR_FFT_CASE(4); break;
    case 2: STR_FFT_CASE(2); break;
    default: STR_FFT_CASE(1); break;
  }
#undef STR_FFT_CASE
  return cudaGetLastError();
}

cudaError_t launch_dft_mode(const void* in, int in_type, void* out, int out_cplx_compute, int N,
                            const int64_t* dims, int mode, const double* d, cudaStream_t s) {
  const int64_t L = dims[mode];
  int64_t inner = 1, total = 1;
  for (int k = 0; k < N; ++k) { total *= dims[k]; if (k < mode) inner *= dims[k]; }
  const int64_t nfib = total / L;
  const double* tw = twiddles(L);
  if (!tw) return cudaErrorMemoryAllocation;
  const int logL = log2_exact(L);
  if (logL > 0) {
    if (out_cplx_compute == 2) return launch_fft<double>(in, in_type, out, 0, nullptr, L, logL, inner, nfib, d, nullptr, 0, tw, s);
    return launch_fft<float>(in, in_type, out, 0, nullptr, L, logL, inner, nfib, d, nullptr, 0, tw, s);
  }
  const int tsize = out_cplx_compute == 2 ? 8 : 4;
  if (L > 16384) return cudaErrorInvalidValue;
  int FB = 16;
  while (FB > 1 && (size_t)(2 * L * FB + 2 * L) * tsize > 96 * 1024) FB /= 2;
  const size_t sm = (size_t)(2 * L * FB + 2 * L) * tsize;
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((nfib + FB - 1) / FB, 152 * 8));
#define STR_DFT_CASE(T, F)                                                                                \
  do {                                                                                                    \
    cudaError_t e = cudaFuncSetAttribute(dft_mode_kernel<T, F>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)sm);                                                        \
    if (e != cudaSuccess) return e;                                                                       \
    launch_k(dft_mode_kernel<T, F>, (unsigned)blocks, 256, sm, s, in, in_type, (T*)out, (int)L, inner, nfib, d, tw); \
  } while (0)
#define STR_DFT_FB(T)                    \
  switch (FB) {                          \
    case 16: STR_DFT_CASE(T, 16); break; \
    case 8: STR_DFT_CASE(T, 8); break;   \
    case 4: STR_DFT_CASE(T, 4); break;   \
    case 2: STR_DFT_CASE(T, 2); break;   \
    default: STR_DFT_CASE(T, 1); break;  \
  }
  if (out_cplx_compute == 2) {
    STR_DFT_FB(double);
  } else {
    STR_DFT_FB(float);
  }
#undef STR_DFT_FB
#undef STR_DFT_CASE
  return cudaGetLastError();
}

// out[k][c] = base[k][c] + Re( d_k * sum_i conj(F(i,k)) Y[i][c] ),
// conj(F(i,k)) = (cos th + i sin th)/sqrt(L), th = 2 pi (i k mod L) / L
__global__ void unmix_rows_kernel(const double* __restrict__ Y, int64_t L, int RR,
                                  const double* __restrict__ d, const double* __restrict__ tw,
                                  const double* __restrict__ base, double* __restrict__ out) {
  PDL_ENTRY();
  const double scale = 1.0 / sqrt((double)L);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L * RR;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e / RR;
    const int c = (int)(e % RR);
    double acc = 0.0;
    int64_t ph = 0;
    for (int64_t i = 0; i < L; ++i) {
      acc += tw[2 * ph] * Y[2 * (i * RR + c)] - tw[2 * ph + 1] * Y[2 * (i * RR + c) + 1];
      ph += k;
      if (ph >= L) ph -= L;
    }
    out[e] = (base ? base[e] : 0.0) + d[k] * acc * scale;
  }
}

cudaError_t launch_unmix_rows(const double* Y, int64_t L, int RR, const double* d,
                              const double* base, double* out, cudaStream_t s) {
  const double* tw = twiddles(L);
  if (!tw) return cudaErrorMemoryAllocation;
  const int logL = log2_exact(L);
  if (logL > 0)   // Y as a (RR, L) tensor, inverse transform along L
    return launch_fft<double>(Y, XT_C64, out, 1, base, L, logL, RR, RR, nullptr, d, 1, tw, s);
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((L * RR + 255) / 256, 2048));
  launch_k(unmix_rows_kernel, (unsigned)blocks, 256, 0, s, Y, L, RR, d, tw, base, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// utilities
// ---------------------------------------------------------------------------
template <typename I, typename O>
__global__ void convert_kernel(const I* __restrict__ in, O* __restrict__ out, int64_t count) {
  PDL_ENTRY();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (O)in[i];
}

cudaError_t launch_convert(const void* in, int in_type, void* out, int out_type, int64_t count,
                           cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 4096));
  if (in_type == XT_F64 && out_type == XT_F32) launch_k(convert_kernel<double, float>, blocks, 256, 0, s, (const double*)in, (float*)out, count);
  else if (in_type == XT_F32 && out_type == XT_F64) launch_k(convert_kernel<float, double>, blocks, 256, 0, s, (const float*)in, (double*)out, count);
  else if (in_type == XT_F64 && out_type == XT_F64) launch_k(convert_kernel<double, double>, blocks, 256, 0, s, (const double*)in, (double*)out, count);
  else if (in_type == XT_F32 && out_type == XT_F32) launch_k(convert_kernel<float, float>, blocks, 256, 0, s, (const float*)in, (float*)out, count);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <typename T>
__global__ void check_finite_kernel(const T* __restrict__ x, int64_t count, int* status) {
  PDL_ENTRY();
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (!isfinite((double)x[i])) bad = true;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, DEV_ERR_NONFINITE);
}
__global__ void check_finite_bf16_kernel(const __nv_bfloat16* __restrict__ x, int64_t count, int* status) {
  PDL_ENTRY();
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(__bfloat162float(x[i]))) bad = true;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, DEV_ERR_NONFINITE);
}

cudaError_t launch_check_finite(const void* X, int xtype, int64_t count, int* status, cudaStream_t s) {
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152 * 8));
  if (xtype == XT_F64) launch_k(check_finite_kernel<double>, blocks, 256, 0, s, (const double*)X, count, status);
  else if (xtype == XT_F32) launch_k(check_finite_kernel<float>, blocks, 256, 0, s, (const float*)X, count, status);
  else launch_k(check_finite_bf16_kernel, blocks, 256, 0, s, (const __nv_bfloat16*)X, count, status);
  return cudaGetLastError();
}
