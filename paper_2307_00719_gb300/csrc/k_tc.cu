// Dense slab MTTKRP on the 5th-generation tensor cores (tcgen05), FP32 results.
//
// The subchain of mode n is split at one contracted mode k (k = 1 when n = 1,
// else k = 1's neighbour 0; both 0-based here as k = 0 / k = 1):
//     G^{!=n}(j) = A(i_A) G_k(i_k) B(i_B),
// A = G_{n+1} ... G_{k-1},  B = G_{k+1} ... G_{n-1}  (cyclic, either may be empty).
// Then  X_[n] G^{!=n}_[2]  (Eq. partial)  is computed in two stages:
//   stage 1  Y = X x_k G_k : a GEMM  [M = E / I_k] x [K = I_k] x [N = R_k R_{k+1}]
//            on tcgen05.mma (kind::tf32) with A tiles fed by TMA, accumulator in
//            TMEM.  FP32 accuracy comes from a 3-term split: X = X_hi + X_lo and
//            G = G_hi + G_lo, both terms rounded to nearest TF32 before the MMA
//            (so the hardware's TF32 conversion is exact and unbiased), products
//            X_hi G_hi + X_hi G_lo + X_lo G_hi.  A BF16 slab is exact in TF32
//            (X_lo = 0), so it needs two products.
//   stage 2  P(i_n, a + R_n b) = sum_{i_A, i_B, c, d} A(b,c) Y(.., c + R_k d) B(d,a)
//            with A and B read from precomputed chain tables (SIMT, FP32).
#include <cuda.h>

#include <algorithm>

#include "kernels.cuh"
#include "ptx.cuh"
#include "tc.cuh"

namespace {


// ---------------------------------------------------------------------------
// stage 1: one CTA per 128-row tile of Y, K in chunks of 32
// ---------------------------------------------------------------------------
template <bool SRC_BF16>
__global__ void __launch_bounds__(128, 1) stage1_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                           const float* __restrict__ Bhi,
                                                           const float* __restrict__ Blo, int M,
                                                           int Kpad, int N, int Npad, uint32_t tmem_cols,
                                                           float* __restrict__ Y, int* status, int cps) {
  // cps > 0: split K -- CTA (x, y) takes the K chunks [y cps, (y + 1) cps) and
  // writes its partial product to Y + y M N
  PDL_ENTRY();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sAhi = smem;                              // 128 x 128 B
  unsigned char* sAlo = smem + 16384;                      // 128 x 128 B
  unsigned char* sBhi = smem + 32768;                      // Npad x 128 B
  unsigned char* sBlo = sBhi + (size_t)Npad * 128;         // Npad x 128 B
  unsigned char* sAraw = sBlo + (size_t)Npad * 128;        // 128 x 32 source elements
  uint64_t* bars = (uint64_t*)(sAraw + 16384);
  uint32_t* tslot = (uint32_t*)(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128;

  if (warp == 0) tmem_alloc(tslot, tmem_cols);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(Npad >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  const uint32_t box_bytes = SRC_BF16 ? 128 * 32 * 2 : 128 * 32 * 4;
  uint32_t ph_tma = 0, ph_mma = 0;
  bool failed = false;
  const int nchunks = Kpad / 32;
  const int cb = cps > 0 ? (int)blockIdx.y * cps : 0;
  const int ce = cps > 0 ? min(nchunks, cb + cps) : nchunks;
  if (cps > 0) Y += (size_t)blockIdx.y * (size_t)M * N;
  for (int c = cb; c < ce && !failed; ++c) {
    if (tid == 0) {
      mbar_expect_tx(&bars[0], box_bytes);
      tma_load_2d(sAraw, &tmA, &bars[0], c * 32, m0);
    }
    // B chunk: rows n < Npad, columns 32c .. 32c+31 of the pre-split operand
    for (int r = tid >> 3; r < Npad; r += 16) {
      const int j = tid & 7;
      const float4 h = *(const float4*)(Bhi + (size_t)r * Kpad + c * 32 + j * 4);
      const float4 l = *(const float4*)(Blo + (size_t)r * Kpad + c * 32 + j * 4);
      *(float4*)(sBhi + sw128_off(r, j)) = h;
      *(float4*)(sBlo + sw128_off(r, j)) = l;
    }
    const bool ok = mbar_wait(&bars[0], ph_tma, kWaitNs);
    ph_tma ^= 1;
    if (__syncthreads_or(!ok)) { failed = true; break; }
    // A chunk: split into hi / lo and write the swizzled operand tiles
    for (int p = 0; p < 8; ++p) {
      const int r = p * 16 + (tid >> 3);
      const int j = tid & 7;
      float4 v;
      if (SRC_BF16) {
        const __nv_bfloat162* q = (const __nv_bfloat162*)(sAraw + r * 64 + j * 8);
        const float2 a = __bfloat1622float2(q[0]), b = __bfloat1622float2(q[1]);
        v = make_float4(a.x, a.y, b.x, b.y);
      } else {
        v = *(const float4*)(sAraw + r * 128 + j * 16);
      }
      const float4 hi = make_float4(tf32_rn(v.x), tf32_rn(v.y), tf32_rn(v.z), tf32_rn(v.w));
      *(float4*)(sAhi + sw128_off(r, j)) = hi;
      if (!SRC_BF16) {
        const float4 lo = make_float4(tf32_rn(v.x - hi.x), tf32_rn(v.y - hi.y), tf32_rn(v.z - hi.z),
                                      tf32_rn(v.w - hi.w));
        *(float4*)(sAlo + sw128_off(r, j)) = lo;
      }
    }
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint64_t ah = desc_sw128(sAhi), al = desc_sw128(sAlo);
      const uint64_t bh = desc_sw128(sBhi), bl = desc_sw128(sBlo);
      // three accumulators: hi*hi products alternate between columns [0, Npad) and
      // [Npad, 2 Npad); the small cross terms go to [2 Npad, 3 Npad).  Shorter
      // accumulation chains keep the accumulator's rounding error down.
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint64_t adv = (uint64_t)(kk * 32) >> 4;   // 8 TF32 = 32 bytes along K
        const int step = (c - cb) * 4 + kk;
        const uint32_t dhi = tmem + (uint32_t)((step & 1) * Npad);
        const uint32_t dx = tmem + (uint32_t)(2 * Npad);
        mma_tf32(dhi, ah + adv, bh + adv, idesc, step >= 2 ? 1u : 0u);
        mma_tf32(dx, ah + adv, bl + adv, idesc, step >= 1 ? 1u : 0u);
        if (!SRC_BF16) mma_tf32(dx, al + adv, bh + adv, idesc, 1u);
      }
      mma_commit(&bars[1]);
    }
    const bool ok2 = mbar_wait(&bars[1], ph_mma, kWaitNs);
    ph_mma ^= 1;
    if (__syncthreads_or(!ok2)) { failed = true; break; }
  }
  tc_fence_after();
  if (!failed) {
    const int row = m0 + 32 * warp + lane;
    const bool two = (ce - cb) * 4 >= 2;   // the second hi*hi accumulator was written
    for (int col = 0; col < Npad; col += 8) {
      const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)col;
      uint32_t v0[8], v1[8], vx[8];
      tmem_ld_x8(base, v0);
      tmem_ld_x8(base + (uint32_t)Npad, v1);
      tmem_ld_x8(base + (uint32_t)(2 * Npad), vx);
      if (row < M) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float y = __uint_as_float(v0[j]) + __uint_as_float(vx[j]);
          if (two) y += __uint_as_float(v1[j]);
          if (col + j < N) Y[(size_t)row * N + col + j] = y;
        }
      }
    }
  } else if (tid == 0) {
    atomicOr(status, DEV_ERR_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

// ---------------------------------------------------------------------------
// stage 1, persistent form: one CTA per SM loops over 128-row tiles.
// * The split B operand (all K chunks) is copied once into shared memory with
//   cp.async, swizzled, overlapping the first tile's TMA load.
// * FP32 slab: TMA loads each A chunk with the 128-byte swizzle, so the raw tile
//   already is the K-major operand.  The tensor core reads an FP32 word as TF32
//   by dropping its 13 low mantissa bits, so the raw tile serves as X_hi =
//   trunc(X) and only X_lo = rn(X - trunc(X)) (exact residual, rounded to the
//   nearest TF32) is formed: X_hi + X_lo equals X to 2^-22 relative, unbiased.
// * BF16 slab: the raw tile is widened to FP32 into the operand tile (exact;
//   no X_lo term).
// * The next tile's A chunks are prefetched by TMA into the other buffer while
//   the current tile is split, multiplied and written out; the epilogue writes
//   whole 32-byte sectors (float4 pairs) of Y.
// ---------------------------------------------------------------------------
template <bool SRC_BF16>
__global__ void __launch_bounds__(128, 1) stage1_tc_persist_kernel(
    const __grid_constant__ CUtensorMap tmA, const float* __restrict__ Bhi, const float* __restrict__ Blo,
    int M, int Kpad, int N, int Npad, uint32_t tmem_cols, float* __restrict__ Y, int* status) {
  PDL_ENTRY();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int nch = Kpad / 32;
  const size_t bchunk = (size_t)Npad * 128;
  unsigned char* sBhi = smem;                                   // nch x (Npad x 128 B)
  unsigned char* sBlo = sBhi + nch * bchunk;
  unsigned char* sA = sBlo + nch * bchunk;
  // FP32: sA = 2 buffers x nch x 16 KB (TMA targets = X_hi), then sLo = nch x 16 KB
  // BF16: sA = nch x 16 KB (widened operand), then sRaw = 2 buffers x nch x 8 KB
  constexpr uint32_t kRawChunk = SRC_BF16 ? 8192u : 16384u;
  unsigned char* sLo = sA + (size_t)2 * nch * 16384;            // FP32 only
  unsigned char* sRaw = sA + (size_t)nch * 16384;               // BF16 only
  unsigned char* tma_base = SRC_BF16 ? sRaw : sA;               // buffer b, chunk c at + (b nch + c) kRawChunk
  unsigned char* after = SRC_BF16 ? sRaw + (size_t)2 * nch * kRawChunk : sLo + (size_t)nch * 16384;
  uint64_t* bars = (uint64_t*)after;                            // tma[0], tma[1], mma
  uint32_t* tslot = (uint32_t*)(bars + 3);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (M + 127) / 128;

  if (warp == 0) tmem_alloc(tslot, tmem_cols);
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  if (tid == 0 && (int)blockIdx.x < ntiles) {
    mbar_expect_tx(&bars[0], kRawChunk * nch);
    for (int c = 0; c < nch; ++c) tma_load_2d(tma_base + (size_t)c * kRawChunk, &tmA, &bars[0], c * 32, blockIdx.x * 128);
  }
  // the whole split B operand, swizzled, once per CTA (asynchronous copies)
  for (int c = 0; c < nch; ++c)
    for (int r = tid >> 3; r < Npad; r += 16) {
      const int j = tid & 7;
      cp_async16(sBhi + c * bchunk + sw128_off(r, j), Bhi + (size_t)r * Kpad + c * 32 + j * 4);
      cp_async16(sBlo + c * bchunk + sw128_off(r, j), Blo + (size_t)r * Kpad + c * 32 + j * 4);
    }
  cp_async_commit();
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(Npad >> 3) << 17) |
                         ((uint32_t)(128 >> 4) << 24);
  uint32_t ph_tma = 0, ph_mma = 0;   // ph_tma bit b: phase of buffer b
  bool failed = false;
  int it = 0;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int buf = it & 1;
    const int tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles) {   // prefetch the next tile into the other buffer
      mbar_expect_tx(&bars[buf ^ 1], kRawChunk * nch);
      for (int c = 0; c < nch; ++c)
        tma_load_2d(tma_base + ((size_t)(buf ^ 1) * nch + c) * kRawChunk, &tmA, &bars[buf ^ 1], c * 32, tn * 128);
    }
    const bool ok = mbar_wait(&bars[buf], (ph_tma >> buf) & 1u, kWaitNs);
    ph_tma ^= 1u << buf;
    if (__syncthreads_or(!ok)) { failed = true; break; }
    const unsigned char* araw = tma_base + (size_t)buf * nch * kRawChunk;
    if (!SRC_BF16) {
      // X_lo at the same (swizzled) position as X in the TMA tile
      for (int q = tid; q < nch * 1024; q += 128) {
        const float4 v = *(const float4*)(araw + (size_t)q * 16);
        const float4 h = make_float4(__uint_as_float(__float_as_uint(v.x) & 0xFFFFE000u),
                                     __uint_as_float(__float_as_uint(v.y) & 0xFFFFE000u),
                                     __uint_as_float(__float_as_uint(v.z) & 0xFFFFE000u),
                                     __uint_as_float(__float_as_uint(v.w) & 0xFFFFE000u));
        *(float4*)(sLo + (size_t)q * 16) =
            make_float4(tf32_rn(v.x - h.x), tf32_rn(v.y - h.y), tf32_rn(v.z - h.z), tf32_rn(v.w - h.w));
      }
    } else {
      for (int c = 0; c < nch; ++c) {
        const unsigned char* raw = araw + (size_t)c * kRawChunk;
        unsigned char* ah = sA + (size_t)c * 16384;
        for (int p = 0; p < 8; ++p) {
          const int r = p * 16 + (tid >> 3);
          const int j = tid & 7;
          const __nv_bfloat162* q = (const __nv_bfloat162*)(raw + r * 64 + j * 8);
          const float2 x0 = __bfloat1622float2(q[0]), x1 = __bfloat1622float2(q[1]);
          *(float4*)(ah + sw128_off(r, j)) = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
      }
    }
    if (it == 0) cp_async_wait_all();
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const unsigned char* ahi = SRC_BF16 ? sA : araw;
      for (int c = 0; c < nch; ++c) {
        const uint64_t ah = desc_sw128(ahi + (size_t)c * (SRC_BF16 ? 16384 : kRawChunk));
        const uint64_t al = desc_sw128(sLo + (size_t)c * 16384);
        const uint64_t bh = desc_sw128(sBhi + c * bchunk), bl = desc_sw128(sBlo + c * bchunk);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
          const uint64_t adv = (uint64_t)(kk * 32) >> 4;
          const int step = c * 4 + kk;
          const uint32_t dhi = tmem + (uint32_t)((step & 1) * Npad);
          const uint32_t dx = tmem + (uint32_t)(2 * Npad);
          mma_tf32(dhi, ah + adv, bh + adv, idesc, step >= 2 ? 1u : 0u);
          mma_tf32(dx, ah + adv, bl + adv, idesc, step >= 1 ? 1u : 0u);
          if (!SRC_BF16) mma_tf32(dx, al + adv, bh + adv, idesc, 1u);
        }
      }
      mma_commit(&bars[2]);
    }
    const bool ok2 = mbar_wait(&bars[2], ph_mma, kWaitNs);
    ph_mma ^= 1;
    if (__syncthreads_or(!ok2)) { failed = true; break; }
    tc_fence_after();
    const int row = t * 128 + 32 * warp + lane;
    const bool vec = (N & 3) == 0;
    for (int col = 0; col < Npad; col += 16) {
      const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)col;
      uint32_t v0[16], v1[16], vx[16];
      tmem_ld_x16_nw(base, v0);
      tmem_ld_x16_nw(base + (uint32_t)Npad, v1);
      tmem_ld_x16_nw(base + (uint32_t)(2 * Npad), vx);
      tmem_wait_ld();
      if (row < M) {
        float y[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          y[j] = (__uint_as_float(v0[j]) + __uint_as_float(vx[j])) + __uint_as_float(v1[j]);
        float* yrow = Y + (size_t)row * N + col;
        if (vec && col + 16 <= N) {
#pragma unroll
          for (int j = 0; j < 16; j += 4) *(float4*)(yrow + j) = make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (col + j < N) yrow[j] = y[j];
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
  if (it == 0) cp_async_wait_all();   // no tile: B copies still complete before exit
  if (failed && tid == 0) atomicOr(status, DEV_ERR_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, tmem_cols);
}

size_t stage1_persist_smem_bytes(int Npad, int nch, bool bf16) {
  const size_t b = (size_t)2 * nch * Npad * 128;
  const size_t a = bf16 ? (size_t)nch * 16384 + (size_t)2 * nch * 8192 : (size_t)3 * nch * 16384;
  return 1024 + b + a + 64;
}

// ---------------------------------------------------------------------------
// stage 1, warp-specialised persistent form (320 threads):
//   warp 0       TMA producer: X tiles into a ring of SA slots
//   warp 1       MMA issuer (one thread): 3-term TF32 products into one of two
//                TMEM accumulator sets, then commits that free the X slot and
//                the X_lo slot and publish the accumulator
//   warps 2-9    workers, two warpgroups: X_lo = rn(X - trunc(X)) (BF16: the
//                widened X) into one of two slots, shared by both groups, then
//                the epilogue of the previous tile (TMEM lanes 32 (warp % 4) ..
//                + 31; the groups take alternate 16-column chunks) while the
//                MMA of the next tile runs
// mbarriers: fullA/emptyA per X slot, fullLo/emptyLo per X_lo slot,
// accFull/accEmpty per accumulator set, bReady for the resident B operand.
// Every wait is bounded (2 s); a role whose wait times out stops and records
// DEV_ERR_TIMEOUT.
// ---------------------------------------------------------------------------
template <bool SRC_BF16, int SA>
__global__ void __launch_bounds__(320, 1) stage1_ws_kernel(
    const __grid_constant__ CUtensorMap tmA, const float* __restrict__ Bhi, const float* __restrict__ Blo,
    int M, int Kpad, int N, int Npad, uint32_t tmem_cols, float* __restrict__ Y, int* status) {
  PDL_ENTRY();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int nch = Kpad / 32;
  const size_t bchunk = (size_t)Npad * 128;
  constexpr uint32_t kRaw = SRC_BF16 ? 8192u : 16384u;   // one X chunk in the ring
  unsigned char* sBhi = smem;                            // nch x Npad x 128 B
  unsigned char* sBlo = sBhi + nch * bchunk;
  unsigned char* sA = sBlo + nch * bchunk;               // SA slots x nch x kRaw
  unsigned char* sLo = sA + (size_t)SA * nch * kRaw;     // 2 slots x nch x 16 KB
  uint64_t* bars = (uint64_t*)(sLo + (size_t)2 * nch * 16384);
  uint64_t* fullA = bars;
  uint64_t* emptyA = bars + SA;
  uint64_t* fullLo = bars + 2 * SA;
  uint64_t* emptyLo = fullLo + 2;
  uint64_t* accFull = emptyLo + 2;
  uint64_t* accEmpty = accFull + 2;
  uint64_t* bReady = accEmpty + 2;
  uint32_t* tslot = (uint32_t*)(bReady + 1);
  int* s_fail = (int*)(tslot + 1);
  float* sEpi = (float*)((unsigned char*)bars + 256);   // 8 warps x 32 rows x 17: epilogue staging
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntiles = (M + 127) / 128;
  const int my_tiles = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (warp == 1) tmem_alloc(tslot, tmem_cols);
  if (tid == 0) {
    for (int i = 0; i < SA; ++i) { mbar_init(&fullA[i], 1); mbar_init(&emptyA[i], 1); }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&fullLo[i], 8);
      mbar_init(&emptyLo[i], 1);
      mbar_init(&accFull[i], 1);
      mbar_init(&accEmpty[i], 8);
    }
    mbar_init(bReady, 256);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool failed = false;

  if (warp == 0) {
    // ---- TMA producer ----
    if (lane == 0) {
      for (int j = 0; j < my_tiles; ++j) {
        const int a = j % SA, ua = j / SA;
        if (!mbar_wait(&emptyA[a], (ua & 1) ^ 1, kWaitNs)) { failed = true; break; }
        const int t = blockIdx.x + j * gridDim.x;
        mbar_expect_tx(&fullA[a], kRaw * nch);
        for (int c = 0; c < nch; ++c)
          tma_load_2d(sA + ((size_t)a * nch + c) * kRaw, &tmA, &fullA[a], c * 32, t * 128);
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(Npad >> 3) << 17) |
                             ((uint32_t)(128 >> 4) << 24);
      if (!mbar_wait(bReady, 0, kWaitNs)) failed = true;
      for (int j = 0; j < my_tiles && !failed; ++j) {
        const int a = j % SA, l = j & 1, ul = j >> 1;
        if (!mbar_wait(&fullLo[l], ul & 1, kWaitNs)) { failed = true; break; }
        if (!mbar_wait(&accEmpty[l], (ul & 1) ^ 1, kWaitNs)) { failed = true; break; }
        tc_fence_after();
        const uint32_t base = tmem + (uint32_t)(l * 3 * Npad);
        for (int c = 0; c < nch; ++c) {
          const unsigned char* ahp = SRC_BF16 ? sLo + ((size_t)l * nch + c) * 16384 : sA + ((size_t)a * nch + c) * kRaw;
          const uint64_t ah = desc_sw128(ahp);
          const uint64_t al = desc_sw128(sLo + ((size_t)l * nch + c) * 16384);
          const uint64_t bh = desc_sw128(sBhi + c * bchunk), bl = desc_sw128(sBlo + c * bchunk);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;
            const int step = c * 4 + kk;
            const uint32_t dhi = base + (uint32_t)((step & 1) * Npad);
            const uint32_t dx = base + (uint32_t)(2 * Npad);
            mma_tf32(dhi, ah + adv, bh + adv, idesc, step >= 2 ? 1u : 0u);
            mma_tf32(dx, ah + adv, bl + adv, idesc, step >= 1 ? 1u : 0u);
            if (!SRC_BF16) mma_tf32(dx, al + adv, bh + adv, idesc, 1u);
          }
        }
        mma_commit(&accFull[l]);
        mma_commit(&emptyA[a]);
        mma_commit(&emptyLo[l]);
      }
      // the last products complete before TMEM is released
      if (!failed && my_tiles > 0) {
        const int jl = my_tiles - 1;
        if (!mbar_wait(&accFull[jl & 1], (jl >> 1) & 1, kWaitNs)) failed = true;
      }
    }
  } else {
    // ---- workers: B staging, X_lo, epilogue ----
    const int wt = tid - 64;                 // 0..255
    const int q = warp & 3;                  // TMEM lane quadrant of this warp
    const int wg = (warp - 2) >> 2;          // worker group: epilogue chunks wg, wg + 2, ..
    for (int c = 0; c < nch; ++c)
      for (int r = wt >> 3; r < Npad; r += 32) {
        const int jx = wt & 7;
        cp_async16(sBhi + c * bchunk + sw128_off(r, jx), Bhi + (size_t)r * Kpad + c * 32 + jx * 4);
        cp_async16(sBlo + c * bchunk + sw128_off(r, jx), Blo + (size_t)r * Kpad + c * 32 + jx * 4);
      }
    cp_async_wait_all();
    fence_proxy_async();
    mbar_arrive(bReady);
    const bool vec = (N & 3) == 0;
    for (int j = 0; j <= my_tiles && !failed; ++j) {
      if (j < my_tiles) {
        const int a = j % SA, ua = j / SA, l = j & 1, ul = j >> 1;
        if (!mbar_wait(&fullA[a], ua & 1, kWaitNs)) { failed = true; break; }
        if (!mbar_wait(&emptyLo[l], (ul & 1) ^ 1, kWaitNs)) { failed = true; break; }
        const unsigned char* araw = sA + (size_t)a * nch * kRaw;
        unsigned char* lo = sLo + (size_t)l * nch * 16384;
        if (!SRC_BF16) {
          for (int e = wt; e < nch * 1024; e += 256 * 4) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (e + 256 * u < nch * 1024) v[u] = *(const float4*)(araw + (size_t)(e + 256 * u) * 16);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              if (e + 256 * u >= nch * 1024) continue;
              const float4 x = v[u];
              const float4 h = make_float4(__uint_as_float(__float_as_uint(x.x) & 0xFFFFE000u),
                                           __uint_as_float(__float_as_uint(x.y) & 0xFFFFE000u),
                                           __uint_as_float(__float_as_uint(x.z) & 0xFFFFE000u),
                                           __uint_as_float(__float_as_uint(x.w) & 0xFFFFE000u));
              *(float4*)(lo + (size_t)(e + 256 * u) * 16) =
                  make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y), tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
            }
          }
        } else {
          for (int c = 0; c < nch; ++c) {
            const unsigned char* raw = araw + (size_t)c * kRaw;
            unsigned char* ah = lo + (size_t)c * 16384;
            for (int p = 0; p < 4; ++p) {
              const int r = p * 32 + (wt >> 3);
              const int jx = wt & 7;
              const __nv_bfloat162* qv = (const __nv_bfloat162*)(raw + r * 64 + jx * 8);
              const float2 x0 = __bfloat1622float2(qv[0]), x1 = __bfloat1622float2(qv[1]);
              *(float4*)(ah + sw128_off(r, jx)) = make_float4(x0.x, x0.y, x1.x, x1.y);
            }
          }
        }
        fence_proxy_async();
        __syncwarp();
        if (lane == 0) mbar_arrive(&fullLo[l]);
      }
      if (j >= 1) {
        const int jp = j - 1, r = jp & 1, ur = jp >> 1;
        if (!mbar_wait(&accFull[r], ur & 1, kWaitNs)) { failed = true; break; }
        tc_fence_after();
        const int t = blockIdx.x + jp * gridDim.x;
        const int row0 = t * 128 + 32 * q;        // first row of this warp's 32
        const uint32_t abase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(r * 3 * Npad);
        float* se = sEpi + (warp - 2) * (32 * 17);
        for (int col = 16 * wg; col < Npad; col += 32) {
          uint32_t v0[16], v1[16], vx[16];
          tmem_ld_x16_nw(abase + (uint32_t)col, v0);
          tmem_ld_x16_nw(abase + (uint32_t)(Npad + col), v1);
          tmem_ld_x16_nw(abase + (uint32_t)(2 * Npad + col), vx);
          tmem_wait_ld();
          float y[16];
#pragma unroll
          for (int u = 0; u < 16; ++u)
            y[u] = (__uint_as_float(v0[u]) + __uint_as_float(vx[u])) + __uint_as_float(v1[u]);
          if (vec) {
            // rows of 16-byte multiples: the lane's row, four floats per store
            const int row = row0 + lane;
            if (row < M) {
              float* yrow = Y + (size_t)row * N + col;
              if (col + 16 <= N) {
#pragma unroll
                for (int u = 0; u < 16; u += 4) *(float4*)(yrow + u) = make_float4(y[u], y[u + 1], y[u + 2], y[u + 3]);
              } else {
#pragma unroll
                for (int u = 0; u < 16; ++u)
                  if (col + u < N) yrow[u] = y[u];
              }
            }
          } else {
            // other widths: through shared memory, so that each store writes two
            // rows' 16 consecutive columns
#pragma unroll
            for (int u = 0; u < 16; ++u) se[lane * 17 + u] = y[u];
            __syncwarp();
            const int cc = lane & 15;
#pragma unroll 4
            for (int i = 0; i < 16; ++i) {
              const int rr = 2 * i + (lane >> 4);
              if (row0 + rr < M && col + cc < N) Y[(size_t)(row0 + rr) * N + col + cc] = se[rr * 17 + cc];
            }
            __syncwarp();
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accEmpty[r]);
      }
    }
  }
  if (failed) *s_fail = 1;
  tc_fence_before();
  __syncthreads();
  if (tid == 0 && *s_fail) atomicOr(status, DEV_ERR_TIMEOUT);
  if (warp == 1) tmem_dealloc(tmem, tmem_cols);
}

size_t stage1_ws_smem_bytes(int Npad, int nch, bool bf16, int sa) {
  const size_t b = (size_t)2 * nch * Npad * 128;
  const size_t raw = (size_t)sa * nch * (bf16 ? 8192 : 16384);
  return 1024 + b + raw + (size_t)2 * nch * 16384 + 256 + 8 * 32 * 17 * 4;
}

// ---------------------------------------------------------------------------
// operand prep: B^T split, [Npad][Kpad], zero padded
// ---------------------------------------------------------------------------
__global__ void prep_b_kernel(const double* __restrict__ G, int K, int N, int Kpad, int Npad,
                              float* __restrict__ Bhi, float* __restrict__ Blo) {
  PDL_ENTRY();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)Kpad * Npad;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(e / Kpad), k = (int)(e % Kpad);
    float h = 0.f, l = 0.f;
    if (n < N && k < K) {
      const double g = G[(int64_t)k * N + n];
      h = tf32_rn((float)g);
      l = tf32_rn((float)(g - (double)h));
    }
    Bhi[e] = h;
    Blo[e] = l;
  }
}

// ---------------------------------------------------------------------------
// swap the two fastest modes of a slab: out[i1 + d1 (i0 + d0 r)] = in[i0 + d0 (i1 + d1 r)]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void transpose01_kernel(const T* __restrict__ in, T* __restrict__ out, int d0, int d1, int64_t rest) {
  PDL_ENTRY();
  __shared__ T tile[2][32][33];
  const int i0b = blockIdx.x * 32, i1b = blockIdx.y * 32;
  // several slices r per CTA (double-buffered tile: one barrier per slice)
  int b = 0;
  for (int64_t r = blockIdx.z; r < rest; r += gridDim.z, b ^= 1) {
    const T* src = in + r * (int64_t)d0 * d1;
    T* dst = out + r * (int64_t)d0 * d1;
    T v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i1 = i1b + threadIdx.y + 8 * u, i0 = i0b + threadIdx.x;
      v[u] = (i0 < d0 && i1 < d1) ? src[(int64_t)i1 * d0 + i0] : (T)0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) tile[b][threadIdx.y + 8 * u][threadIdx.x] = v[u];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i0 = i0b + threadIdx.y + 8 * u, i1 = i1b + threadIdx.x;
      if (i0 < d0 && i1 < d1) dst[(int64_t)i0 * d1 + i1] = tile[b][threadIdx.x][threadIdx.y + 8 * u];
    }
  }
}

// ---------------------------------------------------------------------------
// stage 2 (SIMT).  Per combination q = i_lo + Jlo i_hi the work is one small
// product:
//   B present:          Z = Y_q (R_k x R_{k+1}) . B (R_{k+1} x R_n)      [form YB]
//   A present, B empty: Z = A(i_hi) (R_{n+1} x R_k) . Y_q (R_k x R_n)    [form AY]
//   neither:            Z = Y_q                                           [form Y]
// When A and B are both present (k = 0, Jlo > 1) A depends on i_hi only, so the
// YB products are summed over each run of equal i_hi first and multiplied by
// A(i_hi) once per run.
// CTA per (i_n, split); the split's combinations are staged in chunks of CH
// (Y rows + the per-combination table), double-buffered with cp.async; thread
// (g, o) owns output o of the product and every G-th combination of a chunk.
// Groups are combined in a fixed order (deterministic).
// ---------------------------------------------------------------------------
constexpr int S2_CH = 32;       // combinations per chunk
constexpr int S2_STAGES = 4;    // chunks in the shared-memory ring (S2_STAGES - 1 in flight)
constexpr int S2_THREADS = 256;

__device__ __forceinline__ void s2_issue(const Stage2Args& a, int form, int64_t in, int64_t qa, int nq,
                                         int ystr, int tstr, int tsz, float* sY, float* sT, bool vec) {
  // 8 threads per combination
  const int t = threadIdx.x, j = t >> 3, sub = t & 7;
  if (j >= nq) return;
  const uint32_t q = (uint32_t)(qa + j);
  const uint32_t Jlo = (uint32_t)a.Jlo;
  const uint32_t ilo = q % Jlo, ihi = q / Jlo;
  const int64_t m = (int64_t)ilo + a.Jlo * (in + a.dn * (int64_t)ihi);
  const int RRk = a.Rk * a.Rk1;
  const float* ysrc = a.Y + m * RRk;
  float* ydst = sY + j * ystr;
  const float* tsrc = nullptr;
  if (form == 0) tsrc = a.TB + (int64_t)(a.k == 0 ? ilo : ihi) * tsz;
  else if (form == 1) tsrc = a.TA + (int64_t)ihi * tsz;
  float* tdst = sT + j * tstr;
  if (vec) {
    for (int x = sub * 4; x < RRk; x += 32) cp_async16(ydst + x, ysrc + x);
    if (tsrc)
      for (int x = sub * 4; x < tsz; x += 32) cp_async16(tdst + x, tsrc + x);
  } else {
    for (int x = sub; x < RRk; x += 8) cp_async4(ydst + x, ysrc + x);
    if (tsrc)
      for (int x = sub; x < tsz; x += 8) cp_async4(tdst + x, tsrc + x);
  }
}

// sum_e L[R e] M[e] for a compile-time R (multiple of 4); M is 16-byte aligned
template <int R>
__device__ __forceinline__ float s2_dot(const float* L, const float* M) {
  float v = 0.f;
#pragma unroll
  for (int e = 0; e < R; e += 4) {
    const float4 m = *(const float4*)(M + e);
    v = fmaf(L[R * e], m.x, v);
    v = fmaf(L[R * (e + 1)], m.y, v);
    v = fmaf(L[R * (e + 2)], m.z, v);
    v = fmaf(L[R * (e + 3)], m.w, v);
  }
  return v;
}

// 2 x 2 register block of a product with compile-time R (multiple of 4):
// acc[a + 2b] += sum_e L[(x0 + a) + R e] M[e + R (y0 + b)];  L at x0 (even), M at R y0
template <int R>
__device__ __forceinline__ void s2_dot22(const float* L, const float* M, float (&acc)[4]) {
  float v00 = 0.f, v10 = 0.f, v01 = 0.f, v11 = 0.f;
#pragma unroll
  for (int e = 0; e < R; e += 4) {
    const float4 m0 = *(const float4*)(M + e);
    const float4 m1 = *(const float4*)(M + R + e);
    const float mm0[4] = {m0.x, m0.y, m0.z, m0.w}, mm1[4] = {m1.x, m1.y, m1.z, m1.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float2 l = *(const float2*)(L + R * (e + u));
      v00 = fmaf(l.x, mm0[u], v00);
      v10 = fmaf(l.y, mm0[u], v10);
      v01 = fmaf(l.x, mm1[u], v01);
      v11 = fmaf(l.y, mm1[u], v11);
    }
  }
  acc[0] += v00; acc[1] += v10; acc[2] += v01; acc[3] += v11;
}

// RT > 0: all four ranks equal RT (compile-time strides); RT = 0: any ranks
template <int RT>
__global__ void __launch_bounds__(S2_THREADS, 3) stage2_kernel(Stage2Args a) {
  PDL_ENTRY();
  extern __shared__ __align__(16) float s2[];
  const int Rk = a.Rk, Rk1 = a.Rk1, Rn = a.Rn, Rn1 = a.Rn1;
  const int RRk = Rk * Rk1;
  const int OUTP = Rn * Rn1;
  // form and product shape: out index of product entry (x, y) = y + Rn x
  const int form = a.TB ? 0 : (a.TA ? 1 : 2);
  const bool segA = a.TA && a.TB;          // YB runs multiplied by A(i_hi)
  int X, Yd, inner, tsz;
  if (form == 0) { X = Rk; Yd = Rn; inner = Rk1; tsz = Rk1 * Rn; }
  else if (form == 1) { X = Rn1; Yd = Rn; inner = Rk; tsz = Rn1 * Rk; }
  else { X = Rk; Yd = Rn; inner = 1; tsz = 0; }
  const int PO = X * Yd;                   // outputs of one product
  const int G = max(1, S2_THREADS / PO);   // combination groups
  const int ystr = (RRk + 3) & ~3, tstr = (tsz + 3) & ~3;
  // ring slot b: Y rows at s2 + b S2_CH ystr, tables at s2 + S2_STAGES S2_CH ystr + b S2_CH tstr
  float* const sY0 = s2;
  float* const sT0 = s2 + S2_STAGES * S2_CH * ystr;
  float* sRed = s2 + S2_STAGES * S2_CH * (ystr + tstr);   // G x PO, then PO (segment sums)
  const bool vec = (RRk % 4 == 0) && (tsz % 4 == 0) && ((((uintptr_t)a.Y) & 15) == 0) &&
                   (form == 2 || ((((uintptr_t)(form == 0 ? a.TB : a.TA)) & 15) == 0));
  const int tid = threadIdx.x;
  // RT = 0: one product entry o = (x, y) per thread, G groups of PO threads.
  // RT > 0: a 2 x 2 block of entries per thread (x0..x0+1, y0..y0+1), RT^2/4
  // threads per combination, GR groups.
  constexpr int TPC = RT > 0 ? RT * RT / 4 : 1;
  const int GG = RT > 0 ? S2_THREADS / TPC : G;
  const int g = RT > 0 ? tid / TPC : tid / PO;
  const int o = RT > 0 ? 0 : tid - g * PO;
  const bool act = g < GG;
  const int tt = RT > 0 ? tid - g * TPC : 0;
  const int x = RT > 0 ? 2 * (tt % (RT / 2)) : (act ? o % X : 0);
  const int y = RT > 0 ? 2 * (tt / (RT / 2)) : (act ? o / X : 0);
  constexpr int NV = RT > 0 ? 4 : 1;
  // product entries held: (x + (v & 1), y + (v >> 1)) for RT > 0, else (x, y)
  auto oidx = [&](int v) { return RT > 0 ? (x + (v & 1)) + X * (y + (v >> 1)) : o; };
  const int64_t in = blockIdx.x;
  const int64_t ncomb = a.Jlo * a.Jhi;
  const int64_t q0 = (int64_t)blockIdx.y * a.per, q1 = min(ncomb, q0 + a.per);
  float acc4[NV];       // product sums (per group)
#pragma unroll
  for (int v = 0; v < NV; ++v) acc4[v] = 0.f;
  float outv = 0.f;     // A-multiplied segment sums (threads tid < OUTP)
  // chunk boundaries: never cross an i_hi run when segA
  auto chunk_end = [&](int64_t qa) {
    int64_t e = min(q1, qa + S2_CH);
    if (segA) e = min(e, (qa / a.Jlo + 1) * a.Jlo);
    return e;
  };
  // prologue: the first S2_STAGES - 1 chunks in flight
  int64_t iq = q0;
#pragma unroll
  for (int st = 0; st < S2_STAGES - 1; ++st) {
    if (iq < q1) {
      const int64_t ie = chunk_end(iq);
      s2_issue(a, form, in, iq, (int)(ie - iq), ystr, tstr, tsz, sY0 + st * S2_CH * ystr, sT0 + st * S2_CH * tstr, vec);
      iq = ie;
    }
    cp_async_commit();
  }
  int64_t qa = q0;
  int ci = 0;
  while (qa < q1) {
    const int64_t qe = chunk_end(qa);
    const int nq = (int)(qe - qa);
    const int buf = ci % S2_STAGES;
    {  // chunk ci + S2_STAGES - 1 into the slot of chunk ci - 1 (consumed, barrier passed)
      const int sl = (ci + S2_STAGES - 1) % S2_STAGES;
      if (iq < q1) {
        const int64_t ie = chunk_end(iq);
        s2_issue(a, form, in, iq, (int)(ie - iq), ystr, tstr, tsz, sY0 + sl * S2_CH * ystr, sT0 + sl * S2_CH * tstr,
                 vec);
        iq = ie;
      }
      cp_async_commit();
    }
    cp_async_wait_n<S2_STAGES - 1>();   // chunk ci has landed
    __syncthreads();
    if (act) {
      const float* Yb = sY0 + buf * S2_CH * ystr;
      const float* Tb = sT0 + buf * S2_CH * tstr;
      if (form == 2) {
        for (int j = g; j < nq; j += GG) {
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const int xx = RT > 0 ? x + (v & 1) : x, yy = RT > 0 ? y + (v >> 1) : y;
            acc4[v] += Yb[j * ystr + xx + Rk * yy];
          }
        }
      } else {
        // product entry (x, y) = sum_e L[x + X e] M[e + inner y]:
        // form YB: L = Y_q, M = B;  form AY: L = A, M = Y_q
        const int lstr = form == 0 ? ystr : tstr, mstr = form == 0 ? tstr : ystr;
        const float* Lb = (form == 0 ? Yb : Tb) + x;
        const float* Mb = (form == 0 ? Tb : Yb) + inner * y;
        if constexpr (RT > 0) {
          for (int j = g; j < nq; j += GG) s2_dot22<RT>(Lb + j * lstr, Mb + j * mstr, acc4);
        } else {
          for (int j = g; j < nq; j += GG) {
            const float* lq = Lb + j * lstr;
            const float* mq = Mb + j * mstr;
            float v = 0.f;
            for (int e = 0; e < inner; ++e) v = fmaf(lq[X * e], mq[e], v);
            acc4[0] += v;
          }
        }
      }
    }
    __syncthreads();   // slot `buf` is refilled by the next iteration's issue
    ++ci;
    qa = qe;
    const bool seg_end = segA && (qa >= q1 || (qa % a.Jlo) == 0);
    if (seg_end) {
      // S = sum over groups (fixed order), then out += A(i_hi) S
      if (act) {
#pragma unroll
        for (int v = 0; v < NV; ++v) { sRed[g * PO + oidx(v)] = acc4[v]; acc4[v] = 0.f; }
      }
      __syncthreads();
      float* sS = sRed + GG * PO;
      for (int e = tid; e < PO; e += S2_THREADS) {
        float v = 0.f;
        for (int gg = 0; gg < GG; ++gg) v += sRed[gg * PO + e];
        sS[e] = v;
      }
      __syncthreads();
      const int64_t ihi = (qa - 1) / a.Jlo;
      const float* A = a.TA + ihi * (int64_t)(Rn1 * Rk);
      for (int e = tid; e < OUTP; e += S2_THREADS) {
        const int ob = e / Rn, oa = e - ob * Rn;
        float v = 0.f;
        for (int c = 0; c < Rk; ++c) v = fmaf(A[ob + Rn1 * c], sS[c + Rk * oa], v);
        outv += v;
      }
      __syncthreads();
    }
  }
  cp_async_wait_0();
  float* dst = a.partial + ((int64_t)blockIdx.y * a.dn + in) * OUTP;
  if (segA) {
    for (int e = tid; e < OUTP; e += S2_THREADS) dst[e] = outv;   // tid < OUTP <= 256: one each
    return;
  }
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sRed[g * PO + oidx(v)] = acc4[v];
  }
  __syncthreads();
  for (int e = tid; e < PO; e += S2_THREADS) {
    float v = 0.f;
    for (int gg = 0; gg < GG; ++gg) v += sRed[gg * PO + e];
    const int xx = e % X, yy = e / X;
    dst[yy + Rn * xx] = v;
  }
}

// ---------------------------------------------------------------------------
// stage 2 for small equal ranks R (R^2 <= 49), warp-synchronous: each warp takes
// batches of 32 consecutive combinations, copies their Y rows (and B rows when
// B follows i_lo) into its own shared-memory slice with coalesced loads, then
// lane j forms combination j's whole R x R product in registers
//   O = [A(i_hi)] . Y_q . [B]        (each factor present as in stage2_kernel)
// and accumulates it.  No block-wide barrier until the final fixed-order sum.
// ---------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(128) stage2_warp_kernel(Stage2Args a) {
  PDL_ENTRY();
  constexpr int PO = R * R;
  constexpr int PS = PO | 1;                  // odd per-combination stride: lane reads are conflict-free
  constexpr int NW = 4;
  extern __shared__ __align__(16) float s2w[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sY = s2w + warp * (2 * 32 * PS);
  float* sB = sY + 32 * PS;
  __shared__ float red[NW][PO];
  const bool hasA = a.TA != nullptr, hasB = a.TB != nullptr;
  const bool b_lo = hasB && a.k == 0;         // B follows i_lo (else i_hi)
  const int64_t in = blockIdx.x;
  const int64_t ncomb = a.Jlo * a.Jhi;
  const int64_t q0 = (int64_t)blockIdx.y * a.per, q1 = min(ncomb, q0 + a.per);
  float acc[PO], sacc[PO];
#pragma unroll
  for (int u = 0; u < PO; ++u) acc[u] = sacc[u] = 0.f;
  int64_t cur_hi = -1;
  // acc[w + R x] += sum_c A(h)[x + R c] sacc[c + R w]; sacc = 0
  auto flush = [&](int64_t h) {
    const float* aq = a.TA + h * PO;
    float am[PO];
#pragma unroll
    for (int u = 0; u < PO; ++u) am[u] = __ldg(aq + u);
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int w = 0; w < R; ++w) {
        float v = 0.f;
#pragma unroll
        for (int c = 0; c < R; ++c) v = fmaf(am[x + R * c], sacc[c + R * w], v);
        acc[w + R * x] += v;
      }
#pragma unroll
    for (int u = 0; u < PO; ++u) sacc[u] = 0.f;
  };
  for (int64_t qb = q0 + 32 * warp; qb < q1; qb += 32 * NW) {
    const int nq = (int)min((int64_t)32, q1 - qb);
    const int64_t hi0 = qb / a.Jlo, lo0 = qb - hi0 * a.Jlo;
    const bool one_seg = lo0 + nq <= a.Jlo;   // warp-uniform: rows of the batch are consecutive
    const int64_t q = qb + lane;
    const int64_t ihi = q / a.Jlo, ilo = q - ihi * a.Jlo;
    __syncwarp();
    if (one_seg && nq == 32) {
      // all loads of the batch issued before the first store
      const float* ys = a.Y + (lo0 + a.Jlo * (in + a.dn * hi0)) * PO;
      float v[PO];
#pragma unroll
      for (int i = 0; i < PO; ++i) v[i] = __ldg(ys + lane + 32 * i);
      if (b_lo) {
        const float* bs = a.TB + lo0 * PO;
        float w[PO];
#pragma unroll
        for (int i = 0; i < PO; ++i) w[i] = __ldg(bs + lane + 32 * i);
#pragma unroll
        for (int i = 0; i < PO; ++i) {
          const int f = lane + 32 * i;
          sB[PS == PO ? f : f + f / PO] = w[i];
        }
      }
#pragma unroll
      for (int i = 0; i < PO; ++i) {
        const int f = lane + 32 * i;
        sY[PS == PO ? f : f + f / PO] = v[i];     // j PS + u with f = j PO + u
      }
    } else if (one_seg) {
      const float* ys = a.Y + (lo0 + a.Jlo * (in + a.dn * hi0)) * PO;
      for (int f = lane; f < nq * PO; f += 32) {
        const int j = f / PO, u = f - j * PO;
        sY[j * PS + u] = __ldg(ys + f);
      }
      if (b_lo) {
        const float* bs = a.TB + lo0 * PO;
        for (int f = lane; f < nq * PO; f += 32) {
          const int j = f / PO, u = f - j * PO;
          sB[j * PS + u] = __ldg(bs + f);
        }
      }
    } else if (lane < nq) {
      const float* ys = a.Y + (ilo + a.Jlo * (in + a.dn * ihi)) * PO;
#pragma unroll
      for (int u = 0; u < PO; ++u) sY[lane * PS + u] = __ldg(ys + u);
      if (b_lo) {
#pragma unroll
        for (int u = 0; u < PO; ++u) sB[lane * PS + u] = __ldg(a.TB + ilo * PO + u);
      }
    }
    __syncwarp();
    if (lane < nq) {
      float y[PO];
#pragma unroll
      for (int u = 0; u < PO; ++u) y[u] = sY[lane * PS + u];
      float s[PO];                            // S = Y_q . B   (entry (c, w) at c + R w)
      if (hasB) {
        const float* bq = b_lo ? sB + lane * PS : a.TB + ihi * PO;
#pragma unroll
        for (int w = 0; w < R; ++w) {
          float bc[R];
#pragma unroll
          for (int e = 0; e < R; ++e) bc[e] = b_lo ? bq[e + R * w] : __ldg(bq + e + R * w);
#pragma unroll
          for (int c = 0; c < R; ++c) {
            float v = 0.f;
#pragma unroll
            for (int e = 0; e < R; ++e) v = fmaf(y[c + R * e], bc[e], v);
            s[c + R * w] = v;
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < PO; ++u) s[u] = y[u];
      }
      if (hasA) {
        // A(i_hi) is applied once per run of equal i_hi seen by this lane:
        // S is summed over the run, then O = A(i_hi) S_run joins the sums
        if (ihi != cur_hi) {
          if (cur_hi >= 0) flush(cur_hi);
          cur_hi = ihi;
        }
#pragma unroll
        for (int u = 0; u < PO; ++u) sacc[u] += s[u];
      } else {
#pragma unroll
        for (int x = 0; x < R; ++x)
#pragma unroll
          for (int w = 0; w < R; ++w) acc[w + R * x] += s[x + R * w];
      }
    }
  }
  if (hasA && cur_hi >= 0) flush(cur_hi);
  // fixed-order sums: butterfly within the warp, then warps in order
#pragma unroll
  for (int u = 0; u < PO; ++u) {
    float v = acc[u];
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][u] = v;
  }
  __syncthreads();
  float* dst = a.partial + ((int64_t)blockIdx.y * a.dn + in) * PO;
  for (int e = threadIdx.x; e < PO; e += blockDim.x) {
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) v += red[w][e];
    dst[e] = v;
  }
}

static int stage2_warp_rank(const Stage2Args& a) {
  const bool eq = a.Rk == a.Rk1 && a.Rk == a.Rn && a.Rk == a.Rn1;
  return eq && a.Rk >= 2 && a.Rk <= 7 && a.Rk != 4 ? a.Rk : 0;
}

size_t stage2_smem_bytes(const Stage2Args& a) {
  const int RRk = a.Rk * a.Rk1;
  int tsz = 0, PO = 0;
  if (a.TB) { tsz = a.Rk1 * a.Rn; PO = a.Rk * a.Rn; }
  else if (a.TA) { tsz = a.Rn1 * a.Rk; PO = a.Rn1 * a.Rn; }
  else { PO = a.Rk * a.Rn; }
  // groups: S2_THREADS / PO (one entry per thread) or S2_THREADS / (PO / 4) (2 x 2 blocks)
  const int G = std::max(1, S2_THREADS / std::max(1, PO / 4));
  const int ystr = (RRk + 3) & ~3, tstr = (tsz + 3) & ~3;
  return sizeof(float) * ((size_t)S2_STAGES * S2_CH * (ystr + tstr) + (size_t)G * PO + PO);
}

// ---------------------------------------------------------------------------
// Sampled MTTKRP on the tensor cores (rSTR, Alg. 5 with the sampled subchain of
// Alg. 3):  P_n += X_S[n] diag(w) G^{!=n}_S[2].
//   sampled_rows_kernel: row s of G_S -- the chain G_{n+1}(i_{n+1}) ...
//     G_{n-1}(i_{n-1}) of the sampled slices (column a + R_n b) -- and its
//     weight w_s; also the GEMM operand B = diag(w) G_S, transposed and split
//     into TF32 hi / lo terms.
//   gather_fibres_kernel: A = X_S[n], row i_n, column s = the mode-n fibre of
//     the slab at the sampled indices (K = samples contiguous, TMA-loadable).
// The product then runs as a split-K tcgen05 GEMM (launch_gemm_tc_splitk).
// ---------------------------------------------------------------------------
__global__ void sampled_rows_kernel(MttkrpArgs a, int Kpad, float* __restrict__ Bhi, float* __restrict__ Blo) {
  PDL_ENTRY();
  const int N = a.N, n = a.n;
  const int Ra = a.R[n], Rb = a.R[n + 1];
  const int RR = Ra * Rb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.m * Rb; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = e / Rb;
    const int r = (int)(e - f * Rb);
    double w = a.wscale;
    float v[STR_MAXR], t[STR_MAXR];
    int cols = 0;
    for (int q = 0; q < N - 1; ++q) {
      const int k = (n + 1 + q) % N;
      const int i = a.idxs[(int64_t)k * a.m + f];
      if (a.leverage) w /= a.p[k][i];
      const int Rk = a.R[k], Rk1 = a.R[k + 1];
      const float* g = (const float*)a.core[k] + (int64_t)i * Rk * Rk1;
      if (q == 0) {
#pragma unroll
        for (int c = 0; c < STR_MAXR; ++c) v[c] = c < Rk1 ? g[r + Rk * c] : 0.f;
      } else {
#pragma unroll
        for (int c = 0; c < STR_MAXR; ++c) {
          float sum = 0.f;
          if (c < Rk1)
            for (int x = 0; x < cols; ++x) sum = fmaf(v[x], g[x + Rk * c], sum);
          t[c] = sum;
        }
#pragma unroll
        for (int c = 0; c < STR_MAXR; ++c) v[c] = t[c];
      }
      cols = Rk1;
    }
    // v[c], c < R_n: entry (b = r, a = c) of S_f -> column c + Ra r
    float* gs = (float*)a.gs_out;
    for (int c = 0; c < Ra; ++c) {
      const int col = c + Ra * r;
      if (gs) gs[f * RR + col] = v[c];
      const double val = w * (double)v[c];
      const float hi = tf32_rn((float)val);
      Bhi[(int64_t)col * Kpad + f] = hi;
      Blo[(int64_t)col * Kpad + f] = tf32_rn((float)(val - (double)hi));
    }
    if (r == 0 && a.ws_out) a.ws_out[f] = w;
  }
}

// A[row][s] = X(mode-n fibre at the sampled indices of s, position row); 0 for s >= m
template <typename XT>
__global__ void gather_fibres_kernel(MttkrpArgs a, int Kpad, XT* __restrict__ A) {
  PDL_ENTRY();
  __shared__ int64_t sbase[32];
  const int N = a.N, n = a.n;
  const int64_t In = a.dim[n];
  int64_t stride[STR_MAXN];
  int64_t st = 1;
  for (int k = 0; k < N; ++k) { stride[k] = st; st *= a.dim[k]; }
  const int f = blockIdx.x * 32 + threadIdx.x;
  if (threadIdx.y == 0) {
    int64_t off = -1;
    if (f < a.m) {
      off = 0;
      for (int k = 0; k < N; ++k)
        if (k != n) off += (int64_t)a.idxs[(int64_t)k * a.m + f] * stride[k];
    }
    sbase[threadIdx.x] = off;
  }
  __syncthreads();
  const int64_t off = sbase[threadIdx.x];
  const XT* X = (const XT*)a.X;
  for (int64_t row = blockIdx.y * (int64_t)blockDim.y + threadIdx.y; row < In; row += (int64_t)gridDim.y * blockDim.y) {
    XT v = (XT)0.f;
    if (off >= 0) v = X[off + row * stride[n]];
    if (f < Kpad) A[row * Kpad + f] = v;
  }
}

// Complex samples (KSRFT, mixed slab and cores in complex FP32): P = X_S diag(w)
// conj(G_S) as two real GEMMs over K' = 2 Kpad with A = [Re X_S | Im X_S]:
//   Re P = A [w Re G_S ; w Im G_S],   Im P = A [-w Im G_S ; w Re G_S].
// sampled_rows_cplx_kernel writes G_S (complex, for the Gram), w and both B
// operands (transposed [Npad][2 Kpad], split TF32 hi / lo).
__global__ void sampled_rows_cplx_kernel(MttkrpArgs a, int Kpad, float* __restrict__ Brh, float* __restrict__ Brl,
                                         float* __restrict__ Bih, float* __restrict__ Bil) {
  PDL_ENTRY();
  const int N = a.N, n = a.n;
  const int Ra = a.R[n], Rb = a.R[n + 1];
  const int RR = Ra * Rb;
  const int64_t K2 = 2 * (int64_t)Kpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.m * Rb; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = e / Rb;
    const int r = (int)(e - f * Rb);
    const double w = a.wscale;
    float vr[STR_MAXR], vi[STR_MAXR], tr[STR_MAXR], ti[STR_MAXR];
    int cols = 0;
    for (int q = 0; q < N - 1; ++q) {
      const int k = (n + 1 + q) % N;
      const int i = a.idxs[(int64_t)k * a.m + f];
      const int Rk = a.R[k], Rk1 = a.R[k + 1];
      const float* g = (const float*)a.core[k] + 2 * (int64_t)i * Rk * Rk1;   // interleaved (re, im)
      if (q == 0) {
#pragma unroll
        for (int c = 0; c < STR_MAXR; ++c) {
          vr[c] = c < Rk1 ? g[2 * (r + Rk * c)] : 0.f;
          vi[c] = c < Rk1 ? g[2 * (r + Rk * c) + 1] : 0.f;
        }
      } else {
#pragma unroll
        for (int c = 0; c < STR_MAXR; ++c) {
          float sr = 0.f, si = 0.f;
          if (c < Rk1)
            for (int x = 0; x < cols; ++x) {
              const float gr = g[2 * (x + Rk * c)], gi = g[2 * (x + Rk * c) + 1];
              sr = fmaf(vr[x], gr, fmaf(-vi[x], gi, sr));
              si = fmaf(vr[x], gi, fmaf(vi[x], gr, si));
            }
          tr[c] = sr;
          ti[c] = si;
        }
#pragma unroll
        for (int c = 0; c < STR_MAXR; ++c) { vr[c] = tr[c]; vi[c] = ti[c]; }
      }
      cols = Rk1;
    }
    float* gs = (float*)a.gs_out;
    for (int c = 0; c < Ra; ++c) {
      const int col = c + Ra * r;
      if (gs) { gs[2 * (f * RR + col)] = vr[c]; gs[2 * (f * RR + col) + 1] = vi[c]; }
      const double re = w * (double)vr[c], im = w * (double)vi[c];
      const float reh = tf32_rn((float)re), reL = tf32_rn((float)(re - (double)reh));
      const float imh = tf32_rn((float)im), imL = tf32_rn((float)(im - (double)imh));
      const int64_t o = (int64_t)col * K2;
      Brh[o + f] = reh;          Brl[o + f] = reL;
      Brh[o + Kpad + f] = imh;   Brl[o + Kpad + f] = imL;
      Bih[o + f] = -imh;         Bil[o + f] = -imL;
      Bih[o + Kpad + f] = reh;   Bil[o + Kpad + f] = reL;
    }
    if (r == 0 && a.ws_out) a.ws_out[f] = w;
  }
}

// A[row][s] = Re, A[row][Kpad + s] = Im of the complex mode-n fibre at the
// sampled indices of s; 0 for s >= m
__global__ void gather_fibres_cplx_kernel(MttkrpArgs a, int Kpad, float* __restrict__ A) {
  PDL_ENTRY();
  __shared__ int64_t sbase[32];
  const int N = a.N, n = a.n;
  const int64_t In = a.dim[n];
  int64_t stride[STR_MAXN];
  int64_t st = 1;
  for (int k = 0; k < N; ++k) { stride[k] = st; st *= a.dim[k]; }
  const int f = blockIdx.x * 32 + threadIdx.x;
  if (threadIdx.y == 0) {
    int64_t off = -1;
    if (f < a.m) {
      off = 0;
      for (int k = 0; k < N; ++k)
        if (k != n) off += (int64_t)a.idxs[(int64_t)k * a.m + f] * stride[k];
    }
    sbase[threadIdx.x] = off;
  }
  __syncthreads();
  const int64_t off = sbase[threadIdx.x];
  const float* X = (const float*)a.X;
  for (int64_t row = blockIdx.y * (int64_t)blockDim.y + threadIdx.y; row < In; row += (int64_t)gridDim.y * blockDim.y) {
    float re = 0.f, im = 0.f;
    if (off >= 0) {
      const int64_t o = off + row * stride[n];
      re = X[2 * o];
      im = X[2 * o + 1];
    }
    if (f < Kpad) {
      A[row * 2 * Kpad + f] = re;
      A[row * 2 * Kpad + Kpad + f] = im;
    }
  }
}

// out[2 e] = sum_s Pre[s][e], out[2 e + 1] = sum_s Pim[s][e]   (FP64, fixed order)
__global__ void reduce_cplx_pair_kernel(const float* __restrict__ Pre, const float* __restrict__ Pim, int splits,
                                        int64_t count, double* __restrict__ out) {
  PDL_ENTRY();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int q = 0; q < splits; ++q) {
      sr += (double)Pre[(int64_t)q * count + e];
      si += (double)Pim[(int64_t)q * count + e];
    }
    out[2 * e] = sr;
    out[2 * e + 1] = si;
  }
}

// ---------------------------------------------------------------------------
// tensor maps (driver entry point resolved once through the runtime)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

}  // namespace

void* str_tensor_map_encoder() { return (void*)encode_fn(); }

bool tc_supported(int K, int xtype, const void* base) {
  const int es = xtype == XT_BF16 ? 2 : 4;
  if (xtype != XT_BF16 && xtype != XT_F32) return false;
  if (((uintptr_t)base & 15) != 0) return false;
  if (((int64_t)K * es) % 16 != 0) return false;
  return encode_fn() != nullptr;
}

size_t stage1_smem_bytes(int Npad) { return 1024 + 32768 + 2 * (size_t)Npad * 128 + 16384 + 64; }

cudaError_t launch_prep_b(const double* G, int K, int N, int Kpad, int Npad, float* Bhi, float* Blo,
                          cudaStream_t s) {
  const int64_t total = (int64_t)Kpad * Npad;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 1024));
  launch_k(prep_b_kernel, blocks, 256, 0, s, G, K, N, Kpad, Npad, Bhi, Blo);
  return cudaGetLastError();
}

cudaError_t launch_transpose01(const void* in, void* out, int xtype, int d0, int d1, int64_t rest,
                               cudaStream_t s) {
  // about 16 CTAs per SM in all, each looping over its share of the slices
  const int64_t tiles = (int64_t)ceil_div_i(d0, 32) * ceil_div_i(d1, 32);
  const int64_t zc = std::max<int64_t>(1, std::min<int64_t>(rest, std::min<int64_t>(65535, (152 * 16 + tiles - 1) / tiles)));
  dim3 grid((unsigned)ceil_div_i(d0, 32), (unsigned)ceil_div_i(d1, 32), (unsigned)zc);
  dim3 block(32, 8);
  if (xtype == XT_BF16)
    launch_k(transpose01_kernel<__nv_bfloat16>, grid, block, 0, s, (const __nv_bfloat16*)in, (__nv_bfloat16*)out, d0, d1, rest);
  else
    launch_k(transpose01_kernel<float>, grid, block, 0, s, (const float*)in, (float*)out, d0, d1, rest);
  return cudaGetLastError();
}

cudaError_t launch_stage1_tc(const void* Xa, int xtype, int64_t M, int K, const float* Bhi, const float* Blo,
                             int Kpad, int N, int Npad, float* Y, int* status, cudaStream_t s) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const bool bf16 = xtype == XT_BF16;
  const int es = bf16 ? 2 : 4;
  uint32_t cols = 32;
  while ((int)cols < 3 * Npad) cols <<= 1;
  if (cols > 512) return cudaErrorInvalidValue;
  const int nch = Kpad / 32;
  const size_t smp = stage1_persist_smem_bytes(Npad, nch, bf16);
  const bool persist = smp <= 200 * 1024;
  // FP32 persistent path: the TMA tile lands already swizzled (it is the X_hi operand)
  auto encode = [&](CUtensorMap* tm, bool swz) {
    cuuint64_t gdim[2] = {(cuuint64_t)K, (cuuint64_t)M};
    cuuint64_t gstride[1] = {(cuuint64_t)K * es};
    cuuint32_t box[2] = {32, 128};
    cuuint32_t estr[2] = {1, 1};
    return enc(tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
               const_cast<void*>(Xa), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               swz ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  };
  CUtensorMap tm;
  if (encode(&tm, persist && !bf16) != CUDA_SUCCESS) return cudaErrorInvalidValue;
  // warp-specialised persistent kernel when its rings fit (3 X slots, else 2)
  // and two accumulator sets of 3 Npad TMEM columns each fit in 512 columns
  const size_t ws3 = stage1_ws_smem_bytes(Npad, nch, bf16, 3), ws2 = stage1_ws_smem_bytes(Npad, nch, bf16, 2);
  uint32_t cols_ws = 32;
  while ((int)cols_ws < 6 * Npad) cols_ws <<= 1;
  if (persist && ws2 <= 225 * 1024 && cols_ws <= 512) {
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (M + 127) / 128;
    const unsigned gridp = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, sms));
    const bool three = ws3 <= 225 * 1024;
    const size_t smw = three ? ws3 : ws2;
    auto kern = bf16 ? (three ? stage1_ws_kernel<true, 3> : stage1_ws_kernel<true, 2>)
                     : (three ? stage1_ws_kernel<false, 3> : stage1_ws_kernel<false, 2>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
    if (e != cudaSuccess) return e;
    launch_k(kern, gridp, 320, smw, s, tm, Bhi, Blo, (int)M, Kpad, N, Npad, cols_ws, Y, status);
    return cudaGetLastError();
  }
  if (persist) {
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tiles = (M + 127) / 128;
    const unsigned gridp = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, sms));
    if (bf16) {
      cudaError_t e = cudaFuncSetAttribute(stage1_tc_persist_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
      if (e != cudaSuccess) return e;
      launch_k(stage1_tc_persist_kernel<true>, gridp, 128, smp, s, tm, Bhi, Blo, (int)M, Kpad, N, Npad, cols, Y, status);
    } else {
      cudaError_t e = cudaFuncSetAttribute(stage1_tc_persist_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
      if (e != cudaSuccess) return e;
      launch_k(stage1_tc_persist_kernel<false>, gridp, 128, smp, s, tm, Bhi, Blo, (int)M, Kpad, N, Npad, cols, Y, status);
    }
    return cudaGetLastError();
  }
  const size_t sm = stage1_smem_bytes(Npad);
  const unsigned grid = (unsigned)((M + 127) / 128);
  if (bf16) {
    cudaError_t e = cudaFuncSetAttribute(stage1_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    launch_k(stage1_tc_kernel<true>, grid, 128, sm, s, tm, Bhi, Blo, (int)M, Kpad, N, Npad, cols, Y, status, 0);
  } else {
    cudaError_t e = cudaFuncSetAttribute(stage1_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    launch_k(stage1_tc_kernel<false>, grid, 128, sm, s, tm, Bhi, Blo, (int)M, Kpad, N, Npad, cols, Y, status, 0);
  }
  return cudaGetLastError();
}

// Y_part[y] = A[:, K_y] B[K_y, :] on the tensor cores: A row-major [M][Kpad]
// (FP32 or BF16, K contiguous), B given as the split pair (Bhi, Blo) [Npad][Kpad];
// the K chunks are divided over `splits` CTAs per 128-row tile (split K),
// partial products in Y [splits][M][N]
cudaError_t launch_gemm_tc_splitk(const void* A, int xtype, int64_t M, int Kpad, const float* Bhi,
                                  const float* Blo, int N, int Npad, int splits, float* Y, int* status,
                                  cudaStream_t s) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  const bool bf16 = xtype == XT_BF16;
  const int es = bf16 ? 2 : 4;
  if (Kpad % 32 != 0 || ((uintptr_t)A & 15) != 0 || splits < 1) return cudaErrorInvalidValue;
  uint32_t cols = 32;
  while ((int)cols < 3 * Npad) cols <<= 1;
  if (cols > 512) return cudaErrorInvalidValue;
  const int nch = Kpad / 32;
  const int cps = (nch + splits - 1) / splits;
  const int ns = (nch + cps - 1) / cps;   // every split has at least one chunk
  CUtensorMap tm;
  cuuint64_t gdim[2] = {(cuuint64_t)Kpad, (cuuint64_t)M};
  cuuint64_t gstride[1] = {(cuuint64_t)Kpad * es};
  cuuint32_t box[2] = {32, 128};
  cuuint32_t estr[2] = {1, 1};
  if (enc(&tm, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(A),
          gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const size_t sm = stage1_smem_bytes(Npad);
  dim3 grid((unsigned)((M + 127) / 128), (unsigned)ns);
  if (bf16) {
    cudaError_t e = cudaFuncSetAttribute(stage1_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    launch_k(stage1_tc_kernel<true>, grid, 128, sm, s, tm, Bhi, Blo, (int)M, Kpad, N, Npad, cols, Y, status, cps);
  } else {
    cudaError_t e = cudaFuncSetAttribute(stage1_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    launch_k(stage1_tc_kernel<false>, grid, 128, sm, s, tm, Bhi, Blo, (int)M, Kpad, N, Npad, cols, Y, status, cps);
  }
  return cudaGetLastError();
}

int gemm_tc_splitk_count(int Kpad, int splits) {
  const int nch = Kpad / 32;
  const int cps = (nch + splits - 1) / splits;
  return (nch + cps - 1) / cps;
}

cudaError_t launch_sampled_rows(const MttkrpArgs& a, int Kpad, float* Bhi, float* Blo, cudaStream_t s) {
  const int64_t total = a.m * a.R[a.n + 1];
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 127) / 128, 152 * 8));
  launch_k(sampled_rows_kernel, blocks, 128, 0, s, a, Kpad, Bhi, Blo);
  return cudaGetLastError();
}

cudaError_t launch_sampled_rows_cplx(const MttkrpArgs& a, int Kpad, float* Brh, float* Brl, float* Bih, float* Bil,
                                     cudaStream_t s) {
  const int64_t total = a.m * a.R[a.n + 1];
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((total + 127) / 128, 152 * 8));
  launch_k(sampled_rows_cplx_kernel, blocks, 128, 0, s, a, Kpad, Brh, Brl, Bih, Bil);
  return cudaGetLastError();
}

cudaError_t launch_gather_fibres_cplx(const MttkrpArgs& a, int Kpad, float* A, cudaStream_t s) {
  const int64_t In = a.dim[a.n];
  dim3 block(32, 8);
  dim3 grid((unsigned)(Kpad / 32), (unsigned)std::max<int64_t>(1, std::min<int64_t>((In + 7) / 8, 64)));
  launch_k(gather_fibres_cplx_kernel, grid, block, 0, s, a, Kpad, A);
  return cudaGetLastError();
}

cudaError_t launch_reduce_cplx_pair(const float* Pre, const float* Pim, int splits, int64_t count, double* out,
                                    cudaStream_t s) {
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((count + 255) / 256, 152 * 4));
  launch_k(reduce_cplx_pair_kernel, blocks, 256, 0, s, Pre, Pim, splits, count, out);
  return cudaGetLastError();
}

cudaError_t launch_gather_fibres(const MttkrpArgs& a, int Kpad, void* A, cudaStream_t s) {
  const int64_t In = a.dim[a.n];
  dim3 block(32, 8);
  dim3 grid((unsigned)(Kpad / 32), (unsigned)std::max<int64_t>(1, std::min<int64_t>((In + 7) / 8, 64)));
  if (a.xtype == XT_BF16) launch_k(gather_fibres_kernel<__nv_bfloat16>, grid, block, 0, s, a, Kpad, (__nv_bfloat16*)A);
  else if (a.xtype == XT_F32) launch_k(gather_fibres_kernel<float>, grid, block, 0, s, a, Kpad, (float*)A);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

int stage2_plan_splits(const Stage2Args& a, int64_t* per) {
  const int64_t dn = a.dn, ncomb = a.Jlo * a.Jhi;
  int64_t splits;
  if (stage2_warp_rank(a)) {
    // warp kernel: about eight CTAs of four warps per SM, at least one batch per warp
    splits = std::max<int64_t>(1, (8 * 152 + dn - 1) / dn);
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, ncomb / 128));
  } else {
    splits = std::max<int64_t>(1, (2 * 152 + dn - 1) / dn);
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, ncomb / 128));
  }
  int64_t p = (ncomb + splits - 1) / splits;
  *per = std::max<int64_t>(1, p);
  return (int)((ncomb + *per - 1) / *per);
}

cudaError_t launch_stage2(const Stage2Args& a, cudaStream_t s) {
  if (const int rw = stage2_warp_rank(a)) {
    if (a.Jlo * a.Jhi >= ((int64_t)1 << 40)) return cudaErrorInvalidValue;
    const size_t sm = (size_t)4 * 2 * 32 * ((rw * rw) | 1) * sizeof(float);
    auto kern = rw == 2 ? stage2_warp_kernel<2> : rw == 3 ? stage2_warp_kernel<3> : rw == 5 ? stage2_warp_kernel<5>
              : rw == 6 ? stage2_warp_kernel<6> : stage2_warp_kernel<7>;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)a.dn, (unsigned)a.splits);
    launch_k(kern, grid, 128, sm, s, a);
    return cudaGetLastError();
  }
  const int OUTP = a.Rn * a.Rn1;
  if (OUTP > S2_THREADS || a.Rk * a.Rn > S2_THREADS || a.Rn1 * a.Rn > S2_THREADS ||
      a.Jlo * a.Jhi >= ((int64_t)1 << 31))
    return cudaErrorInvalidValue;
  const size_t sm = stage2_smem_bytes(a);
  if (sm > 200 * 1024) return cudaErrorInvalidValue;
  const bool eq = a.Rk == a.Rk1 && a.Rk == a.Rn && a.Rk == a.Rn1;
  const int rt = eq && (a.Rk == 4 || a.Rk == 8) ? a.Rk : 0;
  auto kern = rt == 4 ? stage2_kernel<4> : rt == 8 ? stage2_kernel<8> : stage2_kernel<0>;
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((unsigned)a.dn, (unsigned)a.splits);
  launch_k(kern, grid, S2_THREADS, sm, s, a);
  return cudaGetLastError();
}
