// Masked TR fit loss and its backward on the 5th-generation tensor cores
// (FP32 data).
//
// With the modes split into a prefix (rows) and a suffix (columns), every entry
// of the tensor ring is a dot product of two chain-table rows:
//     TR(G)(r, c) = sum_k Lm[r][k] Rm[c][k],   K = R_1 R_{k+1} <= 64,
// so the reconstruction of a tile is one small GEMM on tcgen05.mma kind::tf32
// with the accumulator in TMEM.  FP32 accuracy comes from the 3-term split used
// by the MTTKRP: Rm = Rm_hi + Rm_lo, Lm = Lm_hi + Lm_lo (each rounded to the
// nearest TF32), P = Rm_hi Lm_hi + (Rm_hi Lm_lo + Rm_lo Lm_hi), the two groups in
// separate TMEM columns.  The loss is 1/2 sum M (X - P)^2; the backward needs
// W = R^T Lm and Z = R Rm of the masked residual R = M (X - P), from which every
// core gradient follows as a small MTTKRP (in the caller).
//
// Kernels (each walks a contiguous range of tiles per persistent CTA and sums in
// a fixed order):
//   loss_fwd_ws_kernel       forward, warp-specialised (TMA producer warp, MMA
//                            warp, eight epilogue warps), X by TMA
//   loss_bwd_ws_kernel<Z/W>  the two backward passes, warp-specialised, the
//                            residual kept in TMEM as the A operand of G = r B
//   loss_fwd_tc_kernel       forward for X that TMA cannot address (unaligned,
//                            odd prefix row count): X copied asynchronously
//                            into padded shared memory, one 128-thread CTA
//   loss_bwd_tc_kernel<Z/W>  the backward passes for such X, X through registers
//
// A wait that times out (an mbarrier never completing) makes the CTA's partial
// sums NaN, so the loss or the gradients read NaN instead of the kernel hanging.
#include <algorithm>
#include <cmath>

#include "kernels.cuh"
#include "ptx.cuh"
#include "tc.cuh"

namespace {

constexpr int kLT = 128;           // tile edge (rows and columns)
constexpr int kChunkBytes = 16384; // one 32-float chunk of a 128-row operand tile
constexpr int kXS = kLT + 4;       // floats per column of the shared X tile (padded)

// T [n][K] FP32 -> hi, lo [n][64] (TF32 values, K padded with zeros)
__global__ void loss_split_kernel(const float* __restrict__ T, int64_t n, int K, float* __restrict__ hi,
                                  float* __restrict__ lo) {
  PDL_ENTRY();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * 64;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e >> 6;
    const int k = (int)(e & 63);
    const float v = k < K ? T[r * K + k] : 0.f;
    const float h = tf32_rn(v);
    hi[e] = h;
    lo[e] = tf32_rn(v - h);
  }
}

// rows r0 .. r0 + 127 of a split table (n rows) into two K-major 128B-swizzled
// operand tiles of two 32-float chunks each (rows past n are zero)
__device__ __forceinline__ void stage_tile(unsigned char* sh, unsigned char* sl, const float* __restrict__ hi,
                                           const float* __restrict__ lo, int64_t r0, int64_t n, int tid) {
  for (int q = tid; q < kLT * 16; q += 128) {
    const int r = q >> 4, pc = q & 15, c = pc >> 3, j = pc & 7;
    const int off = c * kChunkBytes + sw128_off(r, j);
    if (r0 + r < n) {
      cp_async16(sh + off, hi + (r0 + r) * 64 + c * 32 + j * 4);
      cp_async16(sl + off, lo + (r0 + r) * 64 + c * 32 + j * 4);
    } else {
      *(float4*)(sh + off) = make_float4(0.f, 0.f, 0.f, 0.f);
      *(float4*)(sl + off) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// loss_fwd_tc_kernel: 128-column x 128-row tiles (M = 128 columns, N = 128 rows,
// K padded to 8).  Per tile, the operand tiles are staged, then every thread
// issues asynchronous copies of its column's 128 rows of X (contiguous: X(r, c)
// at r + rows c) into a padded shared-memory tile, which stay in flight while the
// MMAs run; the epilogue thread that owns column c (its TMEM lane) then reads X
// from shared memory (rows padded to 132 floats: conflict-free 16-byte reads)
// with its column's mask bits, and accumulates sum M (X - P)^2.  Column tile
// outer, so the Rm operand is staged once per column tile.
__global__ void __launch_bounds__(128, 1) loss_fwd_tc_kernel(const float* __restrict__ Rhi,
                                                             const float* __restrict__ Rlo,
                                                             const float* __restrict__ Lhi,
                                                             const float* __restrict__ Llo, int64_t rows,
                                                             int64_t cols, int K, const float* __restrict__ X,
                                                             const uint32_t* __restrict__ mask, int64_t nwords,
                                                             int vec, double* __restrict__ loss_part) {
  PDL_ENTRY();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sAh = smem;                       // Rm tile, hi (2 chunks)
  unsigned char* sAl = smem + 2 * kChunkBytes;     // Rm tile, lo
  unsigned char* sBh = smem + 4 * kChunkBytes;     // Lm tile, hi
  unsigned char* sBl = smem + 6 * kChunkBytes;     // Lm tile, lo
  float* sX = (float*)(smem + 8 * kChunkBytes);    // X tile, [column][row], padded rows
  uint64_t* bar = (uint64_t*)(sX + kLT * kXS);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  __shared__ double red[4];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) tmem_alloc(tslot, 256);
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  // D F32, A and B TF32, both K-major, N = 128, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kLT >> 3) << 17) |
                         ((uint32_t)(kLT >> 4) << 24);
  const int64_t nrt = (rows + kLT - 1) / kLT, nct = (cols + kLT - 1) / kLT, ntiles = nrt * nct;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(ntiles, t0 + per);
  const int ksteps = (K + 7) / 8;
  uint32_t ph = 0;
  double lsum = 0.0;
  bool failed = false;
  int64_t cur_cb = -1;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t cb = t / nrt, rb = t - cb * nrt;
    const int64_t c = cb * kLT + 32 * warp + lane;   // this thread's column
    const int64_t r0 = rb * kLT;
    const int nr = (int)min((int64_t)kLT, rows - r0);
    const bool col_ok = c < cols;
    const float* xc = X + r0 + rows * c;
    float* sxc = sX + (32 * warp + lane) * kXS;
    // (1) the operand tiles (one commit group)
    if (cb != cur_cb) {
      stage_tile(sAh, sAl, Rhi, Rlo, cb * kLT, cols, tid);
      cur_cb = cb;
    }
    stage_tile(sBh, sBl, Lhi, Llo, rb * kLT, rows, tid);
    cp_async_commit();
    // (2) the column's rows of X (the newest group: still in flight during the MMAs)
    if (col_ok) {
      if (vec) {
        for (int j = 0; j < nr; j += 4) cp_async16(sxc + j, xc + j);   // nr is a multiple of 4 with vec
      } else {
        for (int j = 0; j < nr; ++j) cp_async4(sxc + j, xc + j);
      }
    }
    cp_async_commit();
    // the column's mask bits for rows r0 .. r0 + nr - 1: bits msh .. msh + 127 of
    // five words from word b0 / 32 on (mw[5] is a zero pad for the last window)
    uint32_t mw[6] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0u};
    const int64_t b0 = r0 + rows * c;
    const uint32_t msh = (uint32_t)(b0 & 31);
    if (mask && col_ok) {
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        const int64_t w = (b0 >> 5) + q;
        mw[q] = w < nwords ? mask[w] : 0u;
      }
    }
    cp_async_wait_n<1>();    // all groups but the newest (X) complete: the operand tiles have landed
    fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint64_t dah = desc_sw128(sAh), dal = desc_sw128(sAl), dbh = desc_sw128(sBh), dbl = desc_sw128(sBl);
      for (int st = 0; st < ksteps; ++st) {
        // chunk st / 4 (16 KB further), 8 TF32 = 32 bytes along K within it
        const uint64_t adv = (uint64_t)((st >> 2) * kChunkBytes + (st & 3) * 32) >> 4;
        mma_tf32(tmem, dah + adv, dbh + adv, idesc, st > 0 ? 1u : 0u);
        mma_tf32(tmem + kLT, dah + adv, dbl + adv, idesc, st > 0 ? 1u : 0u);
        mma_tf32(tmem + kLT, dal + adv, dbh + adv, idesc, 1u);
      }
      mma_commit(bar);
    }
    const bool ok = mbar_wait(bar, ph, kWaitNs);
    ph ^= 1;
    cp_async_wait_n<0>();    // this thread's X copies (it alone reads them)
    if (__syncthreads_or(!ok)) { failed = true; break; }
    tc_fence_after();
    // epilogue: this thread's column of the tile, 16 rows at a time
    float ts = 0.f;
    for (int j0 = 0; j0 < kLT; j0 += 16) {
      uint32_t vh[16], vx[16];
      const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)j0;
      tmem_ld_x16_nw(base, vh);
      tmem_ld_x16_nw(base + kLT, vx);
      tmem_wait_ld();
      if (!col_ok || j0 >= nr) continue;
      float xv[16];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float4 q = *(const float4*)(sxc + j0 + 4 * u);
        xv[4 * u] = q.x; xv[4 * u + 1] = q.y; xv[4 * u + 2] = q.z; xv[4 * u + 3] = q.w;
      }
      uint32_t mb = 0xFFFFu;
      if (mask) {
        // bits msh + j0 .. msh + j0 + 15 of the column's words
        const uint32_t bit = msh + (uint32_t)j0;
        const int q = (int)(bit >> 5);
        uint64_t two = 0;
#pragma unroll
        for (int u = 0; u < 5; ++u)
          if (q == u) two = (uint64_t)mw[u] | ((uint64_t)mw[u + 1] << 32);
        mb = (uint32_t)(two >> (bit & 31)) & 0xFFFFu;
      }
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float p = __uint_as_float(vh[u]) + __uint_as_float(vx[u]);
        const bool keep = (j0 + u < nr) && ((mb >> u) & 1u);
        const float r = keep ? xv[u] - p : 0.f;
        ts = fmaf(r, r, ts);
      }
    }
    lsum += (double)ts;
    tc_fence_before();
    __syncthreads();   // TMEM and the operand tiles are reused by the next tile
  }
  // fixed-order block sum of the per-thread partials
#pragma unroll
  for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) red[warp] = lsum;
  __syncthreads();
  if (tid == 0) loss_part[blockIdx.x] = failed ? (double)NAN : (red[0] + red[1]) + (red[2] + red[3]);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}


// ---------------------------------------------------------------------------
// Backward: the two contractions of the masked residual R = M .* (X - TR(G))
//   W[c][k] = sum_r R(r, c) Lm[r][k]     (suffix side)
//   Z[r][k] = sum_c R(r, c) Rm[c][k]     (prefix side)
// as two passes over X, each with the accumulated side in the TMEM lanes.  A
// pass takes a "lane" table A (W pass: Rm, Z pass: Lm; nL rows) and an "other"
// table B (nO rows, and its transpose BT [KG][ldT]); per 128 x 128 tile:
//   1. P[l][o] = sum_k A[l][k] B[o][k]    (tcgen05, 3-term split, TMEM cols 0..255)
//   2. epilogue, thread = (lane l, half of the o-columns): r = M (X - P), split
//      r = r_hi + r_lo (TF32), stored back into TMEM in place of P (r_hi cols
//      0..127, r_lo 128..255)
//   3. G[l][k] = sum_o r[l][o] B[o][k]    (A = r from TMEM, B = BT tile from shared
//      memory; r_hi B_hi + r_hi B_lo + r_lo B_hi; G in TMEM cols 256..)
// The CTA walks a contiguous range of tiles, lane tile outer.  G is accumulated
// in TMEM over one tile only (48 MMA steps), then each thread adds its lane's row
// into the CTA's partial for the lane tile with FP32 adds (a thread-private row
// of global memory, resident in L2); a second kernel sums the partials of each
// lane tile in CTA order.
// ---------------------------------------------------------------------------
constexpr int kGChunkMax = 64 * 128;   // bytes of one 32-float K chunk of the G operand (KG <= 64 rows)

// rows r0 .. r0 + 127 of a split table [n][64]: 16-byte units j < units of each
// row (the units of k < K); rows past n are zeroed
__device__ __forceinline__ void stage_rows(unsigned char* sh, unsigned char* sl, const float* __restrict__ hi,
                                           const float* __restrict__ lo, int64_t r0, int64_t n, int units, int tid,
                                           int nt) {
  for (int q = tid; q < kLT * units; q += nt) {
    const int r = q / units, u = q - r * units, c = u >> 3, j = u & 7;
    const int off = c * kChunkBytes + sw128_off(r, j);
    if (r0 + r < n) {
      cp_async16(sh + off, hi + (r0 + r) * 64 + 4 * u);
      cp_async16(sl + off, lo + (r0 + r) * 64 + 4 * u);
    } else {
      *(float4*)(sh + off) = make_float4(0.f, 0.f, 0.f, 0.f);
      *(float4*)(sl + off) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// columns o0 .. o0 + 127 of the rows k < K of a transposed split table [KG][ldT]
// into a K-major operand of KG rows and four 32-float chunks (KG x 128 bytes each)
__device__ __forceinline__ void stage_cols(unsigned char* sh, unsigned char* sl, const float* __restrict__ hiT,
                                           const float* __restrict__ loT, int64_t ldT, int64_t o0, int K, int KG,
                                           int tid, int nt) {
  const int chunk = KG * 128;
  for (int q = tid; q < K * 32; q += nt) {
    const int k = q >> 5, u = q & 31, c = u >> 3, j = u & 7;
    const int off = c * chunk + sw128_off(k, j);
    const int64_t o = o0 + 4 * u;
    if (o < ldT) {
      cp_async16(sh + off, hiT + k * ldT + o);
      cp_async16(sl + off, loT + k * ldT + o);
    } else {
      *(float4*)(sh + off) = make_float4(0.f, 0.f, 0.f, 0.f);
      *(float4*)(sl + off) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// T [n][K] -> hiT, loT [KG][ldT] (TF32 values; zero for k >= K or o >= n)
__global__ void loss_splitT_kernel(const float* __restrict__ T, int64_t n, int K, int KG, int64_t ldT,
                                   float* __restrict__ hiT, float* __restrict__ loT) {
  PDL_ENTRY();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)KG * ldT;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / ldT);
    const int64_t o = e - k * ldT;
    const float v = (k < K && o < n) ? T[o * K + k] : 0.f;
    const float h = tf32_rn(v);
    hiT[e] = h;
    loT[e] = tf32_rn(v - h);
  }
}

// ZSIDE = false: W pass (lanes = suffix columns c, o = prefix rows r; X(o, l) at
// o + xrows l).  ZSIDE = true: Z pass (lanes = prefix rows, o = suffix columns;
// X(l, o) at l + xrows o).  part: [grid][maxslots][128][64] FP32 partial sums of G.
// 256 threads: thread tid serves TMEM lane i = tid % 128 and the tile's o-columns
// 64 h .. 64 h + 63, h = tid / 128 (warps w and w + 4 share a lane quarter).  Per
// tile, each thread first loads its 64 values of X into registers (they stay in
// flight while the operands are staged, the previous tile's G MMAs are retired and
// the P MMAs run) and prefetches the next tile's X into L2.
template <bool ZSIDE>
__global__ void __launch_bounds__(256, 1) loss_bwd_tc_kernel(
    const float* __restrict__ Ahi, const float* __restrict__ Alo, const float* __restrict__ Bhi,
    const float* __restrict__ Blo, const float* __restrict__ BThi, const float* __restrict__ BTlo, int64_t nL,
    int64_t nO, int64_t ldT, int K, int KG, int64_t xrows, const float* __restrict__ X,
    const uint32_t* __restrict__ mask, int64_t nwords, int vec, int maxslots, float* __restrict__ part) {
  PDL_ENTRY();
  constexpr int NT = 256, OH = 64;   // threads; o-columns per thread
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sAh = smem;                          // lane-side tile, hi (2 chunks)
  unsigned char* sAl = smem + 2 * kChunkBytes;        // lane-side tile, lo
  unsigned char* sBh = smem + 4 * kChunkBytes;        // other-side tile, hi
  unsigned char* sBl = smem + 6 * kChunkBytes;        // other-side tile, lo
  unsigned char* sGh = smem + 8 * kChunkBytes;        // G operand (BT tile), hi: 4 chunks of KG x 128 B
  unsigned char* sGl = sGh + 4 * kGChunkMax;          // G operand, lo
  uint32_t* sM = (uint32_t*)(sGl + 4 * kGChunkMax);   // [128 columns][5] mask words
  uint32_t* sMw = sM + kLT * 5;                       // [4 lane quarters][128 columns] aligned mask words (Z pass)
  uint64_t* bar = (uint64_t*)(sMw + 4 * kLT);
  uint32_t* tslot = (uint32_t*)(bar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i = tid & (kLT - 1), h = tid >> 7, quarter = warp & 3;

  if (warp == 0) tmem_alloc(tslot, 512);
  if (tid == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // zero every operand byte once: the units past K and the G rows past K stay zero
  for (int q = tid; q < (8 * kChunkBytes + 8 * kGChunkMax) / 16; q += NT)
    ((float4*)smem)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tl = (uint32_t)(32 * quarter) << 16;   // this warp's lane quarter
  // D F32, A and B TF32, K-major; M = 128; N = 128 (P) or KG (G)
  const uint32_t idP = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kLT >> 3) << 17) | ((uint32_t)(kLT >> 4) << 24);
  const uint32_t idG = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(KG >> 3) << 17) | ((uint32_t)(kLT >> 4) << 24);
  const int64_t nLT = (nL + kLT - 1) / kLT, nOT = (nO + kLT - 1) / kLT, ntiles = nLT * nOT;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(ntiles, t0 + per);
  const int64_t lt_first = t0 / nOT;
  const int ksteps = (K + 7) / 8, units = (K + 3) / 4;
  const int gchunk = KG * 128;
  const int gh = KG / 2;   // G columns per thread half (a multiple of 8)
  float* pbase = part + (int64_t)blockIdx.x * maxslots * kLT * 64;
  uint32_t ph = 0;
  bool failed = false, g_pending = false, g_first = false, tile_first = true;
  int64_t cur_lt = -1, g_lt = -1;

  // wait for the pending tile's G MMAs, then add its G (this thread's lane, its
  // half of the columns) into the running partial of its lane tile (or start it,
  // on the lane tile's first tile); the old partial is loaded before the wait.
  // False on a timeout.
  auto retire_g = [&]() -> bool {
    float* dst = pbase + ((g_lt - lt_first) * kLT + i) * 64 + h * gh;
    float4 pv[8];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      pv[q] = (!g_first && 4 * q < gh) ? *(const float4*)(dst + 4 * q) : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool ok = mbar_wait(bar, ph, kWaitNs);
    ph ^= 1;
    if (__syncthreads_or(!ok)) return false;
    tc_fence_after();
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 8) {
      if (c0 >= gh) break;
      uint32_t v[8];
      tmem_ld_x8(tmem + tl + 256 + (uint32_t)(h * gh + c0), v);
#pragma unroll
      for (int u = 0; u < 8; u += 4) {
        float4 a = pv[(c0 + u) >> 2];
        a.x += __uint_as_float(v[u]);
        a.y += __uint_as_float(v[u + 1]);
        a.z += __uint_as_float(v[u + 2]);
        a.w += __uint_as_float(v[u + 3]);
        *(float4*)(dst + c0 + u) = a;
      }
    }
    return true;
  };
  // L2 prefetch of X tile t: 128 segments of contiguous rows, one per thread of
  // the first half
  auto prefetch = [&](int64_t t) {
    if (!vec || t >= t1 || h != 0) return;
    const int64_t l0 = (t / nOT) * kLT, o0 = (t % nOT) * kLT;
    if (ZSIDE) {
      const int64_t c = o0 + i;
      if (c < nO) prefetch_l2_bulk(X + l0 + xrows * c, (uint32_t)min((int64_t)kLT, nL - l0) * 4);
    } else {
      const int64_t c = l0 + i;
      if (c < nL) prefetch_l2_bulk(X + o0 + xrows * c, (uint32_t)min((int64_t)kLT, nO - o0) * 4);
    }
  };

  prefetch(t0);
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t lt = t / nOT, ot = t - lt * nOT;
    const int64_t l0 = lt * kLT, o0 = ot * kLT;
    const int no = (int)min((int64_t)kLT, nO - o0);
    const int oh = 64 * h;            // this thread's first o-column in the tile
    const bool lane_ok = l0 + i < nL;
    // (0) this thread's 64 values of X, then the next tile's X into L2
    float xr[OH];
    if (ZSIDE) {
      const float* xp = X + l0 + i + xrows * (o0 + oh);
#pragma unroll
      for (int u = 0; u < OH; ++u) xr[u] = (lane_ok && oh + u < no) ? __ldcs(xp + xrows * u) : 0.f;
    } else if (vec) {
      const float4* xp = (const float4*)(X + o0 + oh + xrows * (l0 + i));
#pragma unroll
      for (int q = 0; q < OH / 4; ++q) {
        const float4 v = (lane_ok && oh + 4 * q < no) ? __ldcs(xp + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        xr[4 * q] = v.x; xr[4 * q + 1] = v.y; xr[4 * q + 2] = v.z; xr[4 * q + 3] = v.w;
      }
    } else {
      const float* xp = X + o0 + oh + xrows * (l0 + i);
#pragma unroll
      for (int u = 0; u < OH; ++u) xr[u] = (lane_ok && oh + u < no) ? xp[u] : 0.f;
    }
    prefetch(t + 1);
    // (1) the P operands (not read by the G MMAs still in flight)
    if (lt != cur_lt) stage_rows(sAh, sAl, Ahi, Alo, l0, nL, units, tid, NT);
    stage_rows(sBh, sBl, Bhi, Blo, o0, nO, units, tid, NT);
    cp_async_commit();
    // (2) the previous tile's G MMAs read TMEM cols 0..255 and the G operand
    if (g_pending) {
      if (!retire_g()) { failed = true; break; }
      g_pending = false;
    }
    // (3) a new lane tile starts a new partial
    if (lt != cur_lt) {
      cur_lt = lt;
      tile_first = true;
    }
    // (4) the G operand and the tile's mask words
    stage_cols(sGh, sGl, BThi, BTlo, ldT, o0, K, KG, tid, NT);
    for (int q = tid; q < kLT * 5; q += NT) {
      const int g = q / 5, w = q - 5 * g;
      const int64_t col = ZSIDE ? o0 + g : l0 + g;
      const int64_t wi = (((ZSIDE ? l0 : o0) + xrows * col) >> 5) + w;
      const bool ok = mask && col < (ZSIDE ? nO : nL) && wi < nwords;
      if (ok) cp_async4(sM + q, mask + wi);
      else sM[q] = mask ? 0u : 0xFFFFFFFFu;
    }
    cp_async_commit();
    cp_async_wait_n<0>();
    fence_proxy_async();
    __syncthreads();
    // (5) P on the tensor cores
    if (tid == 0) {
      tc_fence_after();
      const uint64_t dah = desc_sw128(sAh), dal = desc_sw128(sAl), dbh = desc_sw128(sBh), dbl = desc_sw128(sBl);
      for (int st = 0; st < ksteps; ++st) {
        const uint64_t adv = (uint64_t)((st >> 2) * kChunkBytes + (st & 3) * 32) >> 4;
        mma_tf32(tmem, dah + adv, dbh + adv, idP, st > 0 ? 1u : 0u);
        mma_tf32(tmem + kLT, dah + adv, dbl + adv, idP, st > 0 ? 1u : 0u);
        mma_tf32(tmem + kLT, dal + adv, dbh + adv, idP, 1u);
      }
      mma_commit(bar);
    }
    // mask bits: per column, the 32 bits of a lane quarter's rows (Z pass) or
    // this thread's five words (W pass)
    uint32_t mw[6] = {0u, 0u, 0u, 0u, 0u, 0u};
    uint32_t msh = 0;
    if (ZSIDE) {
      for (int q = tid; q < 4 * kLT; q += NT) {
        const int w = q >> 7, g = q & (kLT - 1);
        const uint32_t sh = (uint32_t)((l0 + xrows * (o0 + g)) & 31) + 32u * w;
        const uint32_t lo = sM[g * 5 + (sh >> 5)], hi = (sh >> 5) < 4 ? sM[g * 5 + (sh >> 5) + 1] : 0u;
        sMw[q] = (uint32_t)((((uint64_t)hi << 32) | lo) >> (sh & 31));
      }
    } else {
#pragma unroll
      for (int q = 0; q < 5; ++q) mw[q] = sM[i * 5 + q];
      msh = (uint32_t)((o0 + xrows * (l0 + i)) & 31) + (uint32_t)oh;   // bit of row o0 + oh in the window
    }
    const bool ok = mbar_wait(bar, ph, kWaitNs);
    ph ^= 1;
    if (__syncthreads_or(!ok)) { failed = true; break; }   // also orders the sMw writes
    tc_fence_after();
    // (6) epilogue: r = M (X - P) split into TF32 hi + lo, back into TMEM
#pragma unroll
    for (int j0 = 0; j0 < OH; j0 += 16) {
      uint32_t vh[16], vx[16];
      const uint32_t col = (uint32_t)(oh + j0);
      tmem_ld_x16_nw(tmem + tl + col, vh);
      tmem_ld_x16_nw(tmem + tl + kLT + col, vx);
      uint32_t mb;
      if (ZSIDE) {
        mb = 0;
#pragma unroll
        for (int u = 0; u < 16; ++u) mb |= ((sMw[quarter * kLT + oh + j0 + u] >> lane) & 1u) << u;
      } else {
        const uint32_t bit = msh + (uint32_t)j0;   // at most 31 + 64 + 48 = 143
        const int q = (int)(bit >> 5);
        uint64_t two = 0;
#pragma unroll
        for (int u = 0; u < 5; ++u)
          if (q == u) two = (uint64_t)mw[u] | ((uint64_t)mw[u + 1] << 32);
        mb = (uint32_t)(two >> (bit & 31)) & 0xFFFFu;
      }
      tmem_wait_ld();
      uint32_t rh[16], rl[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const float p = __uint_as_float(vh[u]) + __uint_as_float(vx[u]);
        const bool keep = lane_ok && (oh + j0 + u < no) && ((mb >> u) & 1u);
        const float r = keep ? xr[j0 + u] - p : 0.f;
        const float hv = tf32_rn(r);
        rh[u] = __float_as_uint(hv);
        rl[u] = __float_as_uint(tf32_rn(r - hv));
      }
      tmem_st_x16(tmem + tl + col, rh);
      tmem_st_x16(tmem + tl + kLT + col, rl);
    }
    tmem_wait_st();
    tc_fence_before();
    __syncthreads();
    // (7) G = r B on the tensor cores, A = r from TMEM
    if (tid == 0) {
      tc_fence_after();
      const uint64_t dgh = desc_sw128(sGh), dgl = desc_sw128(sGl);
      for (int st = 0; st < kLT / 8; ++st) {
        const uint64_t adv = (uint64_t)((st >> 2) * gchunk + (st & 3) * 32) >> 4;
        const uint32_t a_hi = tmem + (uint32_t)(8 * st), a_lo = tmem + kLT + (uint32_t)(8 * st);
        mma_tf32_ts(tmem + 256, a_hi, dgh + adv, idG, st > 0 ? 1u : 0u);
        mma_tf32_ts(tmem + 256, a_hi, dgl + adv, idG, 1u);
        mma_tf32_ts(tmem + 256, a_lo, dgh + adv, idG, 1u);
      }
      mma_commit(bar);
    }
    g_pending = true;
    g_lt = lt;
    g_first = tile_first;
    tile_first = false;
  }
  if (!failed && g_pending && !retire_g()) failed = true;
  cp_async_wait_n<0>();
  if (failed) {
    // every partial this CTA owns reads NaN, so the gradients do
    for (int64_t q = tid; q < (int64_t)maxslots * kLT * 64; q += NT) pbase[q] = __int_as_float(0x7fc00000);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// Warp-specialised form of the two backward passes (X 16-byte aligned with a
// prefix row count that is a multiple of 4): 128 x 64 tiles (lanes x o) through
// two two-stage shared-memory rings and two TMEM buffers.  Ring A (the operand
// rows and the X tile) is refilled once the epilogue has read its X tile (which
// also means P is done); ring G (the G operand) once G is done, so the refill
// of the next tiles' X does not wait for the G MMAs.
//   warp 0 (producer): per tile, TMA loads of the other side's operand rows (64
//     rows of B hi / lo), of the G operand (KG rows x 64 o of BT hi / lo; both
//     128-byte swizzled, K-major: the tensor cores take TF32 operands K-major
//     only) and of the X tile (one box of 128 rows x 64 columns for the Z pass;
//     two 128-byte-swizzled boxes of 32 rows x 128 columns for the W pass, so
//     that a lane's 16-byte reads of its column are conflict-free), all completing
//     on the stage's full barriers (A: rows and X; G: the G operand); and an L2
//     prefetch of the X tile two tiles ahead.
//   warp 1 (MMA, one thread): P(t) = A B^T into TMEM buffer t % 2 (A = the
//     lane-side rows, held in TMEM for the lane tile); G(t) = r(t) B from the G
//     operand, accumulated in TMEM over the CTA's tiles of a lane tile.  Each is
//     issued as soon as its inputs are ready.
//   warps 2-9 (epilogue, one TMEM lane and 32 of the tile's 64 o-columns per
//     thread): r = M (X - P) split into TF32 hi + lo, back into the buffer; at a
//     lane-tile change, the finished G to the CTA's partial and the new lane-side
//     rows into TMEM.
// TMEM columns: P / r buffers 0..127 and 128..255 (each hh | cross, then r_hi |
// r_lo), G 256..319, A_hi 320..383, A_lo 384..447.
// ---------------------------------------------------------------------------
constexpr int kWT = 64;                   // o-columns per tile
constexpr int kWsBP = 32768;              // B operand: (hi, lo) x 2 chunks x (64 rows x 128 B)
constexpr int kWsG = 32768;               // G operand: (hi, lo) x 2 chunks x (KG <= 64 rows x 128 B)
constexpr int kWsX = 32768;               // X tile, 128 x 64 FP32
constexpr int kWsA = kWsBP + kWsX;        // ring A stage
constexpr int kWsNS = 2;                  // stages of each ring (= TMEM buffers)

template <bool ZSIDE>
__global__ void __launch_bounds__(320, 1) loss_bwd_ws_kernel(
    const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
    const __grid_constant__ CUtensorMap tmGh, const __grid_constant__ CUtensorMap tmGl,
    const __grid_constant__ CUtensorMap tmX, const float* __restrict__ Ahi, const float* __restrict__ Alo, int64_t nL,
    int64_t nO, int K, int KG, int64_t xrows, const uint32_t* __restrict__ mask, int64_t nwords, int maxslots,
    float* __restrict__ part) {
  PDL_ENTRY();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* ringG = smem + kWsNS * kWsA;
  uint64_t* bars = (uint64_t*)(ringG + kWsNS * kWsG);
  uint64_t* full = bars;              // [2] producer -> MMA, epilogue (operand rows and X landed)
  uint64_t* fullg = bars + 2;         // [2] producer -> MMA (G operand landed)
  uint64_t* emptyg = bars + 4;        // [2] MMA -> producer (G(t) done: the G stage is free)
  uint64_t* pfull = bars + 6;         // [2] MMA -> epilogue (P(t) in its TMEM buffer)
  uint64_t* rfull = bars + 8;         // [2] epilogue -> MMA, producer (r(t) written, X(t) read), 256 arrivals
  uint64_t* tfree = bars + 10;        // [2] MMA -> MMA (G(t) done: its TMEM buffer is free)
  uint64_t* gdone = bars + 12;        // MMA -> epilogue (last G of a lane tile done)
  uint64_t* aready = bars + 13;       // epilogue -> MMA (lane-side rows in TMEM), 256 arrivals
  uint32_t* tslot = (uint32_t*)(bars + 14);
  volatile int* s_fail = (volatile int*)(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 1) tmem_alloc(tslot, 512);
  if (tid == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&fullg[b], 1);
      mbar_init(&emptyg[b], 1);
      mbar_init(&pfull[b], 1);
      mbar_init(&rfull[b], 256);
      mbar_init(&tfree[b], 1);
    }
    mbar_init(gdone, 1);
    mbar_init(aready, 256);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int64_t nLT = (nL + kLT - 1) / kLT, nOT = (nO + kWT - 1) / kWT, ntiles = nLT * nOT;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(ntiles, t0 + per);
  const int64_t lt_first = t0 / nOT;
  const int ksteps = (K + 7) / 8, nch = (K + 31) / 32;

  if (warp == 0) {
    // ---------------- producer ----------------
    auto prefetch_x = [&](int64_t t) {
      const int64_t l2 = (t / nOT) * kLT, o2 = (t % nOT) * kWT;
      if (ZSIDE) {
        tma_prefetch_2d(&tmX, (int)l2, (int)o2);
      } else {
        tma_prefetch_2d(&tmX, (int)o2, (int)l2);
        tma_prefetch_2d(&tmX, (int)o2 + 32, (int)l2);
      }
    };
    if (lane == 0)
      for (int64_t t = t0; t < min(t1, t0 + kWsNS); ++t) prefetch_x(t);
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t j = t - t0;
      const int s = (int)(j & 1);
      const uint32_t n = (uint32_t)(j >> 1);
      // ring A: free once the epilogue of tile t - 2 has read its X
      if (j >= kWsNS) {
        const bool ok = mbar_wait(&rfull[s], (n - 1) & 1u, kWaitNs);
        if (__any_sync(0xffffffffu, !ok) || *s_fail) { if (lane == 0) *s_fail = 1; break; }
      }
      const int64_t l0 = (t / nOT) * kLT, o0 = (t % nOT) * kWT;
      unsigned char* st = smem + (size_t)s * kWsA;
      if (lane == 0) {
        mbar_expect_tx(&full[s], (uint32_t)(nch * 2 * 8192 + kLT * kWT * 4));
        for (int c = 0; c < nch; ++c) {
          tma_load_2d(st + c * 8192, &tmBh, &full[s], c * 32, (int)o0);
          tma_load_2d(st + 16384 + c * 8192, &tmBl, &full[s], c * 32, (int)o0);
        }
        // the X tile (X as a 2-D tensor [suffix columns][prefix rows]; zero past its edges)
        unsigned char* sx = st + kWsBP;
        if (ZSIDE) {
          tma_load_2d(sx, &tmX, &full[s], (int)l0, (int)o0);             // [64 o][128 rows], unswizzled
        } else {
          tma_load_2d(sx, &tmX, &full[s], (int)o0, (int)l0);             // [128 lanes][rows o0 .. +31], swizzled
          tma_load_2d(sx + 16384, &tmX, &full[s], (int)o0 + 32, (int)l0);
        }
        if (t + kWsNS < t1) prefetch_x(t + kWsNS);
      }
      __syncwarp();
      // ring G: free once G(t - 2) is done
      if (j >= kWsNS) {
        const bool ok = mbar_wait(&emptyg[s], (n - 1) & 1u, kWaitNs);
        if (__any_sync(0xffffffffu, !ok) || *s_fail) { if (lane == 0) *s_fail = 1; break; }
      }
      if (lane == 0) {
        unsigned char* sg = ringG + (size_t)s * kWsG;
        mbar_expect_tx(&fullg[s], (uint32_t)(2 * 2 * KG * 128));
        for (int c = 0; c < 2; ++c) {
          tma_load_2d(sg + c * KG * 128, &tmGh, &fullg[s], (int)o0 + 32 * c, 0);
          tma_load_2d(sg + 16384 + c * KG * 128, &tmGl, &fullg[s], (int)o0 + 32 * c, 0);
        }
      }
      __syncwarp();
    }
  } else if (warp == 1) {
    // ---------------- MMA issue ----------------
    if (lane == 0) {
      const uint32_t idP = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kWT >> 3) << 17) | ((uint32_t)(kLT >> 4) << 24);
      const uint32_t idG = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(KG >> 3) << 17) | ((uint32_t)(kLT >> 4) << 24);
      bool fail = false;
      // issue P and G in the order their inputs become ready: P(tp) once its
      // stage has landed and G(tp - 2), the last reader of its TMEM buffer, is
      // done, and, for the first tile of a lane tile, once every G of the
      // previous lane tile is issued and the new lane-side rows are in TMEM;
      // G(tg) once the epilogue has written r(tg).
      int64_t tp = t0, tg = t0, lt_p = -1;
      uint32_t m = 0;
      uint64_t t_prog = gtimer();
      while (tg < t1) {
        bool progressed = false;
        if (tp < t1) {
          const int64_t jp = tp - t0;
          const int64_t lt = tp / nOT;
          const bool new_lt = lt != lt_p;
          const int s = (int)(jp & 1), b = s;
          bool can = !new_lt || tp == t0 || tg == tp;
          if (can && jp >= 2) can = mbar_try_wait(&tfree[b], (uint32_t)((jp >> 1) - 1) & 1u);
          if (can && new_lt) can = mbar_try_wait(aready, m & 1u);
          if (can) can = mbar_try_wait(&full[s], (uint32_t)(jp >> 1) & 1u);
          if (can) {
            if (new_lt) ++m;
            tc_fence_after();
            const uint64_t bh = desc_sw128(smem + (size_t)s * kWsA), bl = desc_sw128(smem + (size_t)s * kWsA + 16384);
            const uint32_t d = tmem + 128u * b;
            for (int k8 = 0; k8 < ksteps; ++k8) {
              const uint64_t adv = (uint64_t)((k8 >> 2) * 8192 + (k8 & 3) * 32) >> 4;
              const uint32_t a_hi = tmem + 320u + 8u * k8, a_lo = tmem + 384u + 8u * k8;
              mma_tf32_ts(d, a_hi, bh + adv, idP, k8 > 0 ? 1u : 0u);
              mma_tf32_ts(d + 64u, a_hi, bl + adv, idP, k8 > 0 ? 1u : 0u);
              mma_tf32_ts(d + 64u, a_lo, bh + adv, idP, 1u);
            }
            mma_commit(&pfull[b]);
            lt_p = lt;
            ++tp;
            progressed = true;
          }
        }
        if (tg < tp) {
          const int64_t jg = tg - t0;
          const int s = (int)(jg & 1), b = s;
          if (mbar_try_wait(&rfull[b], (uint32_t)(jg >> 1) & 1u) && mbar_try_wait(&fullg[s], (uint32_t)(jg >> 1) & 1u)) {
            tc_fence_after();
            const bool first = tg == t0 || tg / nOT != (tg - 1) / nOT;
            const uint64_t gh = desc_sw128(ringG + (size_t)s * kWsG);
            const uint64_t gl = desc_sw128(ringG + (size_t)s * kWsG + 16384);
            for (int k8 = 0; k8 < kWT / 8; ++k8) {
              const uint64_t adv = (uint64_t)((k8 >> 2) * KG * 128 + (k8 & 3) * 32) >> 4;
              const uint32_t a_hi = tmem + 128u * b + 8u * k8, a_lo = a_hi + 64u;
              mma_tf32_ts(tmem + 256, a_hi, gh + adv, idG, (first && k8 == 0) ? 0u : 1u);
              mma_tf32_ts(tmem + 256, a_hi, gl + adv, idG, 1u);
              mma_tf32_ts(tmem + 256, a_lo, gh + adv, idG, 1u);
            }
            mma_commit(&emptyg[s]);
            mma_commit(&tfree[b]);
            // the last G of its lane tile: the epilogue may read G out
            if (tg == t1 - 1 || (tg + 1) / nOT != tg / nOT) mma_commit(gdone);
            ++tg;
            progressed = true;
          }
        }
        if (progressed) t_prog = gtimer();
        else if (*s_fail || gtimer() - t_prog > kWaitNs) { fail = true; break; }
      }
      if (fail) *s_fail = 1;
    }
  } else {
    // ---------------- epilogue ----------------
    // warps 2..9: lane quarter warp % 4, o-columns 32 half .. 32 half + 31
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int li = 32 * quarter + lane;                 // TMEM lane = row of the lane tile
    const uint32_t tl = (uint32_t)(32 * quarter) << 16;
    const int ka = 8 * ksteps;                         // lane-side columns the MMAs read
    const int gh = KG / 2;                             // G columns flushed by each half (a multiple of 8)
    float* pbase = part + (int64_t)blockIdx.x * maxslots * kLT * 64;
    bool fail = false;
    int64_t cur_lt = -1;
    uint32_t m = 0;
    // the finished lane tile's G (this lane's row, this half's columns) to the CTA's partial
    auto flush_g = [&](int64_t lt) -> bool {
      const bool ok = mbar_wait(gdone, (m - 1) & 1u, kWaitNs);
      if (__any_sync(0xffffffffu, !ok)) return false;
      tc_fence_after();
      float* dst = pbase + ((lt - lt_first) * kLT + li) * 64 + half * gh;
      for (int c0 = 0; c0 < gh; c0 += 8) {
        uint32_t v[8];
        tmem_ld_x8(tmem + tl + 256u + (uint32_t)(half * gh + c0), v);
        *(float4*)(dst + c0) = make_float4(__uint_as_float(v[0]), __uint_as_float(v[1]), __uint_as_float(v[2]),
                                           __uint_as_float(v[3]));
        *(float4*)(dst + c0 + 4) = make_float4(__uint_as_float(v[4]), __uint_as_float(v[5]),
                                               __uint_as_float(v[6]), __uint_as_float(v[7]));
      }
      return true;
    };
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t j = t - t0;
      const int s = (int)(j & 1), b = s;
      const int64_t lt = t / nOT;
      const int64_t l0 = lt * kLT, o0 = (t % nOT) * kWT;
      const int no = (int)min((int64_t)kWT, nO - o0);
      const bool lane_ok = l0 + li < nL;
      if (lt != cur_lt) {
        if (cur_lt >= 0 && !flush_g(cur_lt)) { fail = true; break; }
        // the lane-side rows of the new lane tile into TMEM (half 0: hi, half 1: lo)
        const float* ar = (half == 0 ? Ahi : Alo) + (l0 + li) * 64;
        for (int c0 = 0; c0 < ka; c0 += 16) {
          uint32_t v[16];
#pragma unroll
          for (int u = 0; u < 16; u += 4) {
            const float4 q = lane_ok ? *(const float4*)(ar + c0 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
            v[u] = __float_as_uint(q.x); v[u + 1] = __float_as_uint(q.y);
            v[u + 2] = __float_as_uint(q.z); v[u + 3] = __float_as_uint(q.w);
          }
          tmem_st_x16(tmem + tl + (half == 0 ? 320u : 384u) + (uint32_t)c0, v);
        }
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(aready);
        cur_lt = lt;
        ++m;
      }
      // mask bits of this thread's 32 o-columns (loaded before the waits)
      uint32_t mword = 0xFFFFFFFFu;   // W pass: bit u = row o0 + 32 half + u of this lane's column
      uint32_t mz = 0xFFFFFFFFu;      // Z pass: lane q holds column 32 half + q for this warp's 32 rows
      if (mask) {
        if (ZSIDE) {
          const int oc = 32 * half + lane;
          mz = 0;
          if (oc < no) {
            const int64_t b0 = l0 + 32 * quarter + xrows * (o0 + oc), w = b0 >> 5;
            const uint32_t lo = w < nwords ? mask[w] : 0u, hi = w + 1 < nwords ? mask[w + 1] : 0u;
            mz = (uint32_t)((((uint64_t)hi << 32) | lo) >> (b0 & 31));
          }
        } else {
          const int64_t b0 = o0 + 32 * half + xrows * (l0 + li), w = b0 >> 5;
          const uint32_t lo = (lane_ok && w < nwords) ? mask[w] : 0u;
          const uint32_t hi = (lane_ok && w + 1 < nwords) ? mask[w + 1] : 0u;
          mword = (uint32_t)((((uint64_t)hi << 32) | lo) >> (b0 & 31));
        }
      }
      const bool ok1 = mbar_wait(&full[s], (uint32_t)(j >> 1) & 1u, kWaitNs);
      const bool ok2 = ok1 && mbar_wait(&pfull[b], (uint32_t)(j >> 1) & 1u, kWaitNs);
      if (__any_sync(0xffffffffu, !ok2) || *s_fail) { fail = true; break; }
      tc_fence_after();
      const float* sX = (const float*)(smem + (size_t)s * kWsA + kWsBP);
      const uint32_t pb = tmem + tl + 128u * b;
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 16) {
        const int cb = 32 * half + c0;   // first o-column of the chunk in the tile
        uint32_t vh[16], vx[16];
        tmem_ld_x16_nw(pb + (uint32_t)cb, vh);
        tmem_ld_x16_nw(pb + 64u + (uint32_t)cb, vx);
        float xv[16];
        uint32_t mb;
        if (ZSIDE) {
#pragma unroll
          for (int u = 0; u < 16; ++u) xv[u] = sX[(cb + u) * kLT + li];
          mb = 0;
#pragma unroll
          for (int u = 0; u < 16; ++u) mb |= ((__shfl_sync(0xffffffffu, mz, c0 + u) >> lane) & 1u) << u;
        } else {
          // rows cb .. cb + 15 of this lane's column: 16-byte units c0 / 4 .. + 3 of its
          // 128-byte row in box half `half`, 128-byte swizzled
          const unsigned char* xrow = (const unsigned char*)sX + half * 16384 + li * 128;
#pragma unroll
          for (int u = 0; u < 16; u += 4) {
            const int unit = (c0 + u) >> 2;
            const float4 q = *(const float4*)(xrow + ((unit ^ (li & 7)) << 4));
            xv[u] = q.x; xv[u + 1] = q.y; xv[u + 2] = q.z; xv[u + 3] = q.w;
          }
          mb = (mword >> c0) & 0xFFFFu;
        }
        tmem_wait_ld();
        uint32_t rh[16], rl[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float p = __uint_as_float(vh[u]) + __uint_as_float(vx[u]);
          const bool keep = lane_ok && (cb + u < no) && ((mb >> u) & 1u);
          const float r = keep ? xv[u] - p : 0.f;
          const float hv = tf32_rn(r);
          rh[u] = __float_as_uint(hv);
          rl[u] = __float_as_uint(tf32_rn(r - hv));
        }
        tmem_st_x16(pb + (uint32_t)cb, rh);
        tmem_st_x16(pb + 64u + (uint32_t)cb, rl);
      }
      tmem_wait_st();
      tc_fence_before();
      mbar_arrive(&rfull[b]);
    }
    if (!fail && cur_lt >= 0 && !flush_g(cur_lt)) fail = true;
    if (fail) {
      *s_fail = 1;
      // every partial this CTA owns reads NaN, so the gradients do
      for (int64_t q = tid - 64; q < (int64_t)maxslots * kLT * 64; q += 256) pbase[q] = __int_as_float(0x7fc00000);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// Warp-specialised forward (X 16-byte aligned with a prefix row count that is a
// multiple of 4): sum M (X - P)^2 over 128 x 64 tiles (lanes = suffix columns,
// o = prefix rows), three shared-memory stages and three TMEM buffers.
//   warp 0 (producer): per tile, TMA loads of the 64 prefix rows of Lm (hi / lo)
//     and of the X tile (two 128-byte-swizzled boxes of 32 rows x 128 columns),
//     on the stage's full barrier; a stage is refilled once the epilogue is done
//     with it.
//   warp 1 (MMA, one thread): P(t) = Rm Lm^T into TMEM buffer t % 3 (the lane
//     tile's Rm rows held in TMEM), once its stage has landed and the epilogue
//     has read the buffer's previous tile.
//   warps 2-9 (epilogue, one TMEM lane and 32 of the tile's o-columns per
//     thread): the masked squared residuals, FP32 per tile and FP64 across
//     tiles; at a lane-tile change, the new Rm rows into TMEM.
// TMEM columns: P buffers 128 b .. 128 b + 127, b = 0..2 (hh | cross), Rm_hi
// 384..447, Rm_lo 448..511.
// ---------------------------------------------------------------------------
constexpr int kFwNS = 3;
constexpr int kFwStage = kWsBP + kWsX;

__global__ void __launch_bounds__(320, 1) loss_fwd_ws_kernel(
    const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
    const __grid_constant__ CUtensorMap tmX, const float* __restrict__ Ahi, const float* __restrict__ Alo, int64_t nL,
    int64_t nO, int K, int64_t xrows, const uint32_t* __restrict__ mask, int64_t nwords,
    double* __restrict__ loss_part) {
  PDL_ENTRY();
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(smem + kFwNS * kFwStage);
  uint64_t* full = bars;              // [3] producer -> MMA, epilogue
  uint64_t* pfull = bars + 3;         // [3] MMA -> epilogue
  uint64_t* rfree = bars + 6;         // [3] epilogue -> producer, MMA (stage and buffer read), 256 arrivals
  uint64_t* aready = bars + 9;        // epilogue -> MMA (Rm rows in TMEM), 256 arrivals
  uint32_t* tslot = (uint32_t*)(bars + 10);
  volatile int* s_fail = (volatile int*)(tslot + 1);
  __shared__ double red[8];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 1) tmem_alloc(tslot, 512);
  if (tid == 0) {
    for (int q = 0; q < kFwNS; ++q) {
      mbar_init(&full[q], 1);
      mbar_init(&pfull[q], 1);
      mbar_init(&rfree[q], 256);
    }
    mbar_init(aready, 256);
    *s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int64_t nLT = (nL + kLT - 1) / kLT, nOT = (nO + kWT - 1) / kWT, ntiles = nLT * nOT;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * per, t1 = min(ntiles, t0 + per);
  const int ksteps = (K + 7) / 8, nch = (K + 31) / 32;
  double lsum = 0.0;

  if (warp == 0) {
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t j = t - t0;
      const int s = (int)(j % kFwNS);
      const uint32_t n = (uint32_t)(j / kFwNS);
      if (j >= kFwNS) {
        const bool ok = mbar_wait(&rfree[s], (n - 1) & 1u, kWaitNs);
        if (__any_sync(0xffffffffu, !ok) || *s_fail) { if (lane == 0) *s_fail = 1; break; }
      }
      if (lane == 0) {
        const int64_t l0 = (t / nOT) * kLT, o0 = (t % nOT) * kWT;
        unsigned char* st = smem + (size_t)s * kFwStage;
        mbar_expect_tx(&full[s], (uint32_t)(nch * 2 * 8192 + kLT * kWT * 4));
        for (int c = 0; c < nch; ++c) {
          tma_load_2d(st + c * 8192, &tmBh, &full[s], c * 32, (int)o0);
          tma_load_2d(st + 16384 + c * 8192, &tmBl, &full[s], c * 32, (int)o0);
        }
        tma_load_2d(st + kWsBP, &tmX, &full[s], (int)o0, (int)l0);
        tma_load_2d(st + kWsBP + 16384, &tmX, &full[s], (int)o0 + 32, (int)l0);
      }
      __syncwarp();
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idP = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kWT >> 3) << 17) | ((uint32_t)(kLT >> 4) << 24);
      int64_t lt_p = -1;
      uint32_t m = 0;
      bool fail = false;
      for (int64_t t = t0; t < t1; ++t) {
        const int64_t j = t - t0;
        const int s = (int)(j % kFwNS);
        const uint32_t n = (uint32_t)(j / kFwNS);
        const int64_t lt = t / nOT;
        bool ok = true;
        if (lt != lt_p) { ok = mbar_wait(aready, m & 1u, kWaitNs); ++m; }
        if (ok && j >= kFwNS) ok = mbar_wait(&rfree[s], (n - 1) & 1u, kWaitNs);
        if (ok) ok = mbar_wait(&full[s], n & 1u, kWaitNs);
        if (!ok || *s_fail) { fail = true; break; }
        tc_fence_after();
        const uint64_t bh = desc_sw128(smem + (size_t)s * kFwStage), bl = desc_sw128(smem + (size_t)s * kFwStage + 16384);
        const uint32_t d = tmem + 128u * s;
        for (int k8 = 0; k8 < ksteps; ++k8) {
          const uint64_t adv = (uint64_t)((k8 >> 2) * 8192 + (k8 & 3) * 32) >> 4;
          const uint32_t a_hi = tmem + 384u + 8u * k8, a_lo = tmem + 448u + 8u * k8;
          mma_tf32_ts(d, a_hi, bh + adv, idP, k8 > 0 ? 1u : 0u);
          mma_tf32_ts(d + 64u, a_hi, bl + adv, idP, k8 > 0 ? 1u : 0u);
          mma_tf32_ts(d + 64u, a_lo, bh + adv, idP, 1u);
        }
        mma_commit(&pfull[s]);
        lt_p = lt;
      }
      if (fail) *s_fail = 1;
    }
  } else {
    const int quarter = warp & 3, half = (warp - 2) >> 2;
    const int li = 32 * quarter + lane;
    const uint32_t tl = (uint32_t)(32 * quarter) << 16;
    const int ka = 8 * ksteps;
    bool fail = false;
    int64_t cur_lt = -1;
    for (int64_t t = t0; t < t1; ++t) {
      const int64_t j = t - t0;
      const int s = (int)(j % kFwNS);
      const uint32_t n = (uint32_t)(j / kFwNS);
      const int64_t lt = t / nOT;
      const int64_t l0 = lt * kLT, o0 = (t % nOT) * kWT;
      const int no = (int)min((int64_t)kWT, nO - o0);
      const bool lane_ok = l0 + li < nL;
      if (lt != cur_lt) {
        // every P of the previous lane tile is done (this thread waited for it)
        const float* ar = (half == 0 ? Ahi : Alo) + (l0 + li) * 64;
        for (int c0 = 0; c0 < ka; c0 += 16) {
          uint32_t v[16];
#pragma unroll
          for (int u = 0; u < 16; u += 4) {
            const float4 q = lane_ok ? *(const float4*)(ar + c0 + u) : make_float4(0.f, 0.f, 0.f, 0.f);
            v[u] = __float_as_uint(q.x); v[u + 1] = __float_as_uint(q.y);
            v[u + 2] = __float_as_uint(q.z); v[u + 3] = __float_as_uint(q.w);
          }
          tmem_st_x16(tmem + tl + (half == 0 ? 384u : 448u) + (uint32_t)c0, v);
        }
        tmem_wait_st();
        tc_fence_before();
        mbar_arrive(aready);
        cur_lt = lt;
      }
      uint32_t mword = 0xFFFFFFFFu;   // bit u = row o0 + 32 half + u of this lane's column
      if (mask) {
        const int64_t b0 = o0 + 32 * half + xrows * (l0 + li), w = b0 >> 5;
        const uint32_t lo = (lane_ok && w < nwords) ? mask[w] : 0u;
        const uint32_t hi = (lane_ok && w + 1 < nwords) ? mask[w + 1] : 0u;
        mword = (uint32_t)((((uint64_t)hi << 32) | lo) >> (b0 & 31));
      }
      const bool ok1 = mbar_wait(&full[s], n & 1u, kWaitNs);
      const bool ok2 = ok1 && mbar_wait(&pfull[s], n & 1u, kWaitNs);
      if (__any_sync(0xffffffffu, !ok2) || *s_fail) { fail = true; break; }
      tc_fence_after();
      const unsigned char* xrow = smem + (size_t)s * kFwStage + kWsBP + half * 16384 + li * 128;
      const uint32_t pb = tmem + tl + 128u * s;
      float ts = 0.f;
#pragma unroll
      for (int c0 = 0; c0 < 32; c0 += 16) {
        const int cb = 32 * half + c0;
        uint32_t vh[16], vx[16];
        tmem_ld_x16_nw(pb + (uint32_t)cb, vh);
        tmem_ld_x16_nw(pb + 64u + (uint32_t)cb, vx);
        float xv[16];
#pragma unroll
        for (int u = 0; u < 16; u += 4) {
          const int unit = (c0 + u) >> 2;
          const float4 q = *(const float4*)(xrow + ((unit ^ (li & 7)) << 4));
          xv[u] = q.x; xv[u + 1] = q.y; xv[u + 2] = q.z; xv[u + 3] = q.w;
        }
        const uint32_t mb = (mword >> c0) & 0xFFFFu;
        tmem_wait_ld();
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const float p = __uint_as_float(vh[u]) + __uint_as_float(vx[u]);
          const bool keep = lane_ok && (cb + u < no) && ((mb >> u) & 1u);
          const float r = keep ? xv[u] - p : 0.f;
          ts = fmaf(r, r, ts);
        }
      }
      lsum += (double)ts;
      tc_fence_before();
      mbar_arrive(&rfree[s]);
    }
    if (fail) *s_fail = 1;
  }
  // fixed-order block sum of the epilogue threads' partials
#pragma unroll
  for (int o = 16; o; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  tc_fence_before();
  __syncthreads();
  if (warp >= 2 && lane == 0) red[warp - 2] = lsum;
  __syncthreads();
  if (tid == 0) {
    double tot = 0.0;
    for (int w = 0; w < 8; ++w) tot += red[w];
    loss_part[blockIdx.x] = *s_fail ? (double)NAN : tot;
  }
  if (warp == 1) tmem_dealloc(tmem, 512);
}

// out = sum over the CTAs that covered each lane tile (in CTA order) of their
// partial: out[l * K + k] (W) or out[k * nL + l] (Z, transposed)
__global__ void loss_bwd_tc_reduce_kernel(const float* __restrict__ part, int64_t nL, int64_t nOT, int64_t per,
                                          int maxslots, int K, int transposed, float* __restrict__ out) {
  PDL_ENTRY();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nL * K; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t l;
    int k;
    if (transposed) { k = (int)(e / nL); l = e - k * nL; }
    else { l = e / K; k = (int)(e - l * K); }
    const int64_t lt = l / kLT, il = l - lt * kLT;
    const int64_t b0 = lt * nOT / per, b1 = ((lt + 1) * nOT - 1) / per;
    double acc = 0.0;
    for (int64_t b = b0; b <= b1; ++b) {
      const int64_t slot = lt - (b * per) / nOT;
      acc += (double)part[((b * maxslots + slot) * kLT + il) * 64 + k];
    }
    out[e] = (float)acc;
  }
}

struct BwdPlan {
  int grid, maxslots;
  int64_t per;
};
BwdPlan bwd_plan(int64_t nL, int64_t nO, int ow) {
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nLT = (nL + kLT - 1) / kLT, nOT = (nO + ow - 1) / ow, ntiles = nLT * nOT;
  BwdPlan b;
  b.grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, sms));
  b.per = (ntiles + b.grid - 1) / b.grid;
  b.maxslots = (int)((b.per - 1) / nOT + 2);
  return b;
}

}  // namespace

typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                             const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool loss_fwd_tc_supported(int64_t rows, int64_t cols, int K) { return K >= 1 && K <= 64 && rows >= 1 && cols >= 1; }

size_t loss_fwd_tc_split_bytes(int64_t rows, int64_t cols) { return (size_t)(rows + cols) * 64 * 2 * sizeof(float); }

int loss_fwd_tc_blocks(int64_t rows, int64_t cols) {
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t ntiles = ((rows + kLT - 1) / kLT) * ((cols + kLT - 1) / kLT);
  return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, sms));
}

cudaError_t launch_loss_fwd_tc(const float* Lm, const float* Rm, int64_t rows, int64_t cols, int K, const float* X,
                               const uint32_t* mask, float* split, double* loss_part, cudaStream_t s) {
  float* Lhi = split;
  float* Llo = Lhi + rows * 64;
  float* Rhi = Llo + rows * 64;
  float* Rlo = Rhi + cols * 64;
  const unsigned gl = (unsigned)std::max<int64_t>(1, std::min<int64_t>((rows * 64 + 255) / 256, 152 * 8));
  const unsigned gr = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cols * 64 + 255) / 256, 152 * 8));
  launch_k(loss_split_kernel, gl, 256, 0, s, Lm, rows, K, Lhi, Llo);
  launch_k(loss_split_kernel, gr, 256, 0, s, Rm, cols, K, Rhi, Rlo);
  const int vec = (rows % 4 == 0 && ((uintptr_t)X & 15) == 0) ? 1 : 0;
  const int64_t nwords = (rows * cols + 31) / 32;
  EncodeFn enc = (EncodeFn)str_tensor_map_encoder();
  if (vec && enc && rows < INT32_MAX && cols < INT32_MAX && K <= 64) {
    // warp-specialised form: the Lm rows and the X tiles by TMA (same grid, so the
    // same number of partial sums)
    auto map2d = [&](CUtensorMap* tm, const float* base, int64_t inner, int64_t outer, uint32_t bi, uint32_t bo,
                     bool swz) {
      cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
      cuuint64_t gstride[1] = {(cuuint64_t)inner * 4};
      cuuint32_t box[2] = {bi, bo};
      cuuint32_t estr[2] = {1, 1};
      return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstride, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, swz ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap mLh, mLl, mX;
    if (!map2d(&mLh, Lhi, 64, rows, 32, kWT, true) || !map2d(&mLl, Llo, 64, rows, 32, kWT, true) ||
        !map2d(&mX, X, rows, cols, 32, 128, true))
      return cudaErrorInvalidValue;
    const size_t smf = 1024 + (size_t)kFwNS * kFwStage + 128;
    cudaError_t e = cudaFuncSetAttribute(loss_fwd_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
    if (e != cudaSuccess) return e;
    launch_k(loss_fwd_ws_kernel, (unsigned)loss_fwd_tc_blocks(rows, cols), 320, smf, s, mLh, mLl, mX,
             (const float*)Rhi, (const float*)Rlo, cols, rows, K, rows, mask, nwords, loss_part);
    return cudaGetLastError();
  }
  const size_t smem = 1024 + 8 * (size_t)kChunkBytes + (size_t)kLT * kXS * sizeof(float) + 64;
  cudaError_t e = cudaFuncSetAttribute(loss_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  launch_k(loss_fwd_tc_kernel, (unsigned)loss_fwd_tc_blocks(rows, cols), 128, smem, s, (const float*)Rhi,
           (const float*)Rlo, (const float*)Lhi, (const float*)Llo, rows, cols, K, X, mask, nwords, vec, loss_part);
  return cudaGetLastError();
}

static int64_t round4(int64_t v) { return (v + 3) / 4 * 4; }
static int kg_of(int K) { return (K + 15) / 16 * 16; }
static size_t bwd_smem() {
  return 1024 + 8 * (size_t)kChunkBytes + 8 * (size_t)kGChunkMax + (size_t)kLT * 5 * 4 + 4 * (size_t)kLT * 4 + 64;
}

size_t loss_bwd_tc_ws_bytes(int64_t rows, int64_t cols, int K) {
  const int KG = kg_of(K);
  size_t slots = 0;
  for (int ow : {kLT, kWT}) {
    const BwdPlan pw = bwd_plan(cols, rows, ow), pz = bwd_plan(rows, cols, ow);
    slots = std::max(slots, (size_t)std::max(pw.grid * pw.maxslots, pz.grid * pz.maxslots));
  }
  const size_t part = slots * kLT * 64;
  return ((size_t)(rows + cols) * 64 * 2 + (size_t)KG * (round4(rows) + round4(cols)) * 2 + part) * sizeof(float);
}

cudaError_t launch_loss_bwd_tc(const float* Lm, const float* Rm, int64_t rows, int64_t cols, int K, const float* X,
                               const uint32_t* mask, float* ws, float* Zt, float* W, cudaStream_t s) {
  const int KG = kg_of(K);
  const int64_t ldr = round4(rows), ldc = round4(cols);
  float* Lhi = ws;
  float* Llo = Lhi + rows * 64;
  float* Rhi = Llo + rows * 64;
  float* Rlo = Rhi + cols * 64;
  float* LTh = Rlo + cols * 64;
  float* LTl = LTh + KG * ldr;
  float* RTh = LTl + KG * ldr;
  float* RTl = RTh + KG * ldc;
  float* part = RTl + KG * ldc;
  auto g1 = [](int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 8)); };
  launch_k(loss_split_kernel, g1(rows * 64), 256, 0, s, Lm, rows, K, Lhi, Llo);
  launch_k(loss_split_kernel, g1(cols * 64), 256, 0, s, Rm, cols, K, Rhi, Rlo);
  const size_t smem = bwd_smem();
  cudaError_t e = cudaFuncSetAttribute(loss_bwd_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(loss_bwd_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int vec = (rows % 4 == 0 && ((uintptr_t)X & 15) == 0) ? 1 : 0;
  const int64_t nwords = (rows * cols + 31) / 32;
  EncodeFn enc = (EncodeFn)str_tensor_map_encoder();
  if (vec && enc && rows < INT32_MAX && cols < INT32_MAX) {
    // warp-specialised passes: operand rows and G operands by TMA
    auto map2d = [&](CUtensorMap* tm, const float* base, int64_t inner, int64_t outer, int box_outer) {
      cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
      cuuint64_t gstride[1] = {(cuuint64_t)inner * 4};
      cuuint32_t box[2] = {32, (cuuint32_t)box_outer};
      cuuint32_t estr[2] = {1, 1};
      return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), gdim, gstride, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    // X as [cols][rows]: the Z pass reads 128 x 64 boxes unswizzled, the W pass 32 x 128 boxes swizzled
    auto mapx = [&](CUtensorMap* tm, bool zside) {
      cuuint64_t gdim[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
      cuuint64_t gstride[1] = {(cuuint64_t)rows * 4};
      cuuint32_t box[2] = {zside ? 128u : 32u, zside ? 64u : 128u};
      cuuint32_t estr[2] = {1, 1};
      return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(X), gdim, gstride, box, estr,
                 CU_TENSOR_MAP_INTERLEAVE_NONE, zside ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    };
    CUtensorMap mXw, mXz;
    if (!mapx(&mXw, false) || !mapx(&mXz, true)) return cudaErrorInvalidValue;
    launch_k(loss_splitT_kernel, g1(KG * ldr), 256, 0, s, Lm, rows, K, KG, ldr, LTh, LTl);
    launch_k(loss_splitT_kernel, g1(KG * ldc), 256, 0, s, Rm, cols, K, KG, ldc, RTh, RTl);
    CUtensorMap mLh, mLl, mRh, mRl, mLTh, mLTl, mRTh, mRTl;
    if (!map2d(&mLh, Lhi, 64, rows, kWT) || !map2d(&mLl, Llo, 64, rows, kWT) || !map2d(&mRh, Rhi, 64, cols, kWT) ||
        !map2d(&mRl, Rlo, 64, cols, kWT) || !map2d(&mLTh, LTh, ldr, KG, KG) || !map2d(&mLTl, LTl, ldr, KG, KG) ||
        !map2d(&mRTh, RTh, ldc, KG, KG) || !map2d(&mRTl, RTl, ldc, KG, KG))
      return cudaErrorInvalidValue;
    const size_t smw = 1024 + (size_t)kWsNS * (kWsA + kWsG) + 128;
    e = cudaFuncSetAttribute(loss_bwd_ws_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(loss_bwd_ws_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
    if (e != cudaSuccess) return e;
    const BwdPlan pw = bwd_plan(cols, rows, kWT);
    launch_k(loss_bwd_ws_kernel<false>, (unsigned)pw.grid, 320, smw, s, mLh, mLl, mLTh, mLTl, mXw, (const float*)Rhi,
             (const float*)Rlo, cols, rows, K, KG, rows, mask, nwords, pw.maxslots, part);
    launch_k(loss_bwd_tc_reduce_kernel, g1(cols * K), 256, 0, s, (const float*)part, cols, (rows + kWT - 1) / kWT,
             pw.per, pw.maxslots, K, 0, W);
    const BwdPlan pz = bwd_plan(rows, cols, kWT);
    launch_k(loss_bwd_ws_kernel<true>, (unsigned)pz.grid, 320, smw, s, mRh, mRl, mRTh, mRTl, mXz, (const float*)Lhi,
             (const float*)Llo, rows, cols, K, KG, rows, mask, nwords, pz.maxslots, part);
    launch_k(loss_bwd_tc_reduce_kernel, g1(rows * K), 256, 0, s, (const float*)part, rows, (cols + kWT - 1) / kWT,
             pz.per, pz.maxslots, K, 1, Zt);
    return cudaGetLastError();
  }
  // the G operands of the 128 x 128 passes: the other side's tables, transposed
  launch_k(loss_splitT_kernel, g1(KG * ldr), 256, 0, s, Lm, rows, K, KG, ldr, LTh, LTl);
  launch_k(loss_splitT_kernel, g1(KG * ldc), 256, 0, s, Rm, cols, K, KG, ldc, RTh, RTl);
  // W pass: lanes = suffix columns (Rm), o = prefix rows (Lm)
  const BwdPlan pw = bwd_plan(cols, rows, kLT);
  launch_k(loss_bwd_tc_kernel<false>, (unsigned)pw.grid, 256, smem, s, (const float*)Rhi, (const float*)Rlo,
           (const float*)Lhi, (const float*)Llo, (const float*)LTh, (const float*)LTl, cols, rows, ldr, K, KG, rows,
           X, mask, nwords, vec, pw.maxslots, part);
  launch_k(loss_bwd_tc_reduce_kernel, g1(cols * K), 256, 0, s, (const float*)part, cols, (rows + kLT - 1) / kLT,
           pw.per, pw.maxslots, K, 0, W);
  // Z pass: lanes = prefix rows (Lm), o = suffix columns (Rm)
  const BwdPlan pz = bwd_plan(rows, cols, kLT);
  launch_k(loss_bwd_tc_kernel<true>, (unsigned)pz.grid, 256, smem, s, (const float*)Lhi, (const float*)Llo,
           (const float*)Rhi, (const float*)Rlo, (const float*)RTh, (const float*)RTl, rows, cols, ldc, K, KG, rows,
           X, mask, nwords, vec, pz.maxslots, part);
  launch_k(loss_bwd_tc_reduce_kernel, g1(rows * K), 256, 0, s, (const float*)part, rows, (cols + kLT - 1) / kLT,
           pz.per, pz.maxslots, K, 1, Zt);
  return cudaGetLastError();
}
