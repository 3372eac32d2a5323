// Masked TR fit loss, forward, on the 5th-generation tensor cores (FP32 data).
//
// With the modes split into a prefix (rows) and a suffix (columns), every entry
// of the tensor ring is a dot product of two chain-table rows:
//     TR(G)(r, c) = sum_k Lm[r][k] Rm[c][k],   K = R_1 R_{k+1} <= 64,
// so the reconstruction of a 128-column x 128-row tile is one small GEMM
//     P[c][r] = sum_k Rm[c][k] Lm[r][k]
// (M = 128 columns, N = 128 rows, K padded to 8) on tcgen05.mma kind::tf32 with
// the accumulator in TMEM.  FP32 accuracy comes from the 3-term split used by
// the MTTKRP: Rm = Rm_hi + Rm_lo, Lm = Lm_hi + Lm_lo (each rounded to the
// nearest TF32), P = Rm_hi Lm_hi + (Rm_hi Lm_lo + Rm_lo Lm_hi), the two groups
// in separate TMEM columns.  Per tile, the operand tiles are staged, then every
// thread issues asynchronous 16-byte copies of its column's 128 rows of X
// (contiguous: X(r, c) at r + rows c) into a padded shared-memory tile, which
// stay in flight while the MMAs run; the epilogue
// thread that owns column c (its TMEM lane) then reads X from shared memory
// (rows padded to 132 floats: conflict-free 16-byte reads) with its column's
// mask bits, and accumulates sum M (X - P)^2.  One persistent CTA per SM walks
// a contiguous range of tiles (column tile outer, so the Rm operand is staged
// once per column tile).  Loss = 1/2 sum of the per-CTA partial sums (fixed
// order).
//
// A wait that times out (an mbarrier never completing) makes the CTA's partial
// sum NaN, so the loss reads NaN instead of the kernel hanging.
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

}  // namespace

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
  const size_t smem = 1024 + 8 * (size_t)kChunkBytes + (size_t)kLT * kXS * sizeof(float) + 64;
  cudaError_t e = cudaFuncSetAttribute(loss_fwd_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int vec = (rows % 4 == 0 && ((uintptr_t)X & 15) == 0) ? 1 : 0;
  const int64_t nwords = (rows * cols + 31) / 32;
  launch_k(loss_fwd_tc_kernel, (unsigned)loss_fwd_tc_blocks(rows, cols), 128, smem, s, (const float*)Rhi,
           (const float*)Rlo, (const float*)Lhi, (const float*)Llo, rows, cols, K, X, mask, nwords, vec, loss_part);
  return cudaGetLastError();
}
