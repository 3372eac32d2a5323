// Shared device/host definitions for the streaming tensor-ring (STR / rSTR)
// CUDA library.  Everything here is the library's own arithmetic; nothing is
// shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "strtr.h"

#define STR_MAXN 8        // largest tensor order supported
#define STR_MAXR 16       // largest TR-rank supported (R_n R_{n+1} <= 256)
#define STR_MAXRR 256

// ---------------------------------------------------------------------------
// status bits written by device code (atomicOr into the context status word)
// ---------------------------------------------------------------------------
enum : int {
  DEV_ERR_SINGULAR = 1,
  DEV_ERR_NONFINITE = 2,
  DEV_ERR_TIMEOUT = 4,
  DEV_ERR_RANGE = 8,
};

// ---------------------------------------------------------------------------
// complex helpers (interleaved re, im)
// ---------------------------------------------------------------------------
template <typename T> struct cplx { T re, im; };

template <typename T> __device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// a * conj(b)
template <typename T> __device__ __forceinline__ cplx<T> cmulc(cplx<T> a, cplx<T> b) {
  return {a.re * b.re + a.im * b.im, a.im * b.re - a.re * b.im};
}

// ---------------------------------------------------------------------------
// element loads converting the slab's storage type to the compute type
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ T load_as(const double* p) { return (T)(*p); }
template <typename T> __device__ __forceinline__ T load_as(const float* p) { return (T)(*p); }
template <typename T> __device__ __forceinline__ T load_as(const __nv_bfloat16* p) {
  return (T)__bfloat162float(*p);
}

// ---------------------------------------------------------------------------
// Philox4x64-10 counter-based generator (Salmon et al., SC'11).
// key = (seed, 0); counter = (s, k, tau, purpose << 32 | stream); word 0 is used.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t philox_word0(uint64_t c0, uint64_t c1, uint64_t c2,
                                                 uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += W0; k1 += W1; }
    uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
    uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  return c0;
}

__device__ __forceinline__ uint64_t draw_u64(uint64_t seed, uint64_t s, uint64_t k, uint64_t tau,
                                             uint32_t purpose, uint32_t stream) {
  return philox_word0(s, k, tau, ((uint64_t)purpose << 32) | stream, seed, 0ull);
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (cp.async): every thread issues its
// copies back to back so they are all in flight at once, then waits for them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(smem_dst)),
               "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_n() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// programmatic dependent launch.  Every kernel of the library is launched with
// programmatic stream serialisation allowed, so it can be scheduled while the
// previous kernel of its stream is still running, and starts with PDL_ENTRY:
// wait until every prerequisite grid has completed and its writes are visible,
// then allow the next kernel of the stream to be scheduled.  No kernel touches
// global memory before the wait, so the ordering is the stream's own.
// ---------------------------------------------------------------------------
#define PDL_ENTRY()                                          \
  do {                                                       \
    asm volatile("griddepcontrol.wait;" ::: "memory");       \
    asm volatile("griddepcontrol.launch_dependents;" :::);   \
  } while (0)

bool str_pdl_enabled();
// A stream that waited on an event since its last kernel launches its next
// kernel without programmatic serialisation, so the event dependency is a plain
// one (programmatic overlap applies only to kernel-to-kernel order).
void str_mark_cross_wait(cudaStream_t s);
bool str_take_cross_wait(cudaStream_t s);

template <typename... KArgs, typename... Args>
static inline cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                   Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  // the legacy default stream keeps its plain serialisation
  const bool waited = str_take_cross_wait(s);
  cfg.numAttrs = (s == nullptr || s == cudaStreamLegacy || !str_pdl_enabled() || waited) ? 0 : 1;
  return cudaLaunchKernelEx(&cfg, kern, ((KArgs)args)...);
}

// ---------------------------------------------------------------------------
// host-side launch checking
// ---------------------------------------------------------------------------
#define STR_CUDA_TRY(expr)                                                   \
  do {                                                                       \
    cudaError_t _e = (expr);                                                 \
    if (_e != cudaSuccess) { str_set_last_cuda_error(_e, #expr, __FILE__, __LINE__); return STR_ERR_CUDA; } \
  } while (0)

void str_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
void str_set_last_error_text(const char* text);

static inline int ceil_div_i(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
