// FMA-pipe rate probe: the denominators of the step roofline for work that
// runs on the FP32 or FP64 fused multiply-add pipes (the FP64 solve state and
// the SIMT contractions).  Not part of the method; a measurement utility.
//
// Every thread runs `iters` rounds of eight independent FMA chains
// (a_j <- a_j * b + c), so each SM sub-partition has enough independent
// instructions in flight to keep its pipe busy; the block's chains are summed
// into one output element so the compiler cannot drop them.
#include "kernels.cuh"

namespace {

template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(int64_t iters, T b, T c, T* out) {
  T a0 = (T)threadIdx.x * (T)1e-3, a1 = a0 + (T)1, a2 = a0 + (T)2, a3 = a0 + (T)3;
  T a4 = a0 + (T)4, a5 = a0 + (T)5, a6 = a0 + (T)6, a7 = a0 + (T)7;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      a0 = fma(a0, b, c); a1 = fma(a1, b, c); a2 = fma(a2, b, c); a3 = fma(a3, b, c);
      a4 = fma(a4, b, c); a5 = fma(a5, b, c); a6 = fma(a6, b, c); a7 = fma(a7, b, c);
    }
  }
  __shared__ T red[256];
  red[threadIdx.x] = ((a0 + a1) + (a2 + a3)) + ((a4 + a5) + (a6 + a7));
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

}  // namespace

extern "C" str_status str_fma_probe(str_dtype dtype, int ctas, int64_t iters, void* out, double* flop,
                                    void* stream) {
  if (!out || !flop || ctas < 1 || iters < 1) return STR_ERR_INVALID_ARG;
  if (dtype != STR_F32 && dtype != STR_F64) return STR_ERR_DTYPE;
  cudaStream_t s = (cudaStream_t)stream;
  // per thread and iteration: 4 x 8 FMAs = 64 flop
  *flop = 64.0 * (double)iters * 256.0 * (double)ctas;
  if (dtype == STR_F32)
    fma_probe_kernel<float><<<ctas, 256, 0, s>>>(iters, 0.9999999f, 1e-7f, (float*)out);
  else
    fma_probe_kernel<double><<<ctas, 256, 0, s>>>(iters, 0.9999999999, 1e-12, (double*)out);
  STR_CUDA_TRY(cudaGetLastError());
  return STR_OK;
}
