// Masked-loss forward that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code inside a framework whose caching
// allocator owns all device memory (a raw cudaMalloc would bypass its budget
// and can fail once that allocator has taken the free memory), and
// latency-bound loops that cannot afford cudaMalloc's implicit device
// synchronisation.
// For them, tr_masked_loss_fwd_noalloc computes the same value as
// tr_masked_loss_fwd but keeps its scratch (the prefix/suffix product tables
// and the per-block partial sums) in one fixed array in device global memory,
// declared below, instead of memory obtained at run time.
//
// Limits and sharing:
// * The array holds STR_NOALLOC_SCRATCH_BYTES (32 MiB).  Every GPU that loads
//   this library holds that much until the process exits.
// * A call whose tables do not fit returns STR_ERR_SHAPE without launching.
// * Every call shares the one array per device: calls that overlap on the GPU
//   (other streams, other host threads) race and give wrong results.  The
//   array keeps the previous call's contents; every word a call reads it has
//   written earlier in the same call, so nothing needs clearing.
// * The first call on a device looks up the array's device address
//   (cudaGetSymbolAddress, with that device current); make that first call
//   before any stream capture.
#include <mutex>
#include <string>

#include "kernels.cuh"

#define STR_NOALLOC_SCRATCH_BYTES (32ull << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[STR_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device (set-up on first use).
str_status noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    str_set_last_cuda_error(e, "cudaGetDevice", __FILE__, __LINE__);
    return STR_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return STR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      str_set_last_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)", __FILE__, __LINE__);
      return STR_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return STR_OK;
}

size_t round256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" str_status tr_masked_loss_fwd_noalloc(int N, const int64_t* dims, const int* ranks,
                                                 str_dtype dtype, const void* const* cores_dev,
                                                 const void* X_dev, const uint32_t* mask_bits,
                                                 double* loss_dev, void* stream) {
  if (!dims || !ranks || !cores_dev || !X_dev || !loss_dev) return STR_ERR_INVALID_ARG;
  if (dtype != STR_F32 && dtype != STR_F64) return STR_ERR_DTYPE;
  if (N < 3 || N > STR_MAXN) return STR_ERR_SHAPE;
  int R[STR_MAXN + 1];
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1 || ranks[k] < 1 || ranks[k] > STR_MAXR || !cores_dev[k]) return STR_ERR_SHAPE;
    R[k] = ranks[k];
  }
  R[N] = ranks[0];
  const int compute = dtype == STR_F64 ? 2 : 1;
  const size_t es = dtype == STR_F64 ? 8 : 4;
  // a fixed split of the modes: prefix 1..kp, suffix kp+1..N with kp = N/2
  // (tr_masked_loss_fwd may pick another split; the loss agrees to rounding)
  const int kp = N / 2;
  int64_t rows = 1, cols = 1;
  for (int k = 0; k < kp; ++k) rows *= dims[k];
  for (int k = kp; k < N; ++k) cols *= dims[k];
  const int K = R[0] * R[kp];
  // 64 x 64 output blocks (grid x over rows, y over columns), counted in 64 bits
  // and bounded before any byte size is formed from them
  const int64_t gx = (rows + 63) / 64, gy = (cols + 63) / 64;
  const int64_t nb_max = (int64_t)(STR_NOALLOC_SCRATCH_BYTES / (2 * sizeof(double)));
  if (gx > 2147483647LL || gy > 65535 || gx > nb_max / gy) {
    str_set_last_error_text(("tr_masked_loss_fwd_noalloc: " + std::to_string(gx) + " x " + std::to_string(gy) +
                             " blocks of partial sums exceed the fixed scratch array or the grid limits")
                                .c_str());
    return STR_ERR_SHAPE;
  }
  const int64_t nb = gx * gy;
  const size_t off_suffix = round256((size_t)rows * K * es);
  const size_t off_blocks = off_suffix + round256((size_t)cols * K * es);
  const size_t off_sums = off_blocks + round256((size_t)nb * 2 * sizeof(double));
  const size_t need = off_sums + 2 * sizeof(double);
  if (need > STR_NOALLOC_SCRATCH_BYTES) {
    str_set_last_error_text(("tr_masked_loss_fwd_noalloc needs " + std::to_string(need) +
                             " bytes of scratch; the fixed array holds " +
                             std::to_string((unsigned long long)STR_NOALLOC_SCRATCH_BYTES))
                                .c_str());
    return STR_ERR_SHAPE;
  }
  void* base = nullptr;
  str_status st = noalloc_scratch(&base);
  if (st != STR_OK) return st;
  unsigned char* b = (unsigned char*)base;
  void* prefix = b;
  void* suffix = b + off_suffix;
  double* blocks = (double*)(b + off_blocks);
  double* sums = (double*)(b + off_sums);
  cudaStream_t s = (cudaStream_t)stream;
  str_mark_cross_wait(s);   // the caller may have ordered s after other streams
  STR_CUDA_TRY(launch_chain_table(cores_dev, compute, R, N, dims, 0, kp - 1, 0, 0, prefix, s));
  STR_CUDA_TRY(launch_chain_table(cores_dev, compute, R, N, dims, kp, N - 1, 0, 1, suffix, s));
  int64_t nbo = 0;
  STR_CUDA_TRY(launch_recon(prefix, suffix, compute, rows, cols, K, RM_LOSS, X_dev,
                            dtype == STR_F64 ? XT_F64 : XT_F32, mask_bits, nullptr, 0, blocks, &nbo, s));
  STR_CUDA_TRY(launch_sum_blocks(blocks, nbo, 2, sums, 0.5, s));
  STR_CUDA_TRY(cudaMemcpyAsync(loss_dev, sums, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return STR_OK;
}
