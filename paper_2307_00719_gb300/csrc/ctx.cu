// Host orchestration of STR (Alg. 4) and rSTR (Alg. 5 with Algs. 7-9) and the
// C ABI declared in strtr.h.
//
// State layout (all FP64 masters, device resident):
//   spatial core n      G64[n][b]  (I_n x R_nR_{n+1}),  b = committed / working buffer
//   temporal core       GT64       (t_capacity x R_N R_1), rows appended per step
//   P_n, Q_n, E_n       double-buffered like the spatial cores
//   rSTR                idxs[k][b] (m int32), p[k][b] (leverage distributions)
// During a step every buffer a mode writes is the working copy; the step ends
// by flipping the committed index of every mode it updated, so a failed step
// (sync mode) leaves the committed state untouched.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <string>
#include <unordered_set>
#include <vector>

#include "kernels.cuh"

static thread_local std::string g_last_error;
static std::atomic<uint64_t> g_next_uid{1};
static uint64_t next_uid() { return g_next_uid.fetch_add(1); }
// streams that waited on an event since their last kernel launch: every mark is
// kept until that stream's next launch takes it (a lost mark would let a kernel
// overlap, through programmatic serialisation, work it must wait for in full)
namespace {
std::mutex g_cross_mu;
std::unordered_set<cudaStream_t> g_cross_wait;
}
void str_mark_cross_wait(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_cross_mu);
  g_cross_wait.insert(s);
}
bool str_take_cross_wait(cudaStream_t s) {
  std::lock_guard<std::mutex> lk(g_cross_mu);
  return g_cross_wait.erase(s) > 0;
}
// cudaStreamWaitEvent that also marks the stream (see str_mark_cross_wait)
static cudaError_t wait_event(cudaStream_t s, cudaEvent_t e) {
  str_mark_cross_wait(s);
  return cudaStreamWaitEvent(s, e, 0);
}
bool str_pdl_enabled() { return true; }

void str_set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  g_last_error = std::string(cudaGetErrorString(e)) + " in " + what + " (" + file + ":" +
                 std::to_string(line) + ")";
}

void str_set_last_error_text(const char* text) { g_last_error = text; }

namespace {

constexpr uint64_t kSaveMagic = 0x31565254534C4953ull;  // save-format tag

struct DevBuf {
  void* p = nullptr;
  size_t cap = 0;
};

}  // namespace

struct str_ctx {
  int dev = 0;
  int N = 0;
  int64_t I[STR_MAXN] = {};      // I_1..I_{N-1}; I[N-1] = current slab t
  int R[STR_MAXN + 1] = {};      // R_1..R_N, R[N] = R_1
  str_options opt{};
  int compute = 2;               // 1 = FP32 slab arithmetic, 2 = FP64
  int64_t t_rows = 0;            // committed temporal rows
  int64_t step = 0;              // tau
  int64_t last_tn = 0;           // temporal size of the last committed slab
  int sticky = 0;                // async-mode failure latched
  int cur[STR_MAXN] = {};        // committed buffer index per mode
  int upd[STR_MAXN] = {};        // modes written in the current step
  int64_t launches = 0;

  double* G64[STR_MAXN][2] = {};
  float* G32[STR_MAXN][2] = {};
  double* P[STR_MAXN][2] = {};
  double* Q[STR_MAXN][2] = {};
  double* E[STR_MAXN][2] = {};
  double* GT64 = nullptr;        // temporal core storage
  float* GT32 = nullptr;
  int32_t* idxs[STR_MAXN][2] = {};
  double* p[STR_MAXN][2] = {};
  int64_t p_cap[STR_MAXN] = {};

  // per-step scratch
  DevBuf partial, gnew64, gnew32, enew, mtmp, qtmp, lfac, invd, ring0, ring1, gs, ws, gram,
      xstage, xmix0, xmix1, gmix[STR_MAXN], sgn[STR_MAXN], tab0, tab1, bsum, sums;
  // tensor-core MTTKRP scratch: split operand, stage-1 result, chain tables, partials,
  // and the slab with its two fastest modes swapped (made once per slab)
  DevBuf tc_bhi, tc_blo, tc_y2[2], tc_ta, tc_tb, tc_part, tc_xt, wg_part;
  const void* tc_xt_src = nullptr;
  // stage-1 reuse: Y_k = X x_k G_k is kept while the slab and core k are unchanged
  const void* y_slab[2] = {nullptr, nullptr};
  const double* y_core[2] = {nullptr, nullptr};
  uint64_t y_ver[2] = {0, 0};
  uint64_t core_ver[STR_MAXN] = {};   // bumped whenever a core is rewritten
  // chain tables of several cores kept within a step (stage 2 of the MTTKRP)
  struct Chain { int k0 = 0, k1 = -1; bool valid = false; uint64_t ver[STR_MAXN] = {}; const void* cores[STR_MAXN] = {}; DevBuf buf; };
  Chain chains[4];
  // captured update graphs, keyed by buffer parity, slab shape and buffer generation
  struct Graph { int parity; int64_t tn; int xtype; uint64_t gen; cudaGraphExec_t exec; int64_t launches; };
  std::vector<Graph> graphs;
  std::vector<std::pair<int64_t, int>> warm;   // slab shapes already run without capture
  uint64_t gen = 0;                            // bumped whenever a scratch buffer is reallocated
  int* d_status = nullptr;
  int* h_status = nullptr;       // pinned
  double* d_pivot = nullptr;
  unsigned* d_fallbacks = nullptr;   // CTAs of refined solves that took the FP64 fallback
  double* h_sums = nullptr;      // pinned (2 doubles)
  std::vector<void*> owned;
  size_t bytes = 0;
  // profiling: pending (class, start, end) event triples and the event pool
  struct Ev { int cls; cudaEvent_t a, b; int strm; };
  std::vector<Ev> pending;
  std::vector<cudaEvent_t> pool;
  int64_t prof_launch[STR_K_CLASSES] = {};
  double prof_ms[STR_K_CLASSES] = {};
  // identity for batch-graph caching (never reused) and the batch branch stream
  uint64_t uid = 0;
  cudaStream_t bstream = nullptr;
  cudaEvent_t ev_bfork = nullptr, ev_bjoin = nullptr;
  // second stream for the Q-side branch of an update (created on first use)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // third stream: the ring prefix M of the next mode
  cudaStream_t side2 = nullptr;
  cudaEvent_t ev_fork2 = nullptr, ev_join2 = nullptr;
  bool side2_used = false;
  DevBuf mbuf[2];
  DevBuf qf, qlo, fcount, ring2, ring3, levx, chain_scratch, tc_bhi2, tc_blo2;
  bool fcount_dirty = false;     // fcount allocated but not yet cleared on a stream
  const double* qsplit_of = nullptr;   // the Q whose FP32 pair (qf, qlo) is current   // FP32 copy of Q and the last-CTA counter of the fused ring GEMM + factor

  int RR(int n) const { return R[n] * R[n + 1]; }
  int64_t m() const { return opt.m; }
};

namespace {

str_status from_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return STR_OK;
  str_set_last_cuda_error(e, what, __FILE__, __LINE__);
  return e == cudaErrorMemoryAllocation ? STR_ERR_OOM : STR_ERR_CUDA;
}

#define TRY(expr)                                  \
  do {                                             \
    str_status _s = (expr);                        \
    if (_s != STR_OK) return _s;                   \
  } while (0)
cudaEvent_t ev_get(str_ctx* c) {
  if (!c->pool.empty()) { cudaEvent_t e = c->pool.back(); c->pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// launch with optional event timing on the launch stream
#define LCHK(ctx, cls, expr)                                           \
  do {                                                                 \
    str_ctx* _c = (ctx);                                               \
    cudaEvent_t _a = nullptr, _b = nullptr;                            \
    if (_c->opt.profile) { _a = ev_get(_c); cudaEventRecord(_a, s); }  \
    cudaError_t _e = (expr);                                           \
    ++_c->launches;                                                    \
    if (_c->opt.profile) {                                             \
      _b = ev_get(_c);                                                 \
      cudaEventRecord(_b, s);                                          \
      _c->pending.push_back({(cls), _a, _b, s == _c->side ? 1 : s == _c->side2 ? 2 : 0}); \
    }                                                                  \
    if (_e != cudaSuccess) return from_cuda(_e, #expr);                \
  } while (0)
#define LCH(ctx, expr) LCHK(ctx, STR_K_OTHER, expr)
// LCHK on an explicitly named stream
#define LCHKS(ctx, cls, strm, expr) \
  do {                              \
    cudaStream_t s = (strm);        \
    LCHK(ctx, cls, expr);           \
  } while (0)

// New buffers are zeroed before any stream can use them: the zeroing runs on
// the legacy stream, which does not order the non-blocking streams the library
// works on, so it is waited for.  Inside one of the library's own graph captures
// (which a new buffer makes run again directly) the zeroing is deferred to
// zero_pending(), called before that direct run.
thread_local bool g_in_capture = false;
thread_local std::vector<std::pair<void*, size_t>> g_zero_pending;

str_status zero_now(void* p, size_t bytes) {
  if (cudaMemset(p, 0, bytes) != cudaSuccess || cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) {
    cudaGetLastError();
    return STR_ERR_CUDA;
  }
  return STR_OK;
}

str_status zero_pending() {
  str_status st = STR_OK;
  for (auto& z : g_zero_pending)
    if (st == STR_OK) st = zero_now(z.first, z.second);
  g_zero_pending.clear();
  return st;
}

str_status dalloc(str_ctx* c, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) { *p = nullptr; cudaGetLastError(); return from_cuda(e, "cudaMalloc"); }
  c->owned.push_back(*p);
  c->bytes += bytes;
  if (g_in_capture) g_zero_pending.emplace_back(*p, bytes);
  else TRY(zero_now(*p, bytes));
  return STR_OK;
}

template <typename T> str_status dalloc_t(str_ctx* c, T** p, size_t count) {
  void* v = nullptr;
  TRY(dalloc(c, &v, count * sizeof(T)));
  *p = (T*)v;
  return STR_OK;
}

str_status grow(str_ctx* c, DevBuf& b, size_t bytes) {
  if (bytes <= b.cap) return STR_OK;
  if (b.p) {
    auto it = std::find(c->owned.begin(), c->owned.end(), b.p);
    if (it != c->owned.end()) c->owned.erase(it);
    for (auto z = g_zero_pending.begin(); z != g_zero_pending.end();)
      z = z->first == b.p ? g_zero_pending.erase(z) : z + 1;
    cudaFree(b.p);
    c->bytes -= b.cap;
  }
  b.p = nullptr;
  b.cap = 0;
  size_t nb = std::max<size_t>(bytes, 256);
  TRY(dalloc(c, &b.p, nb));
  b.cap = nb;
  c->gen++;
  return STR_OK;
}

int xtype_of(str_dtype d) { return d == STR_BF16 ? XT_BF16 : (d == STR_F32 ? XT_F32 : XT_F64); }
size_t dsize(str_dtype d) { return d == STR_BF16 ? 2 : (d == STR_F32 ? 4 : 8); }

int buf_of(const str_ctx* c, int k) { return c->upd[k] ? 1 - c->cur[k] : c->cur[k]; }

// compute-type pointer of core k as currently seen in the step (k < N-1)
const void* core_c(const str_ctx* c, int k) {
  const int b = buf_of(c, k);
  return c->compute == 2 ? (const void*)c->G64[k][b] : (const void*)c->G32[k][b];
}
const double* E_of(const str_ctx* c, int k) { return c->E[k][buf_of(c, k)]; }

str_status check_status(str_ctx* c, cudaStream_t s, bool* failed) {
  *failed = false;
  STR_CUDA_TRY(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  STR_CUDA_TRY(cudaStreamSynchronize(s));
  const int st = *c->h_status;
  if (st) {
    *failed = true;
    if (st & DEV_ERR_NONFINITE) return STR_ERR_NONFINITE;
    if (st & DEV_ERR_SINGULAR) return STR_ERR_SINGULAR;
    if (st & DEV_ERR_TIMEOUT) return STR_ERR_TIMEOUT;
    return STR_ERR_CUDA;
  }
  return STR_OK;
}

// ---------------------------------------------------------------------------
// building blocks
// ---------------------------------------------------------------------------

// ring product W = E_{k_0} E_{k_1} ... E_{k_{N-2}} (cyclic order n+1..n-1), scattered into
// Qout = base + (H^{!=n})_<2>  (Alg. 4; Prop. subchain_gram)
str_status ring_Q(str_ctx* c, int n, const double* ENew, const double* base, double* Qout,
                  cudaStream_t s) {
  const int N = c->N;
  int order[STR_MAXN];
  for (int t = 0; t < N - 1; ++t) order[t] = (n + 1 + t) % N;
  auto Eptr = [&](int k) -> const double* { return k == N - 1 ? ENew : E_of(c, k); };
  const int RRmax = STR_MAXRR;
  TRY(grow(c, c->ring0, (size_t)RRmax * RRmax * 8));
  TRY(grow(c, c->ring1, (size_t)RRmax * RRmax * 8));
  const double* A = Eptr(order[0]);
  int Mrows = c->R[order[0]] * c->R[order[0]];
  int Kc = c->R[order[0] + 1] * c->R[order[0] + 1];
  double* bufs[2] = {(double*)c->ring0.p, (double*)c->ring1.p};
  int bi = 0;
  for (int t = 1; t < N - 1; ++t) {
    const int k = order[t];
    const double* B = Eptr(k);
    const int Ncols = c->R[k + 1] * c->R[k + 1];
    const bool last = (t == N - 2);
    if (last) {
      float* qh = nullptr;
      float* ql = nullptr;
      if (c->compute == 1) {
        const int RRn = c->RR(n);
        TRY(grow(c, c->qf, (size_t)RRn * RRn * 4));
        TRY(grow(c, c->qlo, (size_t)RRn * RRn * 4));
        qh = (float*)c->qf.p;
        ql = (float*)c->qlo.p;
      }
      LCHK(c, STR_K_GRAM, launch_gemm64(A, B, Qout, Mrows, Kc, Ncols, c->R[n], c->R[n + 1], base, s, qh, ql));
      c->qsplit_of = qh ? Qout : nullptr;
    } else {
      LCHK(c, STR_K_GRAM, launch_gemm64(A, B, bufs[bi], Mrows, Kc, Ncols, 0, 0, nullptr, s));
      A = bufs[bi];
      bi ^= 1;
      Kc = Ncols;
    }
  }
  return STR_OK;
}

// Q_n split as M_n E_{n-1}: M_n = E_{n+1} ... E_{n-2} (the N-2 factors before the
// last, cyclic) does not involve the core updated just before mode n in a
// sweep, so it can be formed ahead of time.  ring_prefix writes M_n into `out`
// (N >= 4; for N = 3, M_n is E_{n+1} itself and *M points there).
str_status ring_prefix(str_ctx* c, int n, const double* ENew, double* out, const double** M, cudaStream_t s) {
  const int N = c->N;
  auto Eptr = [&](int k) -> const double* { return k == N - 1 ? ENew : E_of(c, k); };
  const int f0 = (n + 1) % N;
  if (N == 3) { *M = Eptr(f0); return STR_OK; }
  // own scratch: runs on the third stream beside ring_Q
  TRY(grow(c, c->ring2, (size_t)STR_MAXRR * STR_MAXRR * 8));
  TRY(grow(c, c->ring3, (size_t)STR_MAXRR * STR_MAXRR * 8));
  const double* A = Eptr(f0);
  const int Mrows = c->R[f0] * c->R[f0];
  int Kc = c->R[f0 + 1] * c->R[f0 + 1];
  double* bufs[2] = {(double*)c->ring2.p, (double*)c->ring3.p};
  int bi = 0;
  for (int t = 1; t < N - 2; ++t) {
    const int k = (n + 1 + t) % N;
    const int Ncols = c->R[k + 1] * c->R[k + 1];
    double* dst = (t == N - 3) ? out : bufs[bi];
    LCHK(c, STR_K_GRAM, launch_gemm64(A, Eptr(k), dst, Mrows, Kc, Ncols, 0, 0, nullptr, s));
    A = dst;
    bi ^= 1;
    Kc = Ncols;
  }
  *M = out;
  return STR_OK;
}

// Q_n = base + perm(M_n E_{n-1})
str_status ring_last(str_ctx* c, int n, const double* M, const double* ENew, const double* base, double* Qout,
                     cudaStream_t s) {
  const int N = c->N;
  const int f0 = (n + 1) % N, kl = (n + N - 1) % N;
  const double* El = kl == N - 1 ? ENew : E_of(c, kl);
  LCHK(c, STR_K_GRAM, launch_gemm64(M, El, Qout, c->R[f0] * c->R[f0], c->R[kl] * c->R[kl],
                                    c->R[kl + 1] * c->R[kl + 1], c->R[n], c->R[n + 1], base, s));
  return STR_OK;
}

// Q_n = base + perm(M_n E_{n-1}) and, in the same kernel, the FP32 sweep
// inverse of Q_n that factor_q would produce (FP32 slab arithmetic only)
str_status ring_last_factor(str_ctx* c, int n, const double* M, const double* ENew, const double* base,
                            double* Qout, cudaStream_t s) {
  const int N = c->N;
  const int f0 = (n + 1) % N, kl = (n + N - 1) % N;
  const double* El = kl == N - 1 ? ENew : E_of(c, kl);
  const int RRn = c->RR(n);
  TRY(grow(c, c->lfac, (size_t)RRn * RRn * 8));
  TRY(grow(c, c->invd, (size_t)RRn * 8));
  TRY(grow(c, c->qf, (size_t)RRn * RRn * 4));
  TRY(grow(c, c->qlo, (size_t)RRn * RRn * 4));
  // the last-CTA counter must start at zero (each launch leaves it at zero again):
  // a new buffer is cleared on the stream that runs the kernel, outside any capture
  // (a buffer grown during a capture makes the capture run again directly)
  const void* fc_old = c->fcount.p;
  TRY(grow(c, c->fcount, 16));
  if (c->fcount.p != fc_old) c->fcount_dirty = true;
  if (c->fcount_dirty) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    STR_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusNone) {
      STR_CUDA_TRY(cudaMemsetAsync(c->fcount.p, 0, 16, s));
      c->fcount_dirty = false;
    }
  }
  LCHK(c, STR_K_FACTOR, launch_gemm64_factor(M, El, Qout, c->R[f0] * c->R[f0], c->R[kl] * c->R[kl],
                                             c->R[kl + 1] * c->R[kl + 1], c->R[n], c->R[n + 1], base,
                                             (float*)c->qf.p, (float*)c->qlo.p, (float*)c->lfac.p,
                                             (unsigned*)c->fcount.p, c->d_status, c->d_pivot, s));
  c->qsplit_of = Qout;
  return STR_OK;
}

// solve out = P Q^{-1} (rows x n) in two parts: factor_q depends on Q only,
// apply_q on the factor and P.  FP32 slab arithmetic: FP32 sweep inverse, then
// one FP64-residual refinement step; FP64: LDL^T and substitution.  Writes FP64
// (and the FP32 shadow).
str_status factor_q(str_ctx* c, const double* Qm, int n, cudaStream_t s) {
  TRY(grow(c, c->lfac, (size_t)n * n * 8));
  TRY(grow(c, c->invd, (size_t)n * 8));
  if (c->compute == 1) {
    LCHK(c, STR_K_FACTOR, launch_factor_mixed(Qm, n, (float*)c->lfac.p, c->d_status, c->d_pivot, s));
  } else {
    LCHK(c, STR_K_FACTOR, launch_chol_factor(Qm, n, (double*)c->lfac.p, (double*)c->invd.p, c->d_status, c->d_pivot, s));
  }
  return STR_OK;
}

str_status apply_q(str_ctx* c, const double* Qm, int n, const double* Pm, int64_t rows, double* out64,
                   float* out32, cudaStream_t s, const PartialSum* ps = nullptr) {
  if (c->compute == 1 && apply_df_supported(n)) {
    // the FP32 pair of Q: from the GEMM that formed Q, else split here
    if (c->qsplit_of != Qm) {
      TRY(grow(c, c->qf, (size_t)n * n * 4));
      TRY(grow(c, c->qlo, (size_t)n * n * 4));
      LCHK(c, STR_K_SOLVE, launch_split_pair(Qm, (int64_t)n * n, (float*)c->qf.p, (float*)c->qlo.p, s));
      c->qsplit_of = Qm;
    }
    LCHK(c, STR_K_SOLVE, launch_apply_df((const float*)c->lfac.p, (const float*)c->qf.p, (const float*)c->qlo.p, n,
                                         Pm, rows, out64, out32, ps && ps->part ? ps : nullptr, c->d_status, s,
                                         Qm, c->d_pivot, c->d_fallbacks));
  } else if (c->compute == 1) {
    LCHK(c, STR_K_SOLVE, launch_apply_mixed((const float*)c->lfac.p, Qm, n, Pm, rows, 1, out64, out32,
                                            ps && ps->part ? ps : nullptr, s));
  } else {
    LCHK(c, STR_K_SOLVE, launch_chol_solve((double*)c->lfac.p, (double*)c->invd.p, n, Pm, rows, out64, out32, nullptr, s));
  }
  return STR_OK;
}

str_status solve_rows(str_ctx* c, const double* Qm, int n, const double* Pm, int64_t rows,
                      double* out64, float* out32, cudaStream_t s) {
  TRY(factor_q(c, Qm, n, s));
  return apply_q(c, Qm, n, Pm, rows, out64, out32, s);
}

// second stream of the update: the Q-side chain (Gram of the last updated core,
// ring product, factorisation) runs beside the MTTKRP; ordered by events, so a
// captured update becomes a graph with two branches per mode
str_status fork_side(str_ctx* c, cudaStream_t s) {
  if (!c->side) {
    // the Q-side chain is the critical path of a mode: highest stream priority
    int lo = 0, hi = 0;
    STR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    STR_CUDA_TRY(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, hi));
    STR_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    STR_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
  }
  STR_CUDA_TRY(cudaEventRecord(c->ev_fork, s));
  STR_CUDA_TRY(wait_event(c->side, c->ev_fork));
  return STR_OK;
}

str_status join_side(str_ctx* c, cudaStream_t s) {
  STR_CUDA_TRY(cudaEventRecord(c->ev_join, c->side));
  STR_CUDA_TRY(wait_event(s, c->ev_join));
  if (c->side2_used) {
    STR_CUDA_TRY(cudaEventRecord(c->ev_join2, c->side2));
    STR_CUDA_TRY(wait_event(s, c->ev_join2));
    c->side2_used = false;
  }
  return STR_OK;
}

// third stream: forms M for the next mode from the side stream's current point
// (or, at the start of a step, the slab transpose from the caller's stream)
str_status fork_side2(str_ctx* c, cudaStream_t from = nullptr) {
  if (!c->side2) {
    int lo = 0, hi = 0;
    STR_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    STR_CUDA_TRY(cudaStreamCreateWithPriority(&c->side2, cudaStreamNonBlocking, hi));
    STR_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_fork2, cudaEventDisableTiming));
    STR_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_join2, cudaEventDisableTiming));
  }
  STR_CUDA_TRY(cudaEventRecord(c->ev_fork2, from ? from : c->side));
  STR_CUDA_TRY(wait_event(c->side2, c->ev_fork2));
  c->side2_used = true;
  return STR_OK;
}

// leverage distribution of a core unfolding G (I x RR):  p_i = l_i / rank  (Lemma lev_est)
str_status leverage(str_ctx* c, const double* G, int64_t I, int Ra, int Rb, double* p_out,
                    cudaStream_t s) {
  const int RR = Ra * Rb;
  if (I <= RR) {
    // full row rank: every leverage score is 1, p is uniform
    LCHK(c, STR_K_SOLVE, launch_fill(p_out, I, 1.0 / (double)I, s));
    return STR_OK;
  }
  TRY(grow(c, c->gram, (size_t)RR * RR * 8));
  TRY(grow(c, c->lfac, (size_t)RR * RR * 8));
  TRY(grow(c, c->invd, (size_t)RR * 8));
  LCHK(c, STR_K_GRAM, launch_core_gram(G, I, Ra, Rb, (double*)c->gram.p, nullptr, s));
  if (c->compute == 1 && apply_df_supported(RR)) {
    // FP32 slab arithmetic: x_i = g_i M^{-1} by the FP32 inverse with one
    // refinement step whose residual is FP64-accurate (pair arithmetic), then
    // l_i = g_i . x_i in FP64
    TRY(grow(c, c->qf, (size_t)RR * RR * 4));
    TRY(grow(c, c->qlo, (size_t)RR * RR * 4));
    TRY(grow(c, c->levx, (size_t)I * RR * 8));
    LCHK(c, STR_K_FACTOR, launch_factor_mixed((double*)c->gram.p, RR, (float*)c->lfac.p, c->d_status, nullptr, s));
    LCHK(c, STR_K_SOLVE, launch_split_pair((double*)c->gram.p, (int64_t)RR * RR, (float*)c->qf.p, (float*)c->qlo.p, s));
    c->qsplit_of = (const double*)c->gram.p;
    LCHK(c, STR_K_SOLVE, launch_apply_df((const float*)c->lfac.p, (const float*)c->qf.p, (const float*)c->qlo.p, RR,
                                         G, I, (double*)c->levx.p, nullptr, nullptr, c->d_status, s,
                                         (const double*)c->gram.p, nullptr, c->d_fallbacks));
    LCHK(c, STR_K_SOLVE, launch_leverage_dot(G, (const double*)c->levx.p, I, RR, p_out, s));
    return STR_OK;
  }
  LCHK(c, STR_K_FACTOR, launch_chol_factor((double*)c->gram.p, RR, (double*)c->lfac.p, (double*)c->invd.p, c->d_status, nullptr, s));
  LCHK(c, STR_K_SOLVE, launch_chol_solve((double*)c->lfac.p, (double*)c->invd.p, RR, G, I, nullptr, nullptr, p_out, s));
  return STR_OK;
}

str_status ensure_p(str_ctx* c, int k, int64_t I) {
  if (I <= c->p_cap[k]) return STR_OK;
  for (int b = 0; b < 2; ++b) {
    double* np = nullptr;
    TRY(dalloc_t(c, &np, (size_t)I));
    c->p[k][b] = np;   // old buffers stay owned until destroy (small)
  }
  c->p_cap[k] = I;
  return STR_OK;
}

// MTTKRP over a slab (dense or sampled) for mode n; result reduced into `out`
// (real: out = base + scale * sum; complex: out complex FP64, base ignored)
struct SlabView {
  const void* X;
  int xtype;
  int64_t dim[STR_MAXN];
};

str_status mttkrp_tc(str_ctx* c, const SlabView& v, int n, const void* const* cores, const double* G64k,
                     const double* base, double* out, cudaStream_t s, bool* used, PartialSum* defer);

// Sampled MTTKRP (rSTR) on the tensor cores: rows of G_S and the weighted,
// split GEMM operand; the gathered fibres; a split-K tcgen05 GEMM; the split
// sum (here or deferred to the solve).  Returns without work (used = false)
// when the slab type or sizes do not suit the tensor-core path.
str_status mttkrp_sampled_tc(str_ctx* c, const SlabView& v, int n, const void* const* cores, const int32_t* idxs,
                             bool lev, const double* const* pk, double wscale, const double* base, double* out,
                             void* gs, double* ws, cudaStream_t s, bool* used, PartialSum* defer) {
  *used = false;
  if (v.xtype != XT_F32 && v.xtype != XT_BF16) return STR_OK;
  const int RR = c->RR(n);
  const int64_t In = v.dim[n];
  const int64_t m = c->opt.m;
  if (RR > 160 || In < 32 || m < 32) return STR_OK;
  const int Npad = ((RR + 15) / 16) * 16;
  const int Kpad = (int)(((m + 31) / 32) * 32);
  const size_t es = v.xtype == XT_BF16 ? 2 : 4;
  if (!tc_supported(Kpad, v.xtype, nullptr)) return STR_OK;
  MttkrpArgs a;
  a.X = v.X;
  a.xtype = v.xtype;
  a.N = c->N;
  a.n = n;
  for (int k = 0; k < c->N; ++k) { a.dim[k] = v.dim[k]; a.core[k] = cores[k]; }
  for (int k = 0; k <= c->N; ++k) a.R[k] = c->R[k];
  a.compute = 1;
  a.nfib = m;
  a.idxs = idxs;
  a.m = m;
  a.leverage = lev ? 1 : 0;
  if (lev) for (int k = 0; k < c->N; ++k) a.p[k] = pk[k];
  a.wscale = wscale;
  a.gs_out = gs;
  a.ws_out = ws;
  TRY(grow(c, c->tc_bhi, (size_t)Npad * Kpad * 4));
  TRY(grow(c, c->tc_blo, (size_t)Npad * Kpad * 4));
  TRY(grow(c, c->tc_xt, (size_t)In * Kpad * es));
  STR_CUDA_TRY(cudaMemsetAsync(c->tc_bhi.p, 0, (size_t)Npad * Kpad * 4, s));
  STR_CUDA_TRY(cudaMemsetAsync(c->tc_blo.p, 0, (size_t)Npad * Kpad * 4, s));
  LCHK(c, STR_K_SKETCH, launch_sampled_rows(a, Kpad, (float*)c->tc_bhi.p, (float*)c->tc_blo.p, s));
  LCHK(c, STR_K_SKETCH, launch_gather_fibres(a, Kpad, c->tc_xt.p, s));
  c->tc_xt_src = nullptr;   // the buffer no longer holds the transposed slab
  const int mt = (int)((In + 127) / 128);
  const int want = std::max(1, std::min(Kpad / 32, (2 * 152 + mt - 1) / mt));
  const int splits = gemm_tc_splitk_count(Kpad, want);
  TRY(grow(c, c->tc_part, (size_t)splits * In * RR * 4));
  LCHK(c, STR_K_MTTKRP, launch_gemm_tc_splitk(c->tc_xt.p, v.xtype, In, Kpad, (const float*)c->tc_bhi.p,
                                               (const float*)c->tc_blo.p, RR, Npad, splits, (float*)c->tc_part.p,
                                               c->d_status, s));
  // many splits: a separate parallel reduction is cheaper than summing them in the solve
  if (defer && splits <= 16) {
    defer->part = (const float*)c->tc_part.p;
    defer->splits = splits;
    defer->base = base;
    defer->pout = out;
  } else {
    LCHK(c, STR_K_REDUCE, launch_reduce_partials(c->tc_part.p, 1, 0, splits, In * RR, base, 1.0, out, s));
  }
  *used = true;
  return STR_OK;
}

// Sampled complex MTTKRP (KSRFT, FP32 slab arithmetic) on the tensor cores: two
// real split-K GEMMs for Re P and Im P; out = complex FP64 (interleaved).
str_status mttkrp_sampled_tc_cplx(str_ctx* c, const SlabView& v, int n, const void* const* cores, const int32_t* idxs,
                                  double wscale, double* out, void* gs, double* ws, cudaStream_t s, bool* used) {
  *used = false;
  if (v.xtype != XT_C32) return STR_OK;
  const int RR = c->RR(n);
  const int64_t In = v.dim[n];
  const int64_t m = c->opt.m;
  if (RR > 160 || In < 32 || m < 32) return STR_OK;
  const int Npad = ((RR + 15) / 16) * 16;
  const int Kpad = (int)(((m + 31) / 32) * 32);
  const int K2 = 2 * Kpad;
  if (!tc_supported(K2, XT_F32, nullptr)) return STR_OK;
  MttkrpArgs a;
  a.X = v.X;
  a.xtype = v.xtype;
  a.N = c->N;
  a.n = n;
  for (int k = 0; k < c->N; ++k) { a.dim[k] = v.dim[k]; a.core[k] = cores[k]; }
  for (int k = 0; k <= c->N; ++k) a.R[k] = c->R[k];
  a.compute = 1;
  a.cplx = 1;
  a.nfib = m;
  a.idxs = idxs;
  a.m = m;
  a.wscale = wscale;
  a.gs_out = gs;
  a.ws_out = ws;
  const size_t bsz = (size_t)Npad * K2 * 4;
  TRY(grow(c, c->tc_bhi, bsz));
  TRY(grow(c, c->tc_blo, bsz));
  TRY(grow(c, c->tc_bhi2, bsz));
  TRY(grow(c, c->tc_blo2, bsz));
  TRY(grow(c, c->tc_xt, (size_t)In * K2 * 4));
  STR_CUDA_TRY(cudaMemsetAsync(c->tc_bhi.p, 0, bsz, s));
  STR_CUDA_TRY(cudaMemsetAsync(c->tc_blo.p, 0, bsz, s));
  STR_CUDA_TRY(cudaMemsetAsync(c->tc_bhi2.p, 0, bsz, s));
  STR_CUDA_TRY(cudaMemsetAsync(c->tc_blo2.p, 0, bsz, s));
  LCHK(c, STR_K_SKETCH, launch_sampled_rows_cplx(a, Kpad, (float*)c->tc_bhi.p, (float*)c->tc_blo.p,
                                                 (float*)c->tc_bhi2.p, (float*)c->tc_blo2.p, s));
  LCHK(c, STR_K_SKETCH, launch_gather_fibres_cplx(a, Kpad, (float*)c->tc_xt.p, s));
  c->tc_xt_src = nullptr;   // the buffer no longer holds the transposed slab
  const int mt = (int)((In + 127) / 128);
  const int want = std::max(1, std::min(K2 / 32, (2 * 152 + mt - 1) / mt));
  const int splits = gemm_tc_splitk_count(K2, want);
  const size_t psz = (size_t)splits * In * RR;
  TRY(grow(c, c->tc_part, 2 * psz * 4));
  float* pre = (float*)c->tc_part.p;
  float* pim = pre + psz;
  LCHK(c, STR_K_MTTKRP, launch_gemm_tc_splitk(c->tc_xt.p, XT_F32, In, K2, (const float*)c->tc_bhi.p,
                                               (const float*)c->tc_blo.p, RR, Npad, splits, pre, c->d_status, s));
  LCHK(c, STR_K_MTTKRP, launch_gemm_tc_splitk(c->tc_xt.p, XT_F32, In, K2, (const float*)c->tc_bhi2.p,
                                               (const float*)c->tc_blo2.p, RR, Npad, splits, pim, c->d_status, s));
  LCHK(c, STR_K_REDUCE, launch_reduce_cplx_pair(pre, pim, splits, In * RR, out, s));
  *used = true;
  return STR_OK;
}

str_status mttkrp_into(str_ctx* c, const SlabView& v, int n, const void* const* cores, bool sampled,
                       const int32_t* idxs, bool lev, const double* const* pk, double wscale,
                       bool cplx, const double* base, double* out, void* gs, double* ws,
                       cudaStream_t s, PartialSum* defer = nullptr) {
  if (defer) *defer = PartialSum();
  if (sampled && cplx && c->compute == 1 && c->opt.mttkrp_path == 0) {
    bool used = false;
    TRY(mttkrp_sampled_tc_cplx(c, v, n, cores, idxs, wscale, out, gs, ws, s, &used));
    if (used) return STR_OK;
  }
  if (sampled && !cplx && c->compute == 1 && c->opt.mttkrp_path == 0) {
    bool used = false;
    TRY(mttkrp_sampled_tc(c, v, n, cores, idxs, lev, pk, wscale, base, out, gs, ws, s, &used, defer));
    if (used) return STR_OK;
  }
  if (!sampled && !cplx && c->compute == 1 && c->opt.mttkrp_path == 0) {
    const int kc = (n == 0) ? 1 : 0;
    bool used = false;
    TRY(mttkrp_tc(c, v, n, cores, c->G64[kc][buf_of(c, kc)], base, out, s, &used, defer));
    if (used) return STR_OK;
  }
  MttkrpArgs a;
  a.X = v.X;
  a.xtype = v.xtype;
  a.N = c->N;
  a.n = n;
  for (int k = 0; k < c->N; ++k) { a.dim[k] = v.dim[k]; a.core[k] = cores[k]; }
  for (int k = 0; k <= c->N; ++k) a.R[k] = c->R[k];
  a.compute = c->compute;
  a.cplx = cplx ? 1 : 0;
  if (sampled) {
    a.nfib = c->opt.m;
    a.idxs = idxs;
    a.m = c->opt.m;
    a.leverage = lev ? 1 : 0;
    if (lev) for (int k = 0; k < c->N; ++k) a.p[k] = pk[k];
    a.gs_out = gs;
    a.ws_out = ws;
  } else {
    int64_t J = 1;
    for (int k = 0; k < c->N; ++k) if (k != n) J *= v.dim[k];
    a.nfib = J;
  }
  a.wscale = wscale;
  int64_t per = 0;
  a.splits = mttkrp_plan_splits(a, &per);
  a.fib_per_split = per;
  const int RR = c->RR(n);
  const size_t esize = (c->compute == 2 ? 8 : 4) * (cplx ? 2 : 1);
  TRY(grow(c, c->partial, (size_t)a.splits * v.dim[n] * RR * esize));
  a.partial = c->partial.p;
  LCHK(c, STR_K_MTTKRP, launch_mttkrp(a, s));
  LCHK(c, STR_K_REDUCE, launch_reduce_partials(a.partial, c->compute, a.cplx, a.splits, v.dim[n] * RR, base, 1.0, out, s));
  return STR_OK;
}


// FP32 chain table of cores k0..k1 ([j][R_{k0} x R_{k1+1}], j over i_{k0}.. fastest
// first).  One core is its own table (same layout).  Products of several cores
// are kept for the rest of the step while none of their cores changes.
str_status chain_table_c(str_ctx* c, const void* const* cores, const int64_t* dims, int k0, int k1,
                         const float** out, cudaStream_t s) {
  if (k0 == k1) { *out = (const float*)cores[k0]; return STR_OK; }
  uint64_t ver[STR_MAXN] = {};
  for (int k = k0; k <= k1; ++k) ver[k] = c->core_ver[k];
  for (auto& e : c->chains) {
    if (e.k0 == k0 && e.k1 == k1 && e.valid && std::equal(ver + k0, ver + k1 + 1, e.ver + k0) &&
        std::equal(cores + k0, cores + k1 + 1, e.cores + k0)) {
      *out = (const float*)e.buf.p;
      return STR_OK;
    }
  }
  str_ctx::Chain* slot = nullptr;
  for (auto& e : c->chains) if (!e.valid) { slot = &e; break; }
  if (!slot) slot = &c->chains[0];
  int64_t J = 1;
  for (int j = k0; j <= k1; ++j) J *= dims[j];
  TRY(grow(c, slot->buf, (size_t)J * c->R[k0] * c->R[k1 + 1] * 4));
  if (k1 == k0 + 2 && dims[k0] * dims[k0 + 1] < (1 << 30)) {
    // three cores as two two-core products: (G_k0 G_k0+1) into a scratch table,
    // then that table (a core of I_k0 I_k0+1 slices) times G_k1
    TRY(grow(c, c->chain_scratch, (size_t)dims[k0] * dims[k0 + 1] * c->R[k0] * c->R[k0 + 2] * 4));
    LCHK(c, STR_K_GRAM, launch_chain_table(cores, 1, c->R, c->N, dims, k0, k0 + 1, 0, 0, c->chain_scratch.p, s));
    const void* c2[2] = {c->chain_scratch.p, cores[k1]};
    const int64_t d2[2] = {dims[k0] * dims[k0 + 1], dims[k1]};
    const int r2[3] = {c->R[k0], c->R[k0 + 2], c->R[k1 + 1]};
    LCHK(c, STR_K_GRAM, launch_chain_table(c2, 1, r2, 2, d2, 0, 1, 0, 0, slot->buf.p, s));
  } else {
    LCHK(c, STR_K_GRAM, launch_chain_table(cores, 1, c->R, c->N, dims, k0, k1, 0, 0, slot->buf.p, s));
  }
  slot->k0 = k0;
  slot->k1 = k1;
  slot->valid = true;
  std::copy(ver, ver + STR_MAXN, slot->ver);
  std::copy(cores, cores + c->N, slot->cores);
  *out = (const float*)slot->buf.p;
  return STR_OK;
}

void reset_chains(str_ctx* c) {
  for (auto& e : c->chains) e.valid = false;
}

// Stage 1 of mode 1 (contracted mode 2) needs that mode contiguous: the slab
// with its two fastest modes swapped, made once per slab.  *ok = false when the
// tensor-core path cannot take the slab.
str_status ensure_transposed(str_ctx* c, const SlabView& v, cudaStream_t s, bool* ok) {
  *ok = false;
  if (v.xtype != XT_F32 && v.xtype != XT_BF16) return STR_OK;
  int64_t E = 1;
  for (int j = 0; j < c->N; ++j) E *= v.dim[j];
  const size_t es = v.xtype == XT_BF16 ? 2 : 4;
  if (((size_t)v.dim[1] * es) % 16 != 0) return STR_OK;
  if (c->tc_xt_src != v.X) {
    TRY(grow(c, c->tc_xt, (size_t)E * es));
    LCHK(c, STR_K_OTHER, launch_transpose01(v.X, c->tc_xt.p, v.xtype, (int)v.dim[0], (int)v.dim[1],
                                            E / (v.dim[0] * v.dim[1]), s));
    c->tc_xt_src = v.X;
  }
  *ok = true;
  return STR_OK;
}

// Dense FP32-compute MTTKRP on the tensor cores (two stages, see k_tc.cu).
// cores: FP32 cores as seen in the step (temporal = the slab's rows);
// G64k: FP64 master of the contracted core k.  Returns false (and does
// nothing) when the slab layout does not allow the tensor-core path.
str_status mttkrp_tc(str_ctx* c, const SlabView& v, int n, const void* const* cores, const double* G64k,
                     const double* base, double* out, cudaStream_t s, bool* used, PartialSum* defer) {
  *used = false;
  const int N = c->N;
  const int k = (n == 0) ? 1 : 0;
  int64_t E = 1;
  for (int j = 0; j < N; ++j) E *= v.dim[j];
  const int K = (int)v.dim[k];
  const void* Xa = v.X;
  if (v.xtype != XT_F32 && v.xtype != XT_BF16) return STR_OK;
  if (k == 1) {
    bool ok = false;
    TRY(ensure_transposed(c, v, s, &ok));
    if (!ok) return STR_OK;
    Xa = c->tc_xt.p;
  }
  if (!tc_supported(K, v.xtype, Xa)) return STR_OK;
  const int Rk = c->R[k], Rk1 = c->R[k + 1], RRk = Rk * Rk1;
  const int Npad = ((RRk + 15) / 16) * 16;
  const int Kpad = ((K + 31) / 32) * 32;
  const int64_t M = E / K;
  DevBuf& ybuf = c->tc_y2[k];
  if (!(c->y_slab[k] == v.X && c->y_core[k] == G64k && c->y_ver[k] == c->core_ver[k] && ybuf.p)) {
    TRY(grow(c, c->tc_bhi, (size_t)Npad * Kpad * 4));
    TRY(grow(c, c->tc_blo, (size_t)Npad * Kpad * 4));
    TRY(grow(c, ybuf, (size_t)M * RRk * 4));
    LCHK(c, STR_K_OTHER, launch_prep_b(G64k, K, RRk, Kpad, Npad, (float*)c->tc_bhi.p, (float*)c->tc_blo.p, s));
    LCHK(c, STR_K_MTTKRP, launch_stage1_tc(Xa, v.xtype, M, K, (const float*)c->tc_bhi.p, (const float*)c->tc_blo.p,
                                            Kpad, RRk, Npad, (float*)ybuf.p, c->d_status, s));
    c->y_slab[k] = v.X;
    c->y_core[k] = G64k;
    c->y_ver[k] = c->core_ver[k];
  }
  // stage 2: groups of modes below / above n (mode k excluded), chain tables
  Stage2Args a;
  a.Y = (const float*)ybuf.p;
  a.Rk = Rk; a.Rk1 = Rk1; a.Rn = c->R[n]; a.Rn1 = c->R[n + 1]; a.k = k;
  a.dn = v.dim[n];
  int lo0, lo1, hi0, hi1;   // inclusive mode ranges (lo1 < lo0 = empty)
  if (k == 0) { lo0 = 1; lo1 = n - 1; hi0 = n + 1; hi1 = N - 1; }
  else { lo0 = 1; lo1 = 0; hi0 = 2; hi1 = N - 1; }
  a.Jlo = 1; a.Jhi = 1;
  for (int j = lo0; j <= lo1; ++j) a.Jlo *= v.dim[j];
  for (int j = hi0; j <= hi1; ++j) a.Jhi *= v.dim[j];
  int64_t dims[STR_MAXN];
  for (int j = 0; j < N; ++j) dims[j] = v.dim[j];
  if (k == 0 && hi0 <= hi1) {   // A = G_{n+1} .. G_{N-1}
    TRY(chain_table_c(c, cores, dims, hi0, hi1, &a.TA, s));
  }
  const int b0 = (k == 0) ? lo0 : hi0, b1 = (k == 0) ? lo1 : hi1;
  if (b0 <= b1) {               // B = G_{k+1} .. G_{n-1}
    TRY(chain_table_c(c, cores, dims, b0, b1, &a.TB, s));
  }
  int64_t per = 1;
  a.splits = stage2_plan_splits(a, &per);
  a.per = per;
  const int OUTP = a.Rn * a.Rn1;
  TRY(grow(c, c->tc_part, (size_t)a.splits * a.dn * OUTP * 4));
  a.partial = (float*)c->tc_part.p;
  LCHK(c, STR_K_CONTRACT, launch_stage2(a, s));
  if (defer) {
    defer->part = a.partial;
    defer->splits = a.splits;
    defer->base = base;
    defer->pout = out;
  } else {
    LCHK(c, STR_K_REDUCE, launch_reduce_partials(a.partial, 1, 0, a.splits, a.dn * OUTP, base, 1.0, out, s));
  }
  *used = true;
  return STR_OK;
}

// ---------------------------------------------------------------------------
// slab intake
// ---------------------------------------------------------------------------
str_status take_slab(str_ctx* c, const str_tensor* X, SlabView* v, cudaStream_t s) {
  if (!X || !X->data || !X->dims) return STR_ERR_INVALID_ARG;
  if (X->order != c->N) return STR_ERR_SHAPE;
  if (X->dtype != STR_BF16 && X->dtype != STR_F32 && X->dtype != STR_F64) return STR_ERR_DTYPE;
  int64_t count = 1;
  for (int k = 0; k < c->N; ++k) {
    if (X->dims[k] < 1) return STR_ERR_SHAPE;
    if (k < c->N - 1 && X->dims[k] != c->I[k]) return STR_ERR_SHAPE;
    v->dim[k] = X->dims[k];
    count *= X->dims[k];
  }
  v->xtype = xtype_of(X->dtype);
  c->tc_xt_src = nullptr;
  c->y_slab[0] = c->y_slab[1] = nullptr;
  if (X->on_host) {
    TRY(grow(c, c->xstage, (size_t)count * dsize(X->dtype)));
    STR_CUDA_TRY(cudaMemcpyAsync(c->xstage.p, X->data, (size_t)count * dsize(X->dtype), cudaMemcpyHostToDevice, s));
    v->X = c->xstage.p;
  } else {
    v->X = X->data;
  }
  if (c->opt.check_finite) LCH(c, launch_check_finite(v->X, v->xtype, count, c->d_status, s));
  return STR_OK;
}

// ---------------------------------------------------------------------------
// KSRFT helpers (Definition of the KSRFT; Alg. 9)
// ---------------------------------------------------------------------------
int cplx_type(const str_ctx* c) { return c->compute == 2 ? XT_C64 : XT_C32; }
size_t celem(const str_ctx* c) { return c->compute == 2 ? 16 : 8; }

// signs D_k over dims[k] at step tau (purpose 1)
str_status draw_signs(str_ctx* c, const int64_t* dims, uint64_t tau, cudaStream_t s) {
  for (int k = 0; k < c->N; ++k) {
    TRY(grow(c, c->sgn[k], (size_t)dims[k] * 8));
    LCHK(c, STR_K_SKETCH, launch_signs((double*)c->sgn[k].p, dims[k], c->opt.seed, k + 1, tau, c->opt.stream_id, s));
  }
  return STR_OK;
}

// X_hat = X x_1 F_1 D_1 ... x_N F_N D_N  into xmix (complex compute type); returns pointer
str_status mix_slab(str_ctx* c, const SlabView& v, const void** out, cudaStream_t s) {
  int64_t count = 1;
  for (int k = 0; k < c->N; ++k) count *= v.dim[k];
  TRY(grow(c, c->xmix0, (size_t)count * celem(c)));
  TRY(grow(c, c->xmix1, (size_t)count * celem(c)));
  const void* src = v.X;
  int st = v.xtype;
  void* bufs[2] = {c->xmix0.p, c->xmix1.p};
  int bi = 0;
  for (int k = 0; k < c->N; ++k) {
    LCHK(c, STR_K_DFT, launch_dft_mode(src, st, bufs[bi], c->compute, c->N, v.dim, k, (const double*)c->sgn[k].p, s));
    src = bufs[bi];
    st = cplx_type(c);
    bi ^= 1;
  }
  *out = src;
  return STR_OK;
}

// G_hat_k = G_k x_2 (F_k D_k): DFT along the row index of the unfolding (rows x RR)
str_status mix_core(str_ctx* c, int k, const void* G, int64_t rows, cudaStream_t s) {
  const int RR = c->RR(k);
  TRY(grow(c, c->gmix[k], (size_t)rows * RR * celem(c)));
  const int64_t dims[2] = {RR, rows};
  LCHK(c, STR_K_DFT, launch_dft_mode(G, c->compute == 2 ? XT_F64 : XT_F32, c->gmix[k].p, c->compute, 2, dims, 1,
                         (const double*)c->sgn[k].p, s));
  return STR_OK;
}

// ---------------------------------------------------------------------------
// context creation
// ---------------------------------------------------------------------------
str_status validate_shape(int N, const int64_t* dims, const int* ranks) {
  if (N < 3 || N > STR_MAXN) return STR_ERR_SHAPE;
  if (!dims || !ranks) return STR_ERR_INVALID_ARG;
  for (int k = 0; k < N; ++k) {
    if (ranks[k] < 1 || ranks[k] > STR_MAXR) return STR_ERR_SHAPE;
    if (k < N - 1 && dims[k] < 1) return STR_ERR_SHAPE;
  }
  for (int k = 0; k < N; ++k)
    if (ranks[k] * ranks[(k + 1) % N] > 160) return STR_ERR_SHAPE;
  return STR_OK;
}

str_status ctx_create(str_ctx** out, int N, const int64_t* dims, const int* ranks,
                      const str_options* opt, int64_t t_init) {
  str_options o;
  str_default_options(&o);
  if (opt) o = *opt;
  if (o.compute != STR_F32 && o.compute != STR_F64) return STR_ERR_DTYPE;
  if (o.sweeps < 1 || o.t_capacity < 1 || t_init < 1 || t_init > o.t_capacity) return STR_ERR_INVALID_ARG;
  if (o.sketch != STR_SKETCH_NONE && (o.sketch < 0 || o.sketch > 2 || o.m < 1)) return STR_ERR_INVALID_ARG;
  TRY(validate_shape(N, dims, ranks));
  str_ctx* c = new str_ctx();
  c->uid = next_uid();
  cudaGetDevice(&c->dev);
  c->N = N;
  for (int k = 0; k < N - 1; ++k) c->I[k] = dims[k];
  c->I[N - 1] = t_init;
  for (int k = 0; k < N; ++k) c->R[k] = ranks[k];
  c->R[N] = ranks[0];
  c->opt = o;
  c->compute = o.compute == STR_F64 ? 2 : 1;
  c->t_rows = t_init;
  str_status st = STR_OK;
  auto fail = [&](str_status e) { str_destroy(c); return e; };
  for (int k = 0; k < N - 1; ++k) {
    const int RR = c->RR(k);
    for (int b = 0; b < 2; ++b) {
      if ((st = dalloc_t(c, &c->G64[k][b], (size_t)c->I[k] * RR)) != STR_OK) return fail(st);
      if (c->compute == 1 && (st = dalloc_t(c, &c->G32[k][b], (size_t)c->I[k] * RR)) != STR_OK) return fail(st);
      if ((st = dalloc_t(c, &c->P[k][b], (size_t)c->I[k] * RR)) != STR_OK) return fail(st);
      if ((st = dalloc_t(c, &c->Q[k][b], (size_t)RR * RR)) != STR_OK) return fail(st);
      if ((st = dalloc_t(c, &c->E[k][b], (size_t)RR * RR)) != STR_OK) return fail(st);
    }
  }
  const int RRN = c->RR(N - 1);
  if ((st = dalloc_t(c, &c->GT64, (size_t)o.t_capacity * RRN)) != STR_OK) return fail(st);
  if (c->compute == 1 && (st = dalloc_t(c, &c->GT32, (size_t)o.t_capacity * RRN)) != STR_OK) return fail(st);
  if (o.sketch != STR_SKETCH_NONE) {
    for (int k = 0; k < N; ++k)
      for (int b = 0; b < 2; ++b)
        if ((st = dalloc_t(c, &c->idxs[k][b], (size_t)o.m)) != STR_OK) return fail(st);
  }
  if ((st = dalloc_t(c, &c->d_status, 1)) != STR_OK) return fail(st);
  if ((st = dalloc_t(c, &c->d_pivot, 1)) != STR_OK) return fail(st);
  if ((st = dalloc_t(c, &c->d_fallbacks, 1)) != STR_OK) return fail(st);
  if (cudaMallocHost(&c->h_status, sizeof(int)) != cudaSuccess) return fail(STR_ERR_OOM);
  if (cudaMallocHost(&c->h_sums, 4 * sizeof(double)) != cudaSuccess) return fail(STR_ERR_OOM);
  *c->h_status = 0;
  // dalloc zeroes on the legacy stream, which does not order the non-blocking
  // streams the updates run on: finish the zeroing before any of them starts
  if (cudaDeviceSynchronize() != cudaSuccess) return fail(STR_ERR_CUDA);
  *out = c;
  return STR_OK;
}

// upload host FP64 cores and derive shadows and Gram transfer matrices
str_status upload_cores(str_ctx* c, const double* const* cores, cudaStream_t s) {
  const int N = c->N;
  for (int k = 0; k < N; ++k) {
    const int64_t rows = (k == N - 1) ? c->t_rows : c->I[k];
    const int RR = c->RR(k);
    double* dst = (k == N - 1) ? c->GT64 : c->G64[k][c->cur[k]];
    STR_CUDA_TRY(cudaMemcpyAsync(dst, cores[k], (size_t)rows * RR * 8, cudaMemcpyHostToDevice, s));
    if (c->compute == 1) {
      float* d32 = (k == N - 1) ? c->GT32 : c->G32[k][c->cur[k]];
      LCH(c, launch_convert(dst, XT_F64, d32, XT_F32, rows * RR, s));
    }
    if (k < N - 1) LCHK(c, STR_K_GRAM, launch_core_gram(dst, rows, c->R[k], c->R[k + 1], nullptr, c->E[k][c->cur[k]], s));
    c->core_ver[k]++;
  }
  return STR_OK;
}

const void* temporal_rows_c(const str_ctx* c, int64_t t0) {
  const int RRN = c->RR(c->N - 1);
  return c->compute == 2 ? (const void*)(c->GT64 + t0 * RRN) : (const void*)(c->GT32 + t0 * RRN);
}

double sketch_wscale(const str_ctx* c, int n, const int64_t* dims) {
  if (!c->opt.rescale) return 1.0;
  if (c->opt.sketch == STR_SKETCH_LEVERAGE) return 1.0 / (double)c->opt.m;
  double J = 1.0;
  for (int k = 0; k < c->N; ++k) if (k != n) J *= (double)dims[k];
  return J / (double)c->opt.m;
}

// rSTR initialisation stage (Algs. 7-9): draws at tau = 0, sketched P_n, Q_n
str_status rstr_init_state(str_ctx* c, const SlabView& v, cudaStream_t s) {
  c->qsplit_of = nullptr;
  const int N = c->N;
  const int64_t m = c->opt.m;
  const bool lev = c->opt.sketch == STR_SKETCH_LEVERAGE && c->opt.rescale;
  const bool levdraw = c->opt.sketch == STR_SKETCH_LEVERAGE;
  const bool ks = c->opt.sketch == STR_SKETCH_KSRFT;
  const int cmax = *std::max_element(c->R, c->R + N);
  (void)cmax;
  for (int k = 0; k < N; ++k) {
    const int64_t Ik = v.dim[k];
    if (levdraw) {
      TRY(ensure_p(c, k, Ik));
      const double* G = (k == N - 1) ? c->GT64 : c->G64[k][c->cur[k]];
      TRY(leverage(c, G, Ik, c->R[k], c->R[k + 1], c->p[k][c->cur[k]], s));
    }
    LCHK(c, STR_K_SKETCH, launch_draw_indices(c->idxs[k][c->cur[k]], m, Ik, c->opt.seed, k + 1, 0, c->opt.stream_id,
                               levdraw ? c->p[k][c->cur[k]] : nullptr, s));
  }
  const void* cores[STR_MAXN];
  const void* src = v.X;
  SlabView sv = v;
  if (ks) {
    TRY(draw_signs(c, v.dim, 0, s));
    TRY(mix_slab(c, v, &src, s));
    sv.X = src;
    sv.xtype = cplx_type(c);
    for (int k = 0; k < N; ++k) {
      const void* G = (k == N - 1) ? temporal_rows_c(c, 0) : core_c(c, k);
      TRY(mix_core(c, k, G, v.dim[k], s));
      cores[k] = c->gmix[k].p;
    }
  } else {
    for (int k = 0; k < N - 1; ++k) cores[k] = core_c(c, k);
    cores[N - 1] = temporal_rows_c(c, 0);
  }
  int RRmax = 0;
  for (int k = 0; k < N; ++k) RRmax = std::max(RRmax, c->RR(k));
  TRY(grow(c, c->gs, (size_t)m * RRmax * celem(c)));
  TRY(grow(c, c->wg_part, (size_t)64 * RRmax * RRmax * 8));
  TRY(grow(c, c->ws, (size_t)m * 8));
  int64_t Imax = 0;
  for (int k = 0; k < N; ++k) Imax = std::max(Imax, v.dim[k]);
  TRY(grow(c, c->mtmp, (size_t)Imax * RRmax * 16));
  const int32_t* idx0 = nullptr;
  TRY(grow(c, c->sums, (size_t)N * m * sizeof(int32_t)));
  // gather the per-mode index columns into one [k][m] array
  int32_t* idxcat = (int32_t*)c->sums.p;
  for (int k = 0; k < N; ++k)
    STR_CUDA_TRY(cudaMemcpyAsync(idxcat + (size_t)k * m, c->idxs[k][c->cur[k]], m * 4, cudaMemcpyDeviceToDevice, s));
  idx0 = idxcat;
  const double* pk[STR_MAXN] = {};
  for (int k = 0; k < N; ++k) pk[k] = c->p[k][c->cur[k]];
  for (int n = 0; n < N - 1; ++n) {
    const int RR = c->RR(n);
    double* Pn = c->P[n][c->cur[n]];
    double* Qn = c->Q[n][c->cur[n]];
    const double ws = sketch_wscale(c, n, v.dim);
    if (ks) {
      TRY(mttkrp_into(c, sv, n, cores, true, idx0, false, pk, ws, true, nullptr, (double*)c->mtmp.p, c->gs.p, (double*)c->ws.p, s));
      LCHK(c, STR_K_DFT, launch_unmix_rows((double*)c->mtmp.p, v.dim[n], RR, (const double*)c->sgn[n].p, nullptr, Pn, s));
    } else {
      TRY(mttkrp_into(c, sv, n, cores, true, idx0, lev, pk, ws, false, nullptr, Pn, c->gs.p, (double*)c->ws.p, s));
    }
    LCHK(c, STR_K_SKETCH, launch_weighted_gram(c->gs.p, c->compute, ks ? 1 : 0, (double*)c->ws.p, m, RR, nullptr, Qn, (double*)c->wg_part.p, s));
  }
  return STR_OK;
}

// exact initialisation (Alg. 4): P_n = X0_[n] G^{!=n}_[2], Q_n = ring with Z_N of G_N^init
str_status str_init_state(str_ctx* c, const SlabView& v, cudaStream_t s) {
  c->qsplit_of = nullptr;
  const int N = c->N;
  const int RRN = c->RR(N - 1);
  TRY(grow(c, c->enew, (size_t)RRN * RRN * 8));
  LCHK(c, STR_K_GRAM, launch_core_gram(c->GT64, c->t_rows, c->R[N - 1], c->R[N], nullptr, (double*)c->enew.p, s));
  const void* cores[STR_MAXN];
  for (int k = 0; k < N - 1; ++k) cores[k] = core_c(c, k);
  cores[N - 1] = temporal_rows_c(c, 0);
  reset_chains(c);
  for (int n = 0; n < N - 1; ++n) {
    TRY(mttkrp_into(c, v, n, cores, false, nullptr, false, nullptr, 1.0, false, nullptr, c->P[n][c->cur[n]], nullptr, nullptr, s));
    TRY(ring_Q(c, n, (double*)c->enew.p, nullptr, c->Q[n][c->cur[n]], s));
  }
  return STR_OK;
}

str_status finish_step(str_ctx* c, cudaStream_t s, int64_t t_new) {
  if (!c->opt.async_status) {
    bool failed = false;
    str_status st = check_status(c, s, &failed);
    if (st != STR_OK) {
      for (int k = 0; k < STR_MAXN; ++k) c->upd[k] = 0;
      STR_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
      return st;
    }
  }
  for (int k = 0; k < STR_MAXN; ++k) {
    if (c->upd[k]) c->cur[k] ^= 1;
    c->upd[k] = 0;
  }
  c->t_rows += t_new;
  c->last_tn = t_new;
  c->step += 1;
  return STR_OK;
}

str_status precheck(str_ctx* c, cudaStream_t s) {
  if (c->sticky) return STR_ERR_STATE;
  if (c->opt.async_status) {
    STR_CUDA_TRY(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    STR_CUDA_TRY(cudaStreamSynchronize(s));
    if (*c->h_status) { c->sticky = 1; return STR_ERR_STATE; }
  }
  return STR_OK;
}

// ---------------------------------------------------------------------------
// STR step (Alg. 4), with sweeps
// ---------------------------------------------------------------------------
str_status str_step(str_ctx* c, const SlabView& v, cudaStream_t s) {
  const int N = c->N;
  const int64_t tn = v.dim[N - 1];
  const int RRN = c->RR(N - 1);
  TRY(grow(c, c->gnew64, (size_t)tn * RRN * 8));
  if (c->compute == 1) TRY(grow(c, c->gnew32, (size_t)tn * RRN * 4));
  TRY(grow(c, c->enew, (size_t)RRN * RRN * 8));
  TRY(grow(c, c->mtmp, (size_t)tn * RRN * 8));
  TRY(grow(c, c->qtmp, (size_t)RRN * RRN * 8));
  double* gn64 = (double*)c->gnew64.p;
  const void* gn_c = c->compute == 2 ? (const void*)gn64 : c->gnew32.p;
  // Per mode the update is two branches joined before the solve:
  //   main: MTTKRP  P_n = X_[n] G^{!=n}_[2]  (+ the committed P_n)
  //   side: Gram E of the core updated just before, ring product Q_n, factor of Q_n
  // then G_n = P_n Q_n^{-1} on the main stream.
  int last = -1;   // core whose Gram matrix is still to be formed (-1: none, N-1: temporal)
  reset_chains(c);
  c->qsplit_of = nullptr;
  // ring prefixes M (Q_n = M_n E_{n-1}): M of the next mode is formed on a third
  // stream while the current mode factors; slot = mode parity
  const int RRmax = STR_MAXRR;
  if (N >= 4) {
    TRY(grow(c, c->mbuf[0], (size_t)RRmax * RRmax * 8));
    TRY(grow(c, c->mbuf[1], (size_t)RRmax * RRmax * 8));
  }
  bool have_M = false;           // M of the mode about to run is already formed
  // the slab transpose for mode 1's stage 1 runs beside the temporal mode
  if (c->compute == 1 && c->opt.mttkrp_path == 0 && c->opt.sweeps > 0) {
    TRY(fork_side2(c, s));
    bool ok = false;
    TRY(ensure_transposed(c, v, c->side2, &ok));
  }
  const int nmodes = c->opt.sweeps * N;
  int step_i = 0;                // position in the mode sequence T, 0, 1, .., N-2, T, ..
  auto mode_at = [&](int i) { return (i % N) == 0 ? N - 1 : (i % N) - 1; };
  // side branch of mode n: Gram of the core updated last, M_n (unless formed
  // ahead), Q_n = base + perm(M_n E_{n-1}), its factor; then M of the next mode
  auto side_branch = [&](int n, const double* base, double* Qout, int RRn) -> str_status {
    cudaStream_t s2 = c->side;
    bool factored = false;
    if (last == N - 1)
      LCHKS(c, STR_K_GRAM, s2, launch_core_gram(gn64, tn, c->R[N - 1], c->R[N], nullptr, (double*)c->enew.p, s2));
    else if (last >= 0)
      LCHKS(c, STR_K_GRAM, s2, launch_core_gram(c->G64[last][1 - c->cur[last]], c->I[last], c->R[last],
                                                c->R[last + 1], nullptr, c->E[last][1 - c->cur[last]], s2));
    const double* enew = (const double*)c->enew.p;
    const double* ENew = (n == N - 1) ? nullptr : enew;
    const bool full_ring = N == 3 || (n == N - 1 && last < 0);
    // M of this mode (if not formed ahead), slot = position parity
    const double* M = nullptr;
    if (!full_ring) {
      if (!have_M) TRY(ring_prefix(c, n, ENew, (double*)c->mbuf[step_i & 1].p, &M, s2));
      else M = (const double*)c->mbuf[step_i & 1].p;
    }
    have_M = false;
    if (N >= 4 && step_i + 1 < nmodes) {
      // M of the next mode on the third stream: it needs every E but the one of
      // the core updated in this mode, all formed by now
      const int nx = mode_at(step_i + 1);
      TRY(fork_side2(c));
      const double* Mx = nullptr;
      TRY(ring_prefix(c, nx, enew, (double*)c->mbuf[(step_i + 1) & 1].p, &Mx, c->side2));
      have_M = true;
    }
    if (full_ring) {
      // first temporal mode of the step (E_new of this step not formed yet) or N = 3
      TRY(ring_Q(c, n, ENew, base, Qout, s2));
    } else if (c->compute == 1) {
      TRY(ring_last_factor(c, n, M, enew, base, Qout, s2));
      factored = true;
    } else {
      TRY(ring_last(c, n, M, enew, base, Qout, s2));
    }
    if (!factored) TRY(factor_q(c, Qout, RRn, s2));
    return STR_OK;
  };
  for (int sw = 0; sw < c->opt.sweeps; ++sw) {
    // temporal mode: H^{!=N} ring, M_N = X_[N] G^{!=N}_[2], G_N^new = M_N H^{-1}
    const void* cores[STR_MAXN];
    for (int k = 0; k < N - 1; ++k) cores[k] = core_c(c, k);
    cores[N - 1] = nullptr;
    TRY(fork_side(c, s));
    TRY(side_branch(N - 1, nullptr, (double*)c->qtmp.p, RRN));
    PartialSum ps;
    TRY(mttkrp_into(c, v, N - 1, cores, false, nullptr, false, nullptr, 1.0, false, nullptr, (double*)c->mtmp.p, nullptr, nullptr, s, &ps));
    TRY(join_side(c, s));
    TRY(apply_q(c, (double*)c->qtmp.p, RRN, (double*)c->mtmp.p, tn, gn64,
                c->compute == 1 ? (float*)c->gnew32.p : nullptr, s, &ps));
    c->core_ver[N - 1]++;
    last = N - 1;
    ++step_i;
    // spatial modes in order (Gauss-Seidel)
    for (int n = 0; n < N - 1; ++n) {
      const int RR = c->RR(n);
      const int w = 1 - c->cur[n];
      for (int k = 0; k < N - 1; ++k) cores[k] = core_c(c, k);
      cores[N - 1] = gn_c;
      TRY(fork_side(c, s));
      TRY(side_branch(n, c->Q[n][c->cur[n]], c->Q[n][w], RR));
      TRY(mttkrp_into(c, v, n, cores, false, nullptr, false, nullptr, 1.0, false, c->P[n][c->cur[n]], c->P[n][w], nullptr, nullptr, s, &ps));
      TRY(join_side(c, s));
      TRY(apply_q(c, c->Q[n][w], RR, c->P[n][w], c->I[n], c->G64[n][w],
                  c->compute == 1 ? c->G32[n][w] : nullptr, s, &ps));
      c->upd[n] = 1;
      c->core_ver[n]++;
      last = n;
      ++step_i;
    }
  }
  // Gram matrix of the last core updated (kept with the committed state)
  if (last >= 0 && last < N - 1)
    LCHK(c, STR_K_GRAM, launch_core_gram(c->G64[last][1 - c->cur[last]], c->I[last], c->R[last], c->R[last + 1],
                                         nullptr, c->E[last][1 - c->cur[last]], s));
  return STR_OK;
}

// append the step's new temporal rows after the committed ones (Alg. 4)
str_status append_rows(str_ctx* c, int64_t tn, cudaStream_t s) {
  const int RRN = c->RR(c->N - 1);
  STR_CUDA_TRY(cudaMemcpyAsync(c->GT64 + c->t_rows * RRN, c->gnew64.p, (size_t)tn * RRN * 8, cudaMemcpyDeviceToDevice, s));
  if (c->compute == 1)
    STR_CUDA_TRY(cudaMemcpyAsync(c->GT32 + c->t_rows * RRN, c->gnew32.p, (size_t)tn * RRN * 4, cudaMemcpyDeviceToDevice, s));
  return STR_OK;
}

// str_step through a captured CUDA graph: the slab is staged at a fixed address
// (c->xstage); the first run of a shape is plain, the next one per buffer parity
// is captured, later ones replay.  Every launch of str_step is device work on
// `s`, so the captured graph repeats exactly what a plain run would enqueue.
str_status str_step_graph(str_ctx* c, SlabView& v, int64_t count, size_t es, cudaStream_t s) {
  if (v.X != c->xstage.p) {
    TRY(grow(c, c->xstage, (size_t)count * es));
    STR_CUDA_TRY(cudaMemcpyAsync(c->xstage.p, v.X, (size_t)count * es, cudaMemcpyDeviceToDevice, s));
    v.X = c->xstage.p;
  }
  const int64_t tn = v.dim[c->N - 1];
  const int parity = c->cur[0];
  for (auto& g : c->graphs) {
    if (g.parity == parity && g.tn == tn && g.xtype == v.xtype && g.gen == c->gen) {
      STR_CUDA_TRY(cudaGraphLaunch(g.exec, s));
      for (int k = 0; k < c->N - 1; ++k) { c->upd[k] = 1; c->core_ver[k]++; }
      c->launches = g.launches;
      return STR_OK;
    }
  }
  const std::pair<int64_t, int> shape(tn, v.xtype);
  const bool is_warm = std::find(c->warm.begin(), c->warm.end(), shape) != c->warm.end();
  if (!is_warm) {
    TRY(str_step(c, v, s));
    c->warm.push_back(shape);
    return STR_OK;
  }
  const uint64_t gen0 = c->gen;
  STR_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  g_in_capture = true;
  str_status st = str_step(c, v, s);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  g_in_capture = false;
  {
    const str_status zs = zero_pending();
    if (st == STR_OK) st = zs;
  }
  if (st != STR_OK) { if (graph) cudaGraphDestroy(graph); return st; }
  if (ce != cudaSuccess || c->gen != gen0) {
    // nothing recorded was executed: forget the capture's host-side bookkeeping
    // and run the step directly
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    for (int k = 0; k < STR_MAXN; ++k) c->upd[k] = 0;
    c->y_slab[0] = c->y_slab[1] = nullptr;
    c->tc_xt_src = nullptr;
    c->launches = 0;
    return str_step(c, v, s);
  }
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) return from_cuda(ce, "cudaGraphInstantiate");
  c->graphs.push_back({parity, tn, v.xtype, c->gen, exec, c->launches});
  STR_CUDA_TRY(cudaGraphLaunch(exec, s));
  return STR_OK;
}

// ---------------------------------------------------------------------------
// rSTR step (Alg. 5; schedules of Algs. 7, 8, 9)
// ---------------------------------------------------------------------------
str_status rstr_step(str_ctx* c, const SlabView& v, cudaStream_t s) {
  c->qsplit_of = nullptr;
  const int N = c->N;
  const int64_t m = c->opt.m;
  const int64_t tn = v.dim[N - 1];
  const uint64_t tau = (uint64_t)c->step + 1;
  const bool levdraw = c->opt.sketch == STR_SKETCH_LEVERAGE;
  const bool lev = levdraw && c->opt.rescale;
  const bool ks = c->opt.sketch == STR_SKETCH_KSRFT;
  const int RRN = c->RR(N - 1);
  int RRmax = 0;
  int64_t Imax = tn;
  for (int k = 0; k < N; ++k) RRmax = std::max(RRmax, c->RR(k));
  for (int k = 0; k < N - 1; ++k) Imax = std::max(Imax, c->I[k]);
  TRY(grow(c, c->gnew64, (size_t)tn * RRN * 8));
  if (c->compute == 1) TRY(grow(c, c->gnew32, (size_t)tn * RRN * 4));
  TRY(grow(c, c->mtmp, (size_t)Imax * RRmax * 16));
  TRY(grow(c, c->qtmp, (size_t)RRN * RRN * 8));
  TRY(grow(c, c->gs, (size_t)m * RRmax * celem(c)));
  TRY(grow(c, c->wg_part, (size_t)64 * RRmax * RRmax * 8));
  TRY(grow(c, c->ws, (size_t)m * 8));
  TRY(grow(c, c->sums, (size_t)N * m * 4));
  double* gn64 = (double*)c->gnew64.p;
  const void* gn_c = c->compute == 2 ? (const void*)gn64 : c->gnew32.p;
  int32_t* idxcat = (int32_t*)c->sums.p;
  auto gather_idx = [&]() -> str_status {
    for (int k = 0; k < N; ++k)
      STR_CUDA_TRY(cudaMemcpyAsync(idxcat + (size_t)k * m, c->idxs[k][buf_of(c, k)], m * 4, cudaMemcpyDeviceToDevice, s));
    return STR_OK;
  };
  auto pks = [&](const double** pk) {
    for (int k = 0; k < N; ++k) pk[k] = c->p[k][buf_of(c, k)];
  };
  SlabView sv = v;
  const void* cores[STR_MAXN];
  if (ks) {
    TRY(draw_signs(c, v.dim, tau, s));
    const void* xm = nullptr;
    TRY(mix_slab(c, v, &xm, s));
    sv.X = xm;
    sv.xtype = cplx_type(c);
    for (int k = 0; k < N - 1; ++k) TRY(mix_core(c, k, core_c(c, k), c->I[k], s));
  }
  // ---- temporal mode ----
  for (int k = 0; k < N - 1; ++k) cores[k] = ks ? c->gmix[k].p : core_c(c, k);
  cores[N - 1] = nullptr;
  TRY(gather_idx());
  const double* pk[STR_MAXN];
  pks(pk);
  const double wsN = sketch_wscale(c, N - 1, v.dim);
  if (ks) {
    TRY(mttkrp_into(c, sv, N - 1, cores, true, idxcat, false, pk, wsN, true, nullptr, (double*)c->mtmp.p, c->gs.p, (double*)c->ws.p, s));
    TRY(grow(c, c->gram, (size_t)tn * RRN * 8 + 64));
    LCHK(c, STR_K_DFT, launch_unmix_rows((double*)c->mtmp.p, tn, RRN, (const double*)c->sgn[N - 1].p, nullptr, (double*)c->gram.p, s));
  } else {
    TRY(mttkrp_into(c, sv, N - 1, cores, true, idxcat, lev, pk, wsN, false, nullptr, (double*)c->mtmp.p, c->gs.p, (double*)c->ws.p, s));
  }
  LCHK(c, STR_K_SKETCH, launch_weighted_gram(c->gs.p, c->compute, ks ? 1 : 0, (double*)c->ws.p, m, RRN, nullptr, (double*)c->qtmp.p, (double*)c->wg_part.p, s));
  TRY(solve_rows(c, (double*)c->qtmp.p, RRN, ks ? (double*)c->gram.p : (double*)c->mtmp.p, tn, gn64,
                 c->compute == 1 ? (float*)c->gnew32.p : nullptr, s));
  {
    const int k = N - 1;
    const int w = 1 - c->cur[k];
    if (levdraw) {
      TRY(ensure_p(c, k, tn));
      TRY(leverage(c, gn64, tn, c->R[k], c->R[k + 1], c->p[k][w], s));
    }
    LCHK(c, STR_K_SKETCH, launch_draw_indices(c->idxs[k][w], m, tn, c->opt.seed, k + 1, tau, c->opt.stream_id,
                               levdraw ? c->p[k][w] : nullptr, s));
    c->upd[k] = 1;
    if (ks) TRY(mix_core(c, k, gn_c, tn, s));
  }
  // ---- spatial modes ----
  for (int n = 0; n < N - 1; ++n) {
    const int RR = c->RR(n);
    const int w = 1 - c->cur[n];
    for (int k = 0; k < N - 1; ++k) cores[k] = ks ? c->gmix[k].p : core_c(c, k);
    cores[N - 1] = ks ? c->gmix[N - 1].p : gn_c;
    TRY(gather_idx());
    pks(pk);
    const double wsn = sketch_wscale(c, n, v.dim);
    PartialSum psn;   // the sampled MTTKRP's split partials, summed inside the solve
    if (ks) {
      TRY(mttkrp_into(c, sv, n, cores, true, idxcat, false, pk, wsn, true, nullptr, (double*)c->mtmp.p, c->gs.p, (double*)c->ws.p, s));
      LCHK(c, STR_K_DFT, launch_unmix_rows((double*)c->mtmp.p, c->I[n], RR, (const double*)c->sgn[n].p, c->P[n][c->cur[n]], c->P[n][w], s));
    } else {
      TRY(mttkrp_into(c, sv, n, cores, true, idxcat, lev, pk, wsn, false, c->P[n][c->cur[n]], c->P[n][w], c->gs.p, (double*)c->ws.p, s, &psn));
    }
    LCHK(c, STR_K_SKETCH, launch_weighted_gram(c->gs.p, c->compute, ks ? 1 : 0, (double*)c->ws.p, m, RR, c->Q[n][c->cur[n]], c->Q[n][w], (double*)c->wg_part.p, s));
    TRY(factor_q(c, c->Q[n][w], RR, s));
    TRY(apply_q(c, c->Q[n][w], RR, c->P[n][w], c->I[n], c->G64[n][w], c->compute == 1 ? c->G32[n][w] : nullptr, s,
                &psn));
    c->upd[n] = 1;
    c->core_ver[n]++;
    if (levdraw) {
      TRY(ensure_p(c, n, c->I[n]));
      TRY(leverage(c, c->G64[n][w], c->I[n], c->R[n], c->R[n + 1], c->p[n][w], s));
    }
    LCHK(c, STR_K_SKETCH, launch_draw_indices(c->idxs[n][w], m, c->I[n], c->opt.seed, n + 1, tau, c->opt.stream_id,
                               levdraw ? c->p[n][w] : nullptr, s));
    if (ks) TRY(mix_core(c, n, core_c(c, n), c->I[n], s));
    // E_n is kept current for a later exact update on the same context
    LCHK(c, STR_K_GRAM, launch_core_gram(c->G64[n][w], c->I[n], c->R[n], c->R[n + 1], nullptr, c->E[n][w], s));
  }
  STR_CUDA_TRY(cudaMemcpyAsync(c->GT64 + c->t_rows * RRN, gn64, (size_t)tn * RRN * 8, cudaMemcpyDeviceToDevice, s));
  if (c->compute == 1)
    STR_CUDA_TRY(cudaMemcpyAsync(c->GT32 + c->t_rows * RRN, c->gnew32.p, (size_t)tn * RRN * 4, cudaMemcpyDeviceToDevice, s));
  return STR_OK;
}

// prefix/suffix tables and the recon kernel over temporal rows [t0, t0 + t)
str_status recon_common(const str_ctx* cc, int64_t t0, int64_t t, int mode, const void* X, int xtype,
                        void* out, int out_type, double* sums_out, cudaStream_t s) {
  str_ctx* c = const_cast<str_ctx*>(cc);
  const int N = c->N;
  int64_t dims[STR_MAXN];
  for (int k = 0; k < N - 1; ++k) dims[k] = c->I[k];
  dims[N - 1] = t;
  const int kp = N / 2;   // prefix modes 0..kp-1
  int64_t rows = 1, cols = 1;
  for (int k = 0; k < kp; ++k) rows *= dims[k];
  for (int k = kp; k < N; ++k) cols *= dims[k];
  const int K = c->R[0] * c->R[kp];
  const size_t es = c->compute == 2 ? 8 : 4;
  TRY(grow(c, c->tab0, (size_t)rows * K * es));
  TRY(grow(c, c->tab1, (size_t)cols * K * es));
  const void* cores[STR_MAXN];
  for (int k = 0; k < N - 1; ++k) cores[k] = core_c(c, k);
  cores[N - 1] = temporal_rows_c(c, t0);
  LCH(c, launch_chain_table(cores, c->compute, c->R, N, dims, 0, kp - 1, 0, 0, c->tab0.p, s));
  LCH(c, launch_chain_table(cores, c->compute, c->R, N, dims, kp, N - 1, 0, 1, c->tab1.p, s));
  const int64_t nb = recon_blocks(rows, cols);
  if (mode == RM_FIT) TRY(grow(c, c->bsum, (size_t)nb * 16));
  int64_t nbo = 0;
  LCH(c, launch_recon(c->tab0.p, c->tab1.p, c->compute, rows, cols, K, mode, X, xtype, nullptr, out,
                      out_type, (double*)c->bsum.p, &nbo, s));
  if (mode == RM_FIT) LCH(c, launch_sum_blocks((double*)c->bsum.p, nbo, 2, sums_out, 1.0, s));
  return STR_OK;
}

// stateless workspace for the loss calls (grow-only, per process)
std::mutex g_ws_mu;
struct LossWs {
  void* p = nullptr;
  size_t cap = 0;
} g_loss_ws[4];
// recorded on a loss call's stream after its last use of g_loss_ws; the next
// loss call's stream waits on it first, so calls on different streams run
// their workspace use one after another on the GPU
cudaEvent_t g_ws_done = nullptr;
bool g_ws_recorded = false;

// Orders stream s after the previous loss call's use of the workspace (not
// inside a stream capture, where a wait on an event recorded outside it is not
// allowed; the caller orders captured work itself).
str_status ws_acquire(cudaStream_t s, bool* capturing) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  STR_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
  *capturing = cs != cudaStreamCaptureStatusNone;
  if (!g_ws_done) STR_CUDA_TRY(cudaEventCreateWithFlags(&g_ws_done, cudaEventDisableTiming));
  if (g_ws_recorded && !*capturing) STR_CUDA_TRY(wait_event(s, g_ws_done));
  else str_mark_cross_wait(s);   // the caller may have ordered s after other streams
  return STR_OK;
}

str_status ws_release(cudaStream_t s, bool capturing) {
  if (capturing) return STR_OK;
  STR_CUDA_TRY(cudaEventRecord(g_ws_done, s));
  g_ws_recorded = true;
  return STR_OK;
}

// side streams of the loss backward (per device, created on first use): the
// reduced-trace MTTKRPs of the core gradients are independent and run
// concurrently, forked from and joined back into the caller's stream by events
constexpr int kLossSide = 4;
struct LossSide {
  int dev = -1;
  cudaStream_t st[kLossSide] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kLossSide] = {};
};
LossSide g_loss_side[16];

str_status loss_side(LossSide** out) {
  int dev = 0;
  STR_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 16) return STR_ERR_INVALID_ARG;
  LossSide& ls = g_loss_side[dev];
  if (ls.dev != dev) {
    for (int i = 0; i < kLossSide; ++i) {
      STR_CUDA_TRY(cudaStreamCreateWithFlags(&ls.st[i], cudaStreamNonBlocking));
      STR_CUDA_TRY(cudaEventCreateWithFlags(&ls.join[i], cudaEventDisableTiming));
    }
    STR_CUDA_TRY(cudaEventCreateWithFlags(&ls.fork, cudaEventDisableTiming));
    ls.dev = dev;
  }
  *out = &ls;
  return STR_OK;
}

str_status ws_grow(int i, size_t bytes) {
  if (bytes <= g_loss_ws[i].cap) return STR_OK;
  if (g_loss_ws[i].p) cudaFree(g_loss_ws[i].p);
  g_loss_ws[i].p = nullptr;
  g_loss_ws[i].cap = 0;
  cudaError_t e = cudaMalloc(&g_loss_ws[i].p, bytes);
  if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e, "cudaMalloc"); }
  g_loss_ws[i].cap = bytes;
  return STR_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

str_status str_default_options(str_options* o) {
  if (!o) return STR_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->compute = STR_F64;
  o->sweeps = 1;
  o->rescale = 1;
  o->t_capacity = 65536;
  o->init_max_it = 100;
  o->init_tol = 1e-8;
  o->sketch = STR_SKETCH_NONE;
  o->m = 1000;
  o->seed = 0;
  o->stream_id = 0;
  o->check_finite = 0;
  o->async_status = 0;
  o->profile = 0;
  o->mttkrp_path = 0;
  o->graphs = 1;
  return STR_OK;
}

str_status str_init_cores(str_ctx** out, int N, const int64_t* dims, const int* ranks, int64_t t_init,
                          const double* const* cores, const str_tensor* X0, const str_options* opt,
                          void* stream) {
  if (!out || !cores) return STR_ERR_INVALID_ARG;
  *out = nullptr;
  for (int k = 0; k < N && k < STR_MAXN; ++k) if (!cores[k]) return STR_ERR_INVALID_ARG;
  str_ctx* c = nullptr;
  TRY(ctx_create(&c, N, dims, ranks, opt, t_init));
  cudaStream_t s = (cudaStream_t)stream;
  str_mark_cross_wait(s);   // the caller may have ordered s after other streams
  str_status st = upload_cores(c, cores, s);
  if (st == STR_OK && X0) {
    SlabView v;
    st = take_slab(c, X0, &v, s);
    if (st == STR_OK && v.dim[N - 1] != t_init) st = STR_ERR_SHAPE;
    if (st == STR_OK) st = (c->opt.sketch == STR_SKETCH_NONE) ? str_init_state(c, v, s) : rstr_init_state(c, v, s);
  } else if (st == STR_OK && c->opt.sketch != STR_SKETCH_NONE) {
    st = STR_ERR_INVALID_ARG;   // rSTR needs the initial tensor for its sketches
  }
  if (st == STR_OK) {
    bool failed = false;
    st = check_status(c, s, &failed);
  }
  if (st != STR_OK) { str_destroy(c); return st; }
  *out = c;
  return STR_OK;
}

str_status str_init(str_ctx** out, const str_tensor* X0, const int* ranks, const double* const* guess,
                    const str_options* opt, void* stream) {
  if (!out || !X0 || !ranks || !guess || !X0->dims) return STR_ERR_INVALID_ARG;
  *out = nullptr;
  const int N = X0->order;
  if (N < 3 || N > STR_MAXN) return STR_ERR_SHAPE;
  str_options o;
  str_default_options(&o);
  if (opt) o = *opt;
  const int64_t t_init = X0->dims[N - 1];
  str_ctx* c = nullptr;
  TRY(ctx_create(&c, N, X0->dims, ranks, &o, t_init));
  cudaStream_t s = (cudaStream_t)stream;
  str_mark_cross_wait(s);   // the caller may have ordered s after other streams
  str_status st = upload_cores(c, guess, s);
  SlabView v;
  if (st == STR_OK) st = take_slab(c, X0, &v, s);
  // TR-ALS-NE (Alg. 2) on X0: every core, including the temporal one, in turn
  c->qsplit_of = nullptr;
  double prev = -1.0;
  for (int it = 0; st == STR_OK && it < o.init_max_it; ++it) {
    for (int n = 0; n < N && st == STR_OK; ++n) {
      const int RR = c->RR(n);
      const void* cores[STR_MAXN];
      for (int k = 0; k < N - 1; ++k) cores[k] = core_c(c, k);
      cores[N - 1] = temporal_rows_c(c, 0);
      st = grow(c, c->mtmp, (size_t)v.dim[n] * RR * 8);
      if (st == STR_OK) st = grow(c, c->qtmp, (size_t)RR * RR * 8);
      if (st == STR_OK) st = grow(c, c->enew, (size_t)c->RR(N - 1) * c->RR(N - 1) * 8);
      if (st != STR_OK) break;
      // E of the temporal core (rows t_init) for the ring
      if (n < N - 1) {
        ++c->launches;
        launch_core_gram(c->GT64, t_init, c->R[N - 1], c->R[N], nullptr, (double*)c->enew.p, s);
      }
      st = ring_Q(c, n, (double*)c->enew.p, nullptr, (double*)c->qtmp.p, s);
      if (st == STR_OK) st = mttkrp_into(c, v, n, cores, false, nullptr, false, nullptr, 1.0, false, nullptr, (double*)c->mtmp.p, nullptr, nullptr, s);
      if (st != STR_OK) break;
      double* o64 = (n == N - 1) ? c->GT64 : c->G64[n][c->cur[n]];
      float* o32 = (c->compute == 1) ? ((n == N - 1) ? c->GT32 : c->G32[n][c->cur[n]]) : nullptr;
      st = solve_rows(c, (double*)c->qtmp.p, RR, (double*)c->mtmp.p, v.dim[n], o64, o32, s);
      c->core_ver[n]++;
      if (st == STR_OK && n < N - 1)
        st = from_cuda(launch_core_gram(o64, c->I[n], c->R[n], c->R[n + 1], nullptr, c->E[n][c->cur[n]], s), "core_gram");
    }
    if (st != STR_OK) break;
    double err = 0.0;
    st = grow(c, c->sums, 64);
    if (st != STR_OK) break;
    st = recon_common(c, 0, t_init, RM_FIT, v.X, v.xtype, nullptr, 0, (double*)c->sums.p, s);
    if (st != STR_OK) break;
    if (cudaMemcpyAsync(c->h_sums, c->sums.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) { st = STR_ERR_CUDA; break; }
    err = c->h_sums[1] > 0 ? std::sqrt(c->h_sums[0] / c->h_sums[1]) : 0.0;
    if (prev >= 0.0 && std::fabs(prev - err) < o.init_tol) break;
    prev = err;
  }
  if (st == STR_OK) st = (c->opt.sketch == STR_SKETCH_NONE) ? str_init_state(c, v, s) : rstr_init_state(c, v, s);
  if (st == STR_OK) {
    bool failed = false;
    st = check_status(c, s, &failed);
  }
  if (st != STR_OK) { str_destroy(c); return st; }
  *out = c;
  return STR_OK;
}

str_status str_update(str_ctx* c, const str_tensor* X, void* stream) {
  if (!c) return STR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  str_mark_cross_wait(s);   // the caller may have ordered s after other streams
  TRY(precheck(c, s));
  c->launches = 0;
  SlabView v;
  TRY(take_slab(c, X, &v, s));
  const int64_t tn = v.dim[c->N - 1];
  if (c->t_rows + tn > c->opt.t_capacity) return STR_ERR_CAPACITY;
  str_status st;
  // the legacy default stream cannot be captured: plain launches there
  if (c->opt.graphs && !c->opt.profile && s != nullptr && s != cudaStreamLegacy) {
    int64_t count = 1;
    for (int k = 0; k < c->N; ++k) count *= v.dim[k];
    st = str_step_graph(c, v, count, dsize(X->dtype), s);
  } else {
    st = str_step(c, v, s);
  }
  if (st == STR_OK) st = append_rows(c, tn, s);
  if (st != STR_OK) {
    for (int k = 0; k < STR_MAXN; ++k) c->upd[k] = 0;
    return st;
  }
  return finish_step(c, s, tn);
}

str_status rstr_update(str_ctx* c, const str_tensor* X, str_sketch type, int64_t m, uint64_t seed,
                       void* stream) {
  if (!c) return STR_ERR_INVALID_ARG;
  if (c->opt.sketch == STR_SKETCH_NONE || type != c->opt.sketch || m != c->opt.m || seed != c->opt.seed)
    return STR_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  str_mark_cross_wait(s);   // the caller may have ordered s after other streams
  TRY(precheck(c, s));
  c->launches = 0;
  SlabView v;
  TRY(take_slab(c, X, &v, s));
  const int64_t tn = v.dim[c->N - 1];
  if (c->t_rows + tn > c->opt.t_capacity) return STR_ERR_CAPACITY;
  str_status st = rstr_step(c, v, s);
  if (st != STR_OK) {
    for (int k = 0; k < STR_MAXN; ++k) c->upd[k] = 0;
    return st;
  }
  return finish_step(c, s, tn);
}

// ---------------------------------------------------------------------------
// batched updates: one CUDA graph per (contexts, slab shapes, buffer parities,
// buffer generations) whose branches -- one per context, each the two-branch
// update of str_step -- run concurrently
// ---------------------------------------------------------------------------
struct BatchGraph {
  int dev;
  std::vector<uint64_t> uids;
  std::vector<int64_t> tns;
  std::vector<int> xtypes, parity;
  std::vector<uint64_t> gens;
  cudaGraphExec_t exec;
};
std::mutex g_batch_mu;
std::vector<BatchGraph> g_batch;
// batch keys met once (capture happens when a key comes back): a batch whose
// slab shapes change every step runs as plain concurrent branches
std::vector<uint64_t> g_batch_seen;

void forget_batch_graphs(uint64_t uid) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (size_t i = 0; i < g_batch.size();) {
    if (std::find(g_batch[i].uids.begin(), g_batch[i].uids.end(), uid) != g_batch[i].uids.end()) {
      cudaGraphExecDestroy(g_batch[i].exec);
      g_batch.erase(g_batch.begin() + i);
    } else {
      ++i;
    }
  }
}

uint64_t batch_key(str_ctx* const* ctxs, const std::vector<int64_t>& tns, const std::vector<SlabView>& v, int count) {
  uint64_t h = 1469598103934665603ull;   // FNV-1a over the key fields
  auto mix = [&](uint64_t x) {
    for (int b = 0; b < 8; ++b) { h ^= (x >> (8 * b)) & 0xff; h *= 1099511628211ull; }
  };
  for (int i = 0; i < count; ++i) {
    mix(ctxs[i]->uid);
    mix((uint64_t)tns[i]);
    mix((uint64_t)v[i].xtype);
    mix((uint64_t)ctxs[i]->cur[0]);
    mix(ctxs[i]->gen);
  }
  return h;
}

// true when the key was met before; records it otherwise (bounded list)
bool seen_before(uint64_t key) {
  if (std::find(g_batch_seen.begin(), g_batch_seen.end(), key) != g_batch_seen.end()) return true;
  if (g_batch_seen.size() >= 256) g_batch_seen.erase(g_batch_seen.begin());
  g_batch_seen.push_back(key);
  return false;
}

str_status ensure_bstream(str_ctx* c) {
  if (c->bstream) return STR_OK;
  STR_CUDA_TRY(cudaStreamCreateWithFlags(&c->bstream, cudaStreamNonBlocking));
  STR_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_bfork, cudaEventDisableTiming));
  STR_CUDA_TRY(cudaEventCreateWithFlags(&c->ev_bjoin, cudaEventDisableTiming));
  return STR_OK;
}

// every context's step on its own branch stream: all forked from the same point
// of s, all joined back to s after the last one is enqueued (rSTR steps append
// their own rows)
str_status batch_steps(str_ctx* const* ctxs, std::vector<SlabView>& v, int count, cudaStream_t s,
                       bool randomized = false) {
  for (int i = 0; i < count; ++i) STR_CUDA_TRY(cudaEventRecord(ctxs[i]->ev_bfork, s));
  for (int i = 0; i < count; ++i) {
    str_ctx* c = ctxs[i];
    STR_CUDA_TRY(wait_event(c->bstream, c->ev_bfork));
    TRY(randomized ? rstr_step(c, v[i], c->bstream) : str_step(c, v[i], c->bstream));
    STR_CUDA_TRY(cudaEventRecord(c->ev_bjoin, c->bstream));
  }
  for (int i = 0; i < count; ++i) STR_CUDA_TRY(wait_event(s, ctxs[i]->ev_bjoin));
  return STR_OK;
}

// ---------------------------------------------------------------------------
// Work-list batches: order-3 streams with FP32 slab arithmetic and one sweep
// are updated together by one fixed sequence of launches per step, each
// covering every stream (blocks walk a device list of (stream, tile) items).
// Per mode: core Gram, ring product, FP32 sweep inverse, dense MTTKRP (one
// launch per register-block class), split reduction, refined solve.  The
// per-stream arithmetic is that of str_step (same kernel bodies, same split
// plans and reduction orders), so the results equal one str_update per stream
// wherever str_step would take the SIMT MTTKRP.  Job lists are built once per
// batch layout (contexts, slab shapes, buffer parities and generations) and
// the sequence is captured into a CUDA graph when the layout recurs; only the
// slab pointers and the append destinations are uploaded per step.  The
// staging chunk of the MTTKRP and the rows per block of the refined solve are
// chosen per shape signature by timing candidates on the layout's first step
// (neither changes the arithmetic).
// ---------------------------------------------------------------------------
struct WLTune {
  int bk = 32;                   // fibres staged per MTTKRP chunk (upper limit; reduced to fit shared memory)
  int rows_per_block = 4;        // refined-solve rows per block
};

enum WLKind { WL_GRAM, WL_GEMM, WL_SWEEP, WL_MTTKRP, WL_REDUCE, WL_APPLY, WL_REFINE, WL_COPY };

struct WLLaunch {
  WLKind kind;
  size_t jobs = 0, items = 0;    // byte offsets in the arena
  int n = 0;                     // items (or jobs for the sweep)
  int p0 = 0, p1 = 0, p2 = 0;    // Kmax | (cls, xtype, BK) | nmax
  size_t smem = 0;
};

struct WLLayout {
  int dev = 0;
  std::vector<uint64_t> uids;
  std::vector<int64_t> tns;
  std::vector<int> xtypes, parity;
  std::vector<uint64_t> gens;
  WLTune tune;
  char* arena = nullptr;          // device: static jobs and items, then the per-step region
  size_t dyn_off = 0, dyn_bytes = 0, xptr_off = 0, copyjob_off = 0, status_off = 0, statusptr_off = 0;
  std::vector<WLLaunch> launches;
  std::vector<char> dyn;          // host image of the per-step region
  int* h_status = nullptr;        // pinned, one word per context
  cudaGraphExec_t exec = nullptr;
  int runs = 0;
};

std::mutex g_wl_mu;
std::vector<WLLayout*> g_wl;
struct WLTuned { uint64_t sig; WLTune tune; };
std::vector<WLTuned> g_wl_tuned;

void wl_free(WLLayout* L) {
  if (L->exec) cudaGraphExecDestroy(L->exec);
  if (L->arena) cudaFree(L->arena);
  if (L->h_status) cudaFreeHost(L->h_status);
  delete L;
}

void forget_wl_layouts(uint64_t uid) {
  std::lock_guard<std::mutex> lk(g_wl_mu);
  for (size_t i = 0; i < g_wl.size();) {
    if (std::find(g_wl[i]->uids.begin(), g_wl[i]->uids.end(), uid) != g_wl[i]->uids.end()) {
      wl_free(g_wl[i]);
      g_wl.erase(g_wl.begin() + i);
    } else {
      ++i;
    }
  }
}

bool wl_eligible(const str_ctx* c, const SlabView& v) {
  if (c->N != 3 || c->compute != 1 || c->opt.sweeps != 1 || c->opt.profile) return false;
  if (v.xtype != XT_BF16 && v.xtype != XT_F32 && v.xtype != XT_F64) return false;
  for (int k = 0; k < 3; ++k)
    if (c->RR(k) > 160) return false;
  return true;
}

// shape signature of a batch (what the tuned choice depends on)
uint64_t wl_signature(str_ctx* const* ctxs, const std::vector<int64_t>& tns, const std::vector<SlabView>& v,
                      int count) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](uint64_t x) {
    for (int b = 0; b < 8; ++b) { h ^= (x >> (8 * b)) & 0xff; h *= 1099511628211ull; }
  };
  for (int i = 0; i < count; ++i) {
    const str_ctx* c = ctxs[i];
    mix((uint64_t)c->I[0]); mix((uint64_t)c->I[1]); mix((uint64_t)tns[i]); mix((uint64_t)v[i].xtype);
    for (int k = 0; k < 3; ++k) mix((uint64_t)c->R[k]);
  }
  return h;
}

// dense MTTKRP arguments of mode n of a three-way stream, as mttkrp_into forms them
MttkrpArgs wl_mttkrp_args(str_ctx* c, const SlabView& v, int n, const void* const* cores) {
  MttkrpArgs a;
  a.X = v.X;
  a.xtype = v.xtype;
  a.N = 3;
  a.n = n;
  for (int k = 0; k < 3; ++k) { a.dim[k] = v.dim[k]; a.core[k] = cores[k]; }
  for (int k = 0; k <= 3; ++k) a.R[k] = c->R[k];
  a.compute = 1;
  int64_t J = 1;
  for (int k = 0; k < 3; ++k) if (k != n) J *= v.dim[k];
  a.nfib = J;
  a.wscale = 1.0;
  int64_t per = 0;
  a.splits = mttkrp_plan_splits(a, &per);
  a.fib_per_split = per;
  a.partial = c->partial.p;
  return a;
}

// per-context scratch of a work-list step (the buffers str_step uses)
str_status wl_grow(str_ctx* c, const SlabView& v) {
  const int64_t tn = v.dim[2];
  const int RR0 = c->RR(0), RR1 = c->RR(1), RR2 = c->RR(2);
  TRY(grow(c, c->gnew64, (size_t)tn * RR2 * 8));
  TRY(grow(c, c->gnew32, (size_t)tn * RR2 * 4));
  TRY(grow(c, c->enew, (size_t)RR2 * RR2 * 8));
  TRY(grow(c, c->mtmp, (size_t)tn * RR2 * 8));
  TRY(grow(c, c->qtmp, (size_t)RR2 * RR2 * 8));
  const int RRm = std::max(RR0, std::max(RR1, RR2));
  TRY(grow(c, c->lfac, (size_t)RRm * RRm * 8));
  TRY(grow(c, c->qf, (size_t)RRm * RRm * 4));
  TRY(grow(c, c->qlo, (size_t)RRm * RRm * 4));
  // the largest split-partial buffer of the three MTTKRPs
  size_t part = 0;
  const void* cores[3] = {nullptr, nullptr, nullptr};
  for (int n = 0; n < 3; ++n) {
    MttkrpArgs a = wl_mttkrp_args(c, v, n, cores);
    part = std::max(part, (size_t)a.splits * v.dim[n] * c->RR(n) * 4);
  }
  TRY(grow(c, c->partial, part));
  return STR_OK;
}

// Builds the job lists of one step for every context and uploads them.
str_status wl_build(WLLayout* L, str_ctx* const* ctxs, const std::vector<SlabView>& v, int count) {
  std::vector<char> img;
  auto put = [&](const void* p, size_t bytes) -> size_t {
    size_t off = (img.size() + 255) & ~(size_t)255;
    img.resize(off + bytes);
    if (bytes) std::memcpy(img.data() + off, p, bytes);
    return off;
  };
  L->launches.clear();
  auto add_gram = [&](const std::vector<GramJob>& jobs) {
    std::vector<int2> items;
    for (int j = 0; j < (int)jobs.size(); ++j)
      for (int b = 0; b < core_gram_blocks(jobs[j].Ra * jobs[j].Rb); ++b) items.push_back(make_int2(j, b));
    WLLaunch l{WL_GRAM};
    l.jobs = put(jobs.data(), jobs.size() * sizeof(GramJob));
    l.items = put(items.data(), items.size() * sizeof(int2));
    l.n = (int)items.size();
    L->launches.push_back(l);
  };
  auto add_gemm = [&](const std::vector<GemmJob>& jobs) {
    std::vector<int4> items;
    int Kmax = 1;
    for (int j = 0; j < (int)jobs.size(); ++j) {
      Kmax = std::max(Kmax, jobs[j].K);
      for (int by = 0; by < ceil_div_i(jobs[j].M, 8); ++by)
        for (int bx = 0; bx < ceil_div_i(jobs[j].N, 8); ++bx) items.push_back(make_int4(j, bx, by, 0));
    }
    WLLaunch l{WL_GEMM};
    l.jobs = put(jobs.data(), jobs.size() * sizeof(GemmJob));
    l.items = put(items.data(), items.size() * sizeof(int4));
    l.n = (int)items.size();
    l.p0 = Kmax;
    L->launches.push_back(l);
  };
  auto add_sweep = [&](const std::vector<SweepJob>& jobs) {
    WLLaunch l{WL_SWEEP};
    l.jobs = put(jobs.data(), jobs.size() * sizeof(SweepJob));
    l.n = (int)jobs.size();
    L->launches.push_back(l);
  };
  // MTTKRPs grouped by register-block class; reduction into out (+ base)
  auto add_mttkrp = [&](const std::vector<MttkrpArgs>& jobs, const std::vector<int>& stream_of,
                        const std::vector<double*>& outs, const std::vector<const double*>& bases) {
    for (int cls = 0; cls < 6; ++cls) {
      std::vector<MttkrpArgs> cj;
      std::vector<int4> items;
      int BK = L->tune.bk;
      size_t smem = 0;
      for (int j = 0; j < (int)jobs.size(); ++j) {
        if (mttkrp_class(jobs[j]) != cls) continue;
        while (BK > 4 && mttkrp_smem_bytes(jobs[j], BK) > 96 * 1024) BK /= 2;
      }
      for (int j = 0; j < (int)jobs.size(); ++j) {
        if (mttkrp_class(jobs[j]) != cls) continue;
        const int ji = (int)cj.size();
        cj.push_back(jobs[j]);
        smem = std::max(smem, mttkrp_smem_bytes(jobs[j], BK));
        const int gx = ceil_div_i(jobs[j].dim[jobs[j].n], mttkrp_rows_per_block(jobs[j]));
        for (int by = 0; by < jobs[j].splits; ++by)
          for (int bx = 0; bx < gx; ++bx) items.push_back(make_int4(ji, bx, by, stream_of[j]));
      }
      if (cj.empty()) continue;
      WLLaunch l{WL_MTTKRP};
      l.jobs = put(cj.data(), cj.size() * sizeof(MttkrpArgs));
      l.items = put(items.data(), items.size() * sizeof(int4));
      l.n = (int)items.size();
      l.p0 = cls;
      l.p1 = v[0].xtype;
      l.p2 = BK;
      l.smem = smem;
      L->launches.push_back(l);
    }
    std::vector<ReduceJob> rj;
    std::vector<int2> items;
    for (int j = 0; j < (int)jobs.size(); ++j) {
      ReduceJob r;
      r.partial = (const float*)jobs[j].partial;
      r.splits = jobs[j].splits;
      r.count = jobs[j].dim[jobs[j].n] * jobs[j].R[jobs[j].n] * jobs[j].R[jobs[j].n + 1];
      r.base = bases[j];
      r.out = outs[j];
      for (int64_t b = 0; b < (r.count + 255) / 256; ++b) items.push_back(make_int2(j, (int)b));
      rj.push_back(r);
    }
    WLLaunch l{WL_REDUCE};
    l.jobs = put(rj.data(), rj.size() * sizeof(ReduceJob));
    l.items = put(items.data(), items.size() * sizeof(int2));
    l.n = (int)items.size();
    L->launches.push_back(l);
  };
  auto add_apply = [&](const std::vector<ApplyDF>& jobs) {
    // orders 129..160: the FP32 inverse with an FP64 residual (as apply_q)
    {
      std::vector<RefineJob> rj;
      std::vector<int4> items;
      int nmax = 129;
      size_t smem = 0;
      for (const ApplyDF& a : jobs) {
        if (apply_df_supported(a.n)) continue;
        RefineJob r;
        r.W = a.W; r.Q = a.Q64; r.n = a.n; r.P = a.P; r.rows = a.rows; r.iters = 1;
        r.q_in_smem = refine_q_in_smem(a.n);
        r.out64 = a.out64; r.out32 = a.out32;
        const int ji = (int)rj.size();
        rj.push_back(r);
        nmax = std::max(nmax, a.n);
        smem = std::max(smem, refine_smem(a.n, r.q_in_smem));
        const int64_t nb = std::max<int64_t>(1, (a.rows + L->tune.rows_per_block - 1) / L->tune.rows_per_block);
        for (int64_t b = 0; b < nb; ++b) items.push_back(make_int4(ji, (int)b, (int)nb, 0));
      }
      if (!rj.empty()) {
        WLLaunch l{WL_REFINE};
        l.jobs = put(rj.data(), rj.size() * sizeof(RefineJob));
        l.items = put(items.data(), items.size() * sizeof(int4));
        l.n = (int)items.size();
        l.p0 = nmax;
        l.smem = smem;
        L->launches.push_back(l);
      }
    }
    for (int cpt = 1; cpt <= 2; ++cpt) {
      std::vector<ApplyDF> cj;
      std::vector<int4> items;
      int nmax = 2;
      for (const ApplyDF& a : jobs) {
        if (!apply_df_supported(a.n) || (a.n <= 64 ? 1 : 2) != cpt) continue;
        const int ji = (int)cj.size();
        cj.push_back(a);
        nmax = std::max(nmax, a.n);
        const int64_t nb = std::max<int64_t>(1, (a.rows + L->tune.rows_per_block - 1) / L->tune.rows_per_block);
        for (int64_t b = 0; b < nb; ++b) items.push_back(make_int4(ji, (int)b, (int)nb, 0));
      }
      if (cj.empty()) continue;
      WLLaunch l{WL_APPLY};
      l.jobs = put(cj.data(), cj.size() * sizeof(ApplyDF));
      l.items = put(items.data(), items.size() * sizeof(int4));
      l.n = (int)items.size();
      l.p0 = nmax;
      L->launches.push_back(l);
    }
  };
  auto apply_job = [&](str_ctx* c, const double* Q, int n, const double* P, int64_t rows, double* o64, float* o32) {
    ApplyDF a;
    a.W = (const float*)c->lfac.p;
    a.Qh = (const float*)c->qf.p;
    a.Ql = (const float*)c->qlo.p;
    a.n = n;
    a.rows = rows;
    a.P = P;
    a.out64 = o64;
    a.out32 = o32;
    a.status = c->d_status;
    a.Q64 = Q;
    a.pivot_ratio = c->d_pivot;
    a.fallbacks = c->d_fallbacks;
    return a;
  };
  auto sweep_job = [&](str_ctx* c, const double* Q, int n) {
    SweepJob sj;
    sj.Q = Q;
    sj.n = n;
    sj.W = (float*)c->lfac.p;
    sj.status = c->d_status;
    sj.pivot_ratio = c->d_pivot;
    return sj;
  };
  auto gemm_job = [&](str_ctx* c, const double* A, const double* B, double* C, int M, int K, int N, int pRa, int pRb,
                      const double* base) {
    GemmJob g;
    g.A = A; g.B = B; g.C = C; g.M = M; g.K = K; g.N = N; g.pRa = pRa; g.pRb = pRb; g.base = base;
    g.Qf = (float*)c->qf.p;
    g.Qlo = (float*)c->qlo.p;
    return g;
  };
  auto gram_job = [&](const double* G, int64_t I, int Ra, int Rb, double* E) {
    GramJob g;
    g.G = G; g.I = I; g.Ra = Ra; g.Rb = Rb; g.E = E;
    g.chunk = core_gram_chunk(I, Ra * Rb);
    return g;
  };
  std::vector<int> stream_of(count);
  for (int i = 0; i < count; ++i) stream_of[i] = i;
  // ---- temporal mode (Alg. 4): Q_N = ring(E_1 E_2), M_N, G_N^new = M_N Q_N^{-1} ----
  {
    std::vector<GemmJob> gj;
    std::vector<SweepJob> sj;
    std::vector<MttkrpArgs> mj;
    std::vector<double*> outs;
    std::vector<const double*> bases;
    std::vector<ApplyDF> aj;
    for (int i = 0; i < count; ++i) {
      str_ctx* c = ctxs[i];
      const int* R = c->R;
      gj.push_back(gemm_job(c, E_of(c, 0), E_of(c, 1), (double*)c->qtmp.p, R[0] * R[0], R[1] * R[1], R[2] * R[2],
                            R[2], R[0], nullptr));
      sj.push_back(sweep_job(c, (const double*)c->qtmp.p, c->RR(2)));
      const void* cores[3] = {core_c(c, 0), core_c(c, 1), nullptr};
      mj.push_back(wl_mttkrp_args(c, v[i], 2, cores));
      outs.push_back((double*)c->mtmp.p);
      bases.push_back(nullptr);
      aj.push_back(apply_job(c, (const double*)c->qtmp.p, c->RR(2), (const double*)c->mtmp.p, v[i].dim[2],
                             (double*)c->gnew64.p, (float*)c->gnew32.p));
    }
    add_gemm(gj);
    add_sweep(sj);
    add_mttkrp(mj, stream_of, outs, bases);
    add_apply(aj);
  }
  // ---- spatial modes n = 1, 2 (Gauss-Seidel): Gram of the core updated just before,
  //      Q_n = Q_n^old + ring, P_n = P_n^old + MTTKRP, G_n = P_n Q_n^{-1} ----
  for (int n = 0; n < 2; ++n) {
    std::vector<GramJob> grj;
    std::vector<GemmJob> gj;
    std::vector<SweepJob> sj;
    std::vector<MttkrpArgs> mj;
    std::vector<double*> outs;
    std::vector<const double*> bases;
    std::vector<ApplyDF> aj;
    for (int i = 0; i < count; ++i) {
      str_ctx* c = ctxs[i];
      const int* R = c->R;
      const int w = 1 - c->cur[n];
      if (n == 0) {
        grj.push_back(gram_job((const double*)c->gnew64.p, v[i].dim[2], R[2], R[0], (double*)c->enew.p));
        gj.push_back(gemm_job(c, E_of(c, 1), (const double*)c->enew.p, c->Q[0][w], R[1] * R[1], R[2] * R[2],
                              R[0] * R[0], R[0], R[1], c->Q[0][c->cur[0]]));
      } else {
        const int w0 = 1 - c->cur[0];
        grj.push_back(gram_job(c->G64[0][w0], c->I[0], R[0], R[1], c->E[0][w0]));
        gj.push_back(gemm_job(c, (const double*)c->enew.p, c->E[0][w0], c->Q[1][w], R[2] * R[2], R[0] * R[0],
                              R[1] * R[1], R[1], R[2], c->Q[1][c->cur[1]]));
      }
      sj.push_back(sweep_job(c, c->Q[n][w], c->RR(n)));
      const void* cores[3];
      if (n == 0) { cores[0] = c->G32[0][c->cur[0]]; cores[1] = c->G32[1][c->cur[1]]; }
      else { cores[0] = c->G32[0][1 - c->cur[0]]; cores[1] = c->G32[1][c->cur[1]]; }
      cores[2] = c->gnew32.p;
      mj.push_back(wl_mttkrp_args(c, v[i], n, cores));
      outs.push_back(c->P[n][w]);
      bases.push_back(c->P[n][c->cur[n]]);
      aj.push_back(apply_job(c, c->Q[n][w], c->RR(n), c->P[n][w], c->I[n], c->G64[n][w], c->G32[n][w]));
    }
    add_gram(grj);
    add_gemm(gj);
    add_sweep(sj);
    add_mttkrp(mj, stream_of, outs, bases);
    add_apply(aj);
  }
  // ---- Gram of the last core updated (kept with the committed state) ----
  {
    std::vector<GramJob> grj;
    for (int i = 0; i < count; ++i) {
      str_ctx* c = ctxs[i];
      const int w1 = 1 - c->cur[1];
      grj.push_back(gram_job(c->G64[1][w1], c->I[1], c->R[1], c->R[2], c->E[1][w1]));
    }
    add_gram(grj);
  }
  // ---- append the new temporal rows (copy jobs are per step: the destination moves) ----
  {
    std::vector<int2> items;
    for (int i = 0; i < count; ++i) {
      const int64_t b64 = v[i].dim[2] * ctxs[i]->RR(2) * 8, b32 = b64 / 2;
      for (int64_t b = 0; b < (b64 + 16383) / 16384; ++b) items.push_back(make_int2(2 * i, (int)b));
      for (int64_t b = 0; b < (b32 + 16383) / 16384; ++b) items.push_back(make_int2(2 * i + 1, (int)b));
    }
    WLLaunch l{WL_COPY};
    l.items = put(items.data(), items.size() * sizeof(int2));
    l.n = (int)items.size();
    L->launches.push_back(l);
  }
  // status pointers (for one gathered read of every context's status word)
  {
    std::vector<const int*> sp(count);
    for (int i = 0; i < count; ++i) sp[i] = ctxs[i]->d_status;
    L->statusptr_off = put(sp.data(), sp.size() * sizeof(const int*));
    std::vector<int> zero(count, 0);
    L->status_off = put(zero.data(), zero.size() * sizeof(int));
  }
  // per-step region: slab pointers, then the append copy jobs
  L->dyn_off = (img.size() + 255) & ~(size_t)255;
  L->xptr_off = L->dyn_off;
  L->copyjob_off = L->dyn_off + (((size_t)count * sizeof(void*) + 255) & ~(size_t)255);
  L->dyn_bytes = L->copyjob_off - L->dyn_off + (size_t)2 * count * sizeof(CopyJob);
  img.resize(L->dyn_off + L->dyn_bytes);
  L->dyn.assign(L->dyn_bytes, 0);
  if (L->arena) cudaFree(L->arena);
  L->arena = nullptr;
  cudaError_t e = cudaMalloc(&L->arena, img.size());
  if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e, "cudaMalloc(work list)"); }
  STR_CUDA_TRY(cudaMemcpy(L->arena, img.data(), img.size(), cudaMemcpyHostToDevice));
  if (!L->h_status) STR_CUDA_TRY(cudaMallocHost(&L->h_status, (size_t)count * sizeof(int)));
  return STR_OK;
}

// the step's launches (no host work besides the launches)
str_status wl_launch(WLLayout* L, cudaStream_t s) {
  char* A = L->arena;
  const void* const* xptrs = (const void* const*)(A + L->xptr_off);
  for (const WLLaunch& l : L->launches) {
    switch (l.kind) {
      case WL_GRAM: STR_CUDA_TRY(launch_core_gram_batch((const GramJob*)(A + l.jobs), (const int2*)(A + l.items), l.n, s)); break;
      case WL_GEMM: STR_CUDA_TRY(launch_gemm64_batch((const GemmJob*)(A + l.jobs), (const int4*)(A + l.items), l.n, l.p0, s)); break;
      case WL_SWEEP: STR_CUDA_TRY(launch_sweep_batch((const SweepJob*)(A + l.jobs), l.n, s)); break;
      case WL_MTTKRP:
        STR_CUDA_TRY(launch_mttkrp_batch((const MttkrpArgs*)(A + l.jobs), (const int4*)(A + l.items), xptrs, l.n, l.p0,
                                         l.p1, l.p2, l.smem, s));
        break;
      case WL_REDUCE: STR_CUDA_TRY(launch_reduce_batch((const ReduceJob*)(A + l.jobs), (const int2*)(A + l.items), l.n, s)); break;
      case WL_APPLY: STR_CUDA_TRY(launch_apply_df_batch((const ApplyDF*)(A + l.jobs), (const int4*)(A + l.items), l.n, l.p0, s)); break;
      case WL_REFINE:
        STR_CUDA_TRY(launch_refine_batch((const RefineJob*)(A + l.jobs), (const int4*)(A + l.items), l.n, l.p0, l.smem, s));
        break;
      case WL_COPY: STR_CUDA_TRY(launch_copy_batch((const CopyJob*)(A + L->copyjob_off), (const int2*)(A + l.items), l.n, s)); break;
    }
  }
  return STR_OK;
}

// the per-step region: this step's slab pointers and append destinations
str_status wl_upload(WLLayout* L, str_ctx* const* ctxs, const std::vector<SlabView>& v, int count, cudaStream_t s) {
  const void** xp = (const void**)L->dyn.data();
  CopyJob* cj = (CopyJob*)(L->dyn.data() + (L->copyjob_off - L->dyn_off));
  for (int i = 0; i < count; ++i) {
    str_ctx* c = ctxs[i];
    const int RRN = c->RR(2);
    const int64_t tn = v[i].dim[2];
    xp[i] = v[i].X;
    cj[2 * i].src = c->gnew64.p;
    cj[2 * i].dst = c->GT64 + c->t_rows * RRN;
    cj[2 * i].bytes = tn * RRN * 8;
    cj[2 * i + 1].src = c->gnew32.p;
    cj[2 * i + 1].dst = c->GT32 + c->t_rows * RRN;
    cj[2 * i + 1].bytes = tn * RRN * 4;
  }
  // pageable source: staged by the call, so the host image can be rewritten next step
  STR_CUDA_TRY(cudaMemcpyAsync(L->arena + L->dyn_off, L->dyn.data(), L->dyn_bytes, cudaMemcpyHostToDevice, s));
  return STR_OK;
}

// the layout of this batch (built, tuned and cached on first use; the caller
// holds g_wl_mu)
str_status wl_layout(str_ctx* const* ctxs, const std::vector<int64_t>& tns, const std::vector<SlabView>& v,
                     int count, cudaStream_t s, WLLayout** out) {
  for (WLLayout* L : g_wl) {
    if ((int)L->uids.size() != count || L->dev != ctxs[0]->dev) continue;
    bool same = true;
    for (int i = 0; i < count && same; ++i) {
      const str_ctx* c = ctxs[i];
      same = L->uids[i] == c->uid && L->tns[i] == tns[i] && L->xtypes[i] == v[i].xtype && L->parity[i] == c->cur[0] &&
             L->gens[i] == c->gen;
    }
    if (same) { *out = L; return STR_OK; }
  }
  WLLayout* L = new WLLayout;
  L->dev = ctxs[0]->dev;
  for (int i = 0; i < count; ++i) {
    const str_ctx* c = ctxs[i];
    L->uids.push_back(c->uid);
    L->tns.push_back(tns[i]);
    L->xtypes.push_back(v[i].xtype);
    L->parity.push_back(c->cur[0]);
    L->gens.push_back(c->gen);
  }
  const uint64_t sig = wl_signature(ctxs, tns, v, count);
  bool tuned = false;
  for (const WLTuned& t : g_wl_tuned)
    if (t.sig == sig) { L->tune = t.tune; tuned = true; }
  if (!tuned) {
    // autotune: time every candidate on this step (the step writes working
    // buffers only, so repeating it leaves the committed state as it was)
    const int bks[3] = {8, 16, 32};
    const int rpbs[3] = {1, 4, 16};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    STR_CUDA_TRY(cudaEventCreate(&e0));
    STR_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    WLTune best_t;
    str_status st = STR_OK;
    for (int bi = 0; bi < 3 && st == STR_OK; ++bi)
      for (int ri = 0; ri < 3 && st == STR_OK; ++ri) {
        L->tune.bk = bks[bi];
        L->tune.rows_per_block = rpbs[ri];
        st = wl_build(L, ctxs, v, count);
        if (st != STR_OK) break;
        st = wl_upload(L, ctxs, v, count, s);
        if (st == STR_OK) st = wl_launch(L, s);           // warm-up
        if (st == STR_OK && cudaEventRecord(e0, s) != cudaSuccess) st = STR_ERR_CUDA;
        if (st == STR_OK) st = wl_launch(L, s);
        if (st == STR_OK && cudaEventRecord(e1, s) != cudaSuccess) st = STR_ERR_CUDA;
        float ms = 0.f;
        if (st == STR_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
          st = STR_ERR_CUDA;
        if (st == STR_OK && ms < best) { best = ms; best_t = L->tune; }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != STR_OK) { wl_free(L); return st; }
    L->tune = best_t;
    if (g_wl_tuned.size() >= 64) g_wl_tuned.erase(g_wl_tuned.begin());
    g_wl_tuned.push_back({sig, best_t});
  }
  const str_status st = wl_build(L, ctxs, v, count);
  if (st != STR_OK) { wl_free(L); return st; }
  if (g_wl.size() >= 16) {   // bounded cache: drop the oldest layout
    wl_free(g_wl.front());
    g_wl.erase(g_wl.begin());
  }
  g_wl.push_back(L);
  *out = L;
  return STR_OK;
}

// One step of every context by the work-list launches (on any stream; captured
// and replayed as a graph when the layout recurs on a non-default stream).
// The caller holds g_wl_mu.
str_status wl_step(str_ctx* const* ctxs, const std::vector<int64_t>& tns, const std::vector<SlabView>& v, int count,
                   cudaStream_t s) {
  for (int i = 0; i < count; ++i) TRY(wl_grow(ctxs[i], v[i]));
  WLLayout* L = nullptr;
  TRY(wl_layout(ctxs, tns, v, count, s, &L));
  TRY(wl_upload(L, ctxs, v, count, s));
  const bool can_capture = s != nullptr && s != cudaStreamLegacy;
  if (L->exec) {
    STR_CUDA_TRY(cudaGraphLaunch(L->exec, s));
  } else if (can_capture && L->runs >= 1) {
    cudaGraph_t graph = nullptr;
    STR_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    const str_status st = wl_launch(L, s);
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st != STR_OK || ce != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      if (st != STR_OK) return st;
      return from_cuda(ce, "cudaStreamEndCapture(work list)");
    }
    const cudaError_t ie = cudaGraphInstantiate(&L->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) { L->exec = nullptr; return from_cuda(ie, "cudaGraphInstantiate(work list)"); }
    STR_CUDA_TRY(cudaGraphLaunch(L->exec, s));
  } else {
    TRY(wl_launch(L, s));
  }
  L->runs++;
  for (int i = 0; i < count; ++i) {
    str_ctx* c = ctxs[i];
    c->upd[0] = c->upd[1] = 1;
    for (int k = 0; k < 3; ++k) c->core_ver[k]++;
    c->qsplit_of = nullptr;
    c->launches = (int64_t)L->launches.size();
  }
  return STR_OK;
}

// every context's status word in one read (one synchronisation): device pointer
// list, gathered words and their pinned host copy, grow-only (under g_wl_mu)
const int** g_wl_sptr = nullptr;
int* g_wl_sval = nullptr;
int* g_wl_shost = nullptr;
int g_wl_scap = 0;

str_status wl_statuses(str_ctx* const* ctxs, int count, cudaStream_t s, std::vector<int>* st) {
  if (count > g_wl_scap) {
    if (g_wl_sptr) cudaFree(g_wl_sptr);
    if (g_wl_sval) cudaFree(g_wl_sval);
    if (g_wl_shost) cudaFreeHost(g_wl_shost);
    g_wl_sptr = nullptr; g_wl_sval = nullptr; g_wl_shost = nullptr; g_wl_scap = 0;
    STR_CUDA_TRY(cudaMalloc((void**)&g_wl_sptr, (size_t)count * sizeof(int*)));
    STR_CUDA_TRY(cudaMalloc((void**)&g_wl_sval, (size_t)count * sizeof(int)));
    STR_CUDA_TRY(cudaMallocHost((void**)&g_wl_shost, (size_t)count * sizeof(int)));
    g_wl_scap = count;
  }
  std::vector<const int*> sp(count);
  for (int i = 0; i < count; ++i) sp[i] = ctxs[i]->d_status;
  STR_CUDA_TRY(cudaMemcpyAsync(g_wl_sptr, sp.data(), (size_t)count * sizeof(int*), cudaMemcpyHostToDevice, s));
  STR_CUDA_TRY(launch_gather_ints(g_wl_sptr, count, g_wl_sval, s));
  STR_CUDA_TRY(cudaMemcpyAsync(g_wl_shost, g_wl_sval, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, s));
  STR_CUDA_TRY(cudaStreamSynchronize(s));
  st->assign(g_wl_shost, g_wl_shost + count);
  return STR_OK;
}

bool wl_candidates(str_ctx* const* ctxs, int count) {
  for (int i = 0; i < count; ++i) {
    const str_ctx* c = ctxs[i];
    if (!c || c->sticky || c->N != 3 || c->compute != 1 || c->opt.sweeps != 1 || c->opt.profile) return false;
    for (int k = 0; k < 3; ++k)
      if (c->RR(k) > 160) return false;
  }
  return count > 0;
}

// str_update_batch for a batch of work-list candidates: all or none committed
str_status wl_update_batch(str_ctx* const* ctxs, const str_tensor* const* X, int count, cudaStream_t s) {
  std::vector<SlabView> v(count);
  std::vector<int64_t> tns(count);
  for (int i = 0; i < count; ++i) {
    str_ctx* c = ctxs[i];
    TRY(take_slab(c, X[i], &v[i], s));
    tns[i] = v[i].dim[2];
    if (c->t_rows + tns[i] > c->opt.t_capacity) return STR_ERR_CAPACITY;
    if (!wl_eligible(c, v[i])) return STR_ERR_DTYPE;
  }
  std::lock_guard<std::mutex> lk(g_wl_mu);
  // a device failure of an earlier step (no-synchronisation contexts) latches the context
  std::vector<int> st0;
  TRY(wl_statuses(ctxs, count, s, &st0));
  for (int i = 0; i < count; ++i)
    if (st0[i]) { ctxs[i]->sticky = ctxs[i]->opt.async_status ? 1 : 0; return STR_ERR_STATE; }
  str_status st = wl_step(ctxs, tns, v, count, s);
  bool sync_any = false;
  for (int i = 0; i < count; ++i) sync_any = sync_any || !ctxs[i]->opt.async_status;
  std::vector<int> st1;
  if (st == STR_OK && sync_any) st = wl_statuses(ctxs, count, s, &st1);
  bool fail = st != STR_OK;
  for (int i = 0; i < count && !fail && sync_any; ++i) {
    if (ctxs[i]->opt.async_status || !st1[i]) continue;
    fail = true;
    st = (st1[i] & DEV_ERR_NONFINITE) ? STR_ERR_NONFINITE
         : (st1[i] & DEV_ERR_SINGULAR) ? STR_ERR_SINGULAR : (st1[i] & DEV_ERR_TIMEOUT) ? STR_ERR_TIMEOUT : STR_ERR_CUDA;
  }
  for (int i = 0; i < count; ++i) {
    str_ctx* c = ctxs[i];
    if (fail) {
      for (int k = 0; k < STR_MAXN; ++k) c->upd[k] = 0;
      cudaMemsetAsync(c->d_status, 0, sizeof(int), s);
      continue;
    }
    for (int k = 0; k < STR_MAXN; ++k) { if (c->upd[k]) c->cur[k] ^= 1; c->upd[k] = 0; }
    c->t_rows += tns[i];
    c->last_tn = tns[i];
    c->step += 1;
  }
  return st;
}

str_status str_update_batch(str_ctx* const* ctxs, const str_tensor* const* X, int count, int randomized,
                            void* stream) {
  if (!ctxs || !X || count < 0) return STR_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  str_mark_cross_wait(s);   // the caller may have ordered s after other streams
  for (int i = 0; i < count; ++i) if (!ctxs[i] || !X[i]) return STR_ERR_INVALID_ARG;
  if (!randomized && wl_candidates(ctxs, count)) return wl_update_batch(ctxs, X, count, s);
  // enqueue every context's step with status checks deferred, then commit all or none
  std::vector<int64_t> tns(count);
  for (int i = 0; i < count; ++i) {
    str_ctx* c = ctxs[i];
    if (!c) return STR_ERR_INVALID_ARG;
    TRY(precheck(c, s));
    if (randomized && c->opt.sketch == STR_SKETCH_NONE) return STR_ERR_STATE;
  }
  str_status st = STR_OK;
  int done = 0;
  // concurrent branches on a non-default stream; rSTR steps are not captured into
  // a replayed graph (each step's draws take the step number as a launch argument)
  bool concurrent = count > 0 && s != nullptr && s != cudaStreamLegacy;
  for (int i = 0; i < count; ++i)
    if (ctxs[i]->opt.profile) concurrent = false;
  if (!concurrent) {
    for (int i = 0; i < count && st == STR_OK; ++i) {
      str_ctx* c = ctxs[i];
      c->launches = 0;
      SlabView v;
      st = take_slab(c, X[i], &v, s);
      if (st != STR_OK) break;
      tns[i] = v.dim[c->N - 1];
      if (c->t_rows + tns[i] > c->opt.t_capacity) { st = STR_ERR_CAPACITY; break; }
      st = randomized ? rstr_step(c, v, s) : str_step(c, v, s);
      if (st == STR_OK && !randomized) st = append_rows(c, tns[i], s);
      done = i + 1;
    }
  } else {
    // slabs staged at each context's fixed address, then every update as one
    // branch of a captured batch graph (plain concurrent branches until every
    // context has run its slab shape once)
    std::vector<SlabView> v(count);
    bool graphs = true, warm = true;
    for (int i = 0; i < count && st == STR_OK; ++i) {
      str_ctx* c = ctxs[i];
      c->launches = 0;
      st = take_slab(c, X[i], &v[i], s);
      if (st != STR_OK) break;
      tns[i] = v[i].dim[c->N - 1];
      if (c->t_rows + tns[i] > c->opt.t_capacity) { st = STR_ERR_CAPACITY; break; }
      st = ensure_bstream(c);
      if (st != STR_OK) break;
      int64_t cnt = 1;
      for (int k = 0; k < c->N; ++k) cnt *= v[i].dim[k];
      if (v[i].X != c->xstage.p) {
        st = grow(c, c->xstage, (size_t)cnt * dsize(X[i]->dtype));
        if (st != STR_OK) break;
        if (cudaMemcpyAsync(c->xstage.p, v[i].X, (size_t)cnt * dsize(X[i]->dtype), cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess) { st = STR_ERR_CUDA; break; }
        v[i].X = c->xstage.p;
      }
      if (!c->opt.graphs || randomized) graphs = false;
      const std::pair<int64_t, int> shape(tns[i], v[i].xtype);
      if (std::find(c->warm.begin(), c->warm.end(), shape) == c->warm.end()) warm = false;
    }
    if (st == STR_OK) {
      done = count;
      BatchGraph* hit = nullptr;
      std::unique_lock<std::mutex> lk(g_batch_mu);
      if (graphs && warm) {
        for (auto& g : g_batch) {
          if ((int)g.uids.size() != count) continue;
          bool same = true;
          for (int i = 0; i < count && same; ++i) {
            const str_ctx* c = ctxs[i];
            same = g.uids[i] == c->uid && g.tns[i] == tns[i] && g.xtypes[i] == v[i].xtype &&
                   g.parity[i] == c->cur[0] && g.gens[i] == c->gen && g.dev == c->dev;
          }
          if (same) { hit = &g; break; }
        }
      }
      if (hit) {
        if (cudaGraphLaunch(hit->exec, s) != cudaSuccess) st = STR_ERR_CUDA;
        for (int i = 0; i < count; ++i)
          for (int k = 0; k < ctxs[i]->N - 1; ++k) { ctxs[i]->upd[k] = 1; ctxs[i]->core_ver[k]++; }
      } else if (graphs && warm && !seen_before(batch_key(ctxs, tns, v, count))) {
        lk.unlock();
        st = batch_steps(ctxs, v, count, s);
      } else if (graphs && warm) {
        std::vector<uint64_t> gen0(count);
        for (int i = 0; i < count; ++i) gen0[i] = ctxs[i]->gen;
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = STR_ERR_CUDA;
        if (st == STR_OK) {
          g_in_capture = true;
          st = batch_steps(ctxs, v, count, s);
          const cudaError_t ce = cudaStreamEndCapture(s, &graph);
          g_in_capture = false;
          {
            const str_status zs = zero_pending();
            if (st == STR_OK) st = zs;
          }
          bool moved = false;
          for (int i = 0; i < count; ++i) moved = moved || ctxs[i]->gen != gen0[i];
          if (st == STR_OK && (ce != cudaSuccess || moved)) {
            // a buffer grew during capture: nothing recorded ran; run the branches directly
            if (graph) cudaGraphDestroy(graph);
            graph = nullptr;
            cudaGetLastError();
            for (int i = 0; i < count; ++i) {
              for (int k = 0; k < STR_MAXN; ++k) ctxs[i]->upd[k] = 0;
              ctxs[i]->y_slab[0] = ctxs[i]->y_slab[1] = nullptr;
              ctxs[i]->tc_xt_src = nullptr;
            }
            st = batch_steps(ctxs, v, count, s);
          } else if (st == STR_OK) {
            cudaGraphExec_t exec = nullptr;
            const cudaError_t ie = cudaGraphInstantiate(&exec, graph, cudaGraphInstantiateFlagUseNodePriority);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
              st = from_cuda(ie, "cudaGraphInstantiate(batch)");
            } else {
              BatchGraph g;
              g.dev = ctxs[0]->dev;
              for (int i = 0; i < count; ++i) {
                const str_ctx* c = ctxs[i];
                g.uids.push_back(c->uid);
                g.tns.push_back(tns[i]);
                g.xtypes.push_back(v[i].xtype);
                g.parity.push_back(c->cur[0]);
                g.gens.push_back(c->gen);
              }
              g.exec = exec;
              if (g_batch.size() >= 64) {   // bounded cache: drop the oldest graph
                cudaGraphExecDestroy(g_batch.front().exec);
                g_batch.erase(g_batch.begin());
              }
              g_batch.push_back(g);
              if (cudaGraphLaunch(exec, s) != cudaSuccess) st = STR_ERR_CUDA;
            }
          } else if (graph) {
            cudaGraphDestroy(graph);
          }
        }
      } else {
        lk.unlock();
        st = batch_steps(ctxs, v, count, s, randomized != 0);
        for (int i = 0; i < count && st == STR_OK; ++i) {
          const std::pair<int64_t, int> shape(tns[i], v[i].xtype);
          if (std::find(ctxs[i]->warm.begin(), ctxs[i]->warm.end(), shape) == ctxs[i]->warm.end())
            ctxs[i]->warm.push_back(shape);
        }
      }
    }
    for (int i = 0; i < done && st == STR_OK && !randomized; ++i) st = append_rows(ctxs[i], tns[i], s);
  }
  bool any_fail = st != STR_OK;
  if (!any_fail) {
    for (int i = 0; i < count; ++i) {
      str_ctx* c = ctxs[i];
      if (c->opt.async_status) continue;
      bool failed = false;
      str_status e = check_status(c, s, &failed);
      if (e != STR_OK) { st = e; any_fail = true; }
    }
  }
  for (int i = 0; i < done; ++i) {
    str_ctx* c = ctxs[i];
    if (any_fail) {
      for (int k = 0; k < STR_MAXN; ++k) c->upd[k] = 0;
      cudaMemsetAsync(c->d_status, 0, sizeof(int), s);
      continue;
    }
    for (int k = 0; k < STR_MAXN; ++k) { if (c->upd[k]) c->cur[k] ^= 1; c->upd[k] = 0; }
    c->t_rows += tns[i];
    c->last_tn = tns[i];
    c->step += 1;
  }
  return st;
}

str_status tr_reconstruct(const str_ctx* c, int64_t t0, int64_t t1, void* out, str_dtype dtype, void* stream) {
  if (!c || !out) return STR_ERR_INVALID_ARG;
  if (t0 < 0 || t1 <= t0 || t1 > c->t_rows) return STR_ERR_SHAPE;
  if (dtype != STR_F32 && dtype != STR_F64) return STR_ERR_DTYPE;
  return recon_common(c, t0, t1 - t0, RM_WRITE, nullptr, 0, out, xtype_of(dtype), nullptr, (cudaStream_t)stream);
}

str_status tr_fit_error(const str_ctx* cc, const str_tensor* X, int64_t t0, double* rel_err, void* stream) {
  if (!cc || !X || !rel_err || !X->data || !X->dims) return STR_ERR_INVALID_ARG;
  str_ctx* c = const_cast<str_ctx*>(cc);
  cudaStream_t s = (cudaStream_t)stream;
  str_mark_cross_wait(s);   // the caller may have ordered s after other streams
  if (X->order != c->N) return STR_ERR_SHAPE;
  for (int k = 0; k < c->N - 1; ++k) if (X->dims[k] != c->I[k]) return STR_ERR_SHAPE;
  const int64_t t = X->dims[c->N - 1];
  if (t0 < 0 || t < 1 || t0 + t > c->t_rows) return STR_ERR_SHAPE;
  int64_t count = 1;
  for (int k = 0; k < c->N; ++k) count *= X->dims[k];
  const void* Xd = X->data;
  if (X->on_host) {
    TRY(grow(c, c->xstage, (size_t)count * dsize(X->dtype)));
    STR_CUDA_TRY(cudaMemcpyAsync(c->xstage.p, X->data, (size_t)count * dsize(X->dtype), cudaMemcpyHostToDevice, s));
    Xd = c->xstage.p;
  }
  TRY(grow(c, c->sums, 64));
  TRY(recon_common(c, t0, t, RM_FIT, Xd, xtype_of(X->dtype), nullptr, 0, (double*)c->sums.p, s));
  STR_CUDA_TRY(cudaMemcpyAsync(c->h_sums, c->sums.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  STR_CUDA_TRY(cudaStreamSynchronize(s));
  *rel_err = c->h_sums[1] > 0 ? std::sqrt(c->h_sums[0] / c->h_sums[1]) : 0.0;
  return STR_OK;
}

int64_t str_num_time_rows(const str_ctx* c) { return c ? c->t_rows : -1; }

str_status str_get_core(const str_ctx* c, int n, double* host_out) {
  if (!c || !host_out || n < 1 || n > c->N) return STR_ERR_INVALID_ARG;
  const int k = n - 1;
  const int RR = c->RR(k);
  const double* src = (k == c->N - 1) ? c->GT64 : c->G64[k][c->cur[k]];
  const int64_t rows = (k == c->N - 1) ? c->t_rows : c->I[k];
  STR_CUDA_TRY(cudaDeviceSynchronize());
  STR_CUDA_TRY(cudaMemcpy(host_out, src, (size_t)rows * RR * 8, cudaMemcpyDeviceToHost));
  return STR_OK;
}

str_status str_get_pq(const str_ctx* c, int n, double* hP, double* hQ) {
  if (!c || n < 1 || n > c->N - 1) return STR_ERR_INVALID_ARG;
  const int k = n - 1;
  const int RR = c->RR(k);
  STR_CUDA_TRY(cudaDeviceSynchronize());
  if (hP) STR_CUDA_TRY(cudaMemcpy(hP, c->P[k][c->cur[k]], (size_t)c->I[k] * RR * 8, cudaMemcpyDeviceToHost));
  if (hQ) STR_CUDA_TRY(cudaMemcpy(hQ, c->Q[k][c->cur[k]], (size_t)RR * RR * 8, cudaMemcpyDeviceToHost));
  return STR_OK;
}

str_status str_get_samples(const str_ctx* c, int k1, int64_t* host_idxs, double* host_p) {
  if (!c || !host_idxs || k1 < 1 || k1 > c->N) return STR_ERR_INVALID_ARG;
  if (c->opt.sketch == STR_SKETCH_NONE) return STR_ERR_STATE;
  const int k = k1 - 1;
  std::vector<int32_t> tmp((size_t)c->opt.m);
  STR_CUDA_TRY(cudaDeviceSynchronize());
  STR_CUDA_TRY(cudaMemcpy(tmp.data(), c->idxs[k][c->cur[k]], (size_t)c->opt.m * 4, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < c->opt.m; ++i) host_idxs[i] = tmp[i];
  if (host_p) {
    if (c->opt.sketch != STR_SKETCH_LEVERAGE) return STR_ERR_STATE;
    // p_k covers the rows the draw used: I_k, or the last slab's t for the temporal mode
    const int64_t rows = (k == c->N - 1) ? (c->step == 0 ? c->t_rows : c->last_tn) : c->I[k];
    STR_CUDA_TRY(cudaMemcpy(host_p, c->p[k][c->cur[k]], (size_t)rows * 8, cudaMemcpyDeviceToHost));
  }
  return STR_OK;
}

// ---------------------------------------------------------------------------
// checkpoint: header, then committed device arrays in a fixed order
// ---------------------------------------------------------------------------
struct SaveHeader {
  uint64_t magic;
  int32_t N, compute;
  int64_t I[STR_MAXN];
  int32_t R[STR_MAXN + 1];
  str_options opt;
  int64_t t_rows, step, last_tn;
  int64_t p_rows[STR_MAXN];
};

static size_t save_size(const str_ctx* c, SaveHeader* h) {
  const int N = c->N;
  std::memset(h, 0, sizeof(*h));
  h->magic = kSaveMagic;
  h->N = N;
  h->compute = c->compute;
  for (int k = 0; k < STR_MAXN; ++k) h->I[k] = c->I[k];
  for (int k = 0; k <= STR_MAXN; ++k) h->R[k] = c->R[k];
  h->opt = c->opt;
  h->t_rows = c->t_rows;
  h->step = c->step;
  h->last_tn = c->last_tn;
  size_t sz = sizeof(SaveHeader);
  for (int k = 0; k < N - 1; ++k) {
    const size_t RR = c->RR(k);
    sz += (c->I[k] * RR + c->I[k] * RR + RR * RR + RR * RR) * 8;  // G, P, Q, E
  }
  sz += (size_t)c->t_rows * c->RR(N - 1) * 8;
  if (c->opt.sketch != STR_SKETCH_NONE) {
    sz += (size_t)N * c->opt.m * 4;
    if (c->opt.sketch == STR_SKETCH_LEVERAGE)
      for (int k = 0; k < N; ++k) { h->p_rows[k] = c->p_cap[k]; sz += (size_t)c->p_cap[k] * 8; }
  }
  return sz;
}

str_status str_save(const str_ctx* c, void* buf, size_t* len) {
  if (!c || !len) return STR_ERR_INVALID_ARG;
  SaveHeader h;
  const size_t need = save_size(c, &h);
  if (!buf) { *len = need; return STR_OK; }
  if (*len < need) { *len = need; return STR_ERR_INVALID_ARG; }
  STR_CUDA_TRY(cudaDeviceSynchronize());
  char* o = (char*)buf;
  std::memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  auto d2h = [&](const void* src, size_t bytes) -> bool {
    if (cudaMemcpy(o, src, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    o += bytes;
    return true;
  };
  const int N = c->N;
  for (int k = 0; k < N - 1; ++k) {
    const size_t RR = c->RR(k);
    const int b = c->cur[k];
    if (!d2h(c->G64[k][b], c->I[k] * RR * 8) || !d2h(c->P[k][b], c->I[k] * RR * 8) ||
        !d2h(c->Q[k][b], RR * RR * 8) || !d2h(c->E[k][b], RR * RR * 8)) return STR_ERR_CUDA;
  }
  if (!d2h(c->GT64, (size_t)c->t_rows * c->RR(N - 1) * 8)) return STR_ERR_CUDA;
  if (c->opt.sketch != STR_SKETCH_NONE) {
    for (int k = 0; k < N; ++k) if (!d2h(c->idxs[k][c->cur[k]], (size_t)c->opt.m * 4)) return STR_ERR_CUDA;
    if (c->opt.sketch == STR_SKETCH_LEVERAGE)
      for (int k = 0; k < N; ++k) if (c->p_cap[k] && !d2h(c->p[k][c->cur[k]], (size_t)c->p_cap[k] * 8)) return STR_ERR_CUDA;
  }
  *len = need;
  return STR_OK;
}

str_status str_load(str_ctx** out, const void* buf, size_t len, void* stream) {
  if (!out || !buf || len < sizeof(SaveHeader)) return STR_ERR_INVALID_ARG;
  *out = nullptr;
  SaveHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (h.magic != kSaveMagic) return STR_ERR_INVALID_ARG;
  const int N = h.N;
  if (N < 3 || N > STR_MAXN) return STR_ERR_SHAPE;
  int64_t dims[STR_MAXN];
  int ranks[STR_MAXN];
  for (int k = 0; k < N; ++k) { dims[k] = h.I[k]; ranks[k] = h.R[k]; }
  str_ctx* c = nullptr;
  TRY(ctx_create(&c, N, dims, ranks, &h.opt, h.t_rows));
  SaveHeader h2;
  c->I[N - 1] = h.I[N - 1];
  if (save_size(c, &h2) > len) { str_destroy(c); return STR_ERR_INVALID_ARG; }
  cudaStream_t s = (cudaStream_t)stream;
  str_mark_cross_wait(s);   // the caller may have ordered s after other streams
  const char* p = (const char*)buf + sizeof(SaveHeader);
  str_status st = STR_OK;
  auto h2d = [&](void* dst, size_t bytes) {
    if (st == STR_OK && cudaMemcpy(dst, p, bytes, cudaMemcpyHostToDevice) != cudaSuccess) st = STR_ERR_CUDA;
    p += bytes;
  };
  for (int k = 0; k < N - 1; ++k) {
    const size_t RR = c->RR(k);
    h2d(c->G64[k][0], c->I[k] * RR * 8);
    h2d(c->P[k][0], c->I[k] * RR * 8);
    h2d(c->Q[k][0], RR * RR * 8);
    h2d(c->E[k][0], RR * RR * 8);
    if (st == STR_OK && c->compute == 1) st = from_cuda(launch_convert(c->G64[k][0], XT_F64, c->G32[k][0], XT_F32, c->I[k] * RR, s), "convert");
  }
  const int RRN = c->RR(N - 1);
  h2d(c->GT64, (size_t)h.t_rows * RRN * 8);
  if (st == STR_OK && c->compute == 1) st = from_cuda(launch_convert(c->GT64, XT_F64, c->GT32, XT_F32, h.t_rows * RRN, s), "convert");
  if (c->opt.sketch != STR_SKETCH_NONE) {
    for (int k = 0; k < N; ++k) h2d(c->idxs[k][0], (size_t)c->opt.m * 4);
    if (c->opt.sketch == STR_SKETCH_LEVERAGE)
      for (int k = 0; k < N; ++k) {
        if (h.p_rows[k] == 0) continue;
        if (st == STR_OK) st = ensure_p(c, k, h.p_rows[k]);
        h2d(c->p[k][0], (size_t)h.p_rows[k] * 8);
      }
  }
  c->step = h.step;
  c->last_tn = h.last_tn;
  // the uploads ran on the legacy stream: complete them before any other stream reads
  if (st == STR_OK) st = from_cuda(cudaDeviceSynchronize(), "sync");
  if (st != STR_OK) { str_destroy(c); return st; }
  *out = c;
  return STR_OK;
}

str_status str_get_stats(const str_ctx* c, str_stats* stats) {
  if (!c || !stats) return STR_ERR_INVALID_ARG;
  std::memset(stats, 0, sizeof(*stats));
  stats->steps = c->step;
  stats->time_rows = c->t_rows;
  stats->kernel_launches = c->launches;
  stats->device_bytes = (int64_t)c->bytes;
  double piv = 0.0;
  if (cudaMemcpy(&piv, c->d_pivot, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return STR_ERR_CUDA;
  stats->min_pivot_ratio = piv;
  unsigned fb = 0;
  if (cudaMemcpy(&fb, c->d_fallbacks, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return STR_ERR_CUDA;
  stats->fp64_fallbacks = fb;
  str_ctx* m = const_cast<str_ctx*>(c);
  // optional launch timeline (profiling mode): STRTR_TIMELINE names a file that
  // receives one line per timed launch: class, stream (0 caller, 1-2 side
  // streams), start and end in ms from the first timed launch
  const char* tl_path = std::getenv("STRTR_TIMELINE");
  FILE* tl = (tl_path && !m->pending.empty()) ? std::fopen(tl_path, "a") : nullptr;
  for (auto& e : m->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(e.b) != cudaSuccess || cudaEventElapsedTime(&ms, e.a, e.b) != cudaSuccess) {
      if (tl) std::fclose(tl);
      return STR_ERR_CUDA;
    }
    if (tl) {
      float t0 = 0.f;
      cudaEventElapsedTime(&t0, m->pending.front().a, e.a);
      std::fprintf(tl, "%d %d %.4f %.4f\n", e.cls, e.strm, t0, t0 + ms);
    }
    m->prof_ms[e.cls] += ms;
    m->prof_launch[e.cls] += 1;
    m->pool.push_back(e.a);
    m->pool.push_back(e.b);
  }
  if (tl) { std::fprintf(tl, "--\n"); std::fclose(tl); }
  m->pending.clear();
  for (int k = 0; k < STR_K_CLASSES; ++k) {
    stats->class_launches[k] = m->prof_launch[k];
    stats->class_ms[k] = m->prof_ms[k];
    m->prof_launch[k] = 0;
    m->prof_ms[k] = 0.0;
  }
  return STR_OK;
}

str_status str_sync(str_ctx* c) {
  if (!c) return STR_ERR_INVALID_ARG;
  STR_CUDA_TRY(cudaDeviceSynchronize());
  if (c->sticky) return STR_ERR_STATE;
  int st = 0;
  STR_CUDA_TRY(cudaMemcpy(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    c->sticky = c->opt.async_status ? 1 : 0;
    if (st & DEV_ERR_NONFINITE) return STR_ERR_NONFINITE;
    if (st & DEV_ERR_SINGULAR) return STR_ERR_SINGULAR;
    return STR_ERR_TIMEOUT;
  }
  return STR_OK;
}

const char* str_status_string(str_status s) {
  switch (s) {
    case STR_OK: return "ok";
    case STR_ERR_INVALID_ARG: return "invalid argument";
    case STR_ERR_SHAPE: return "unsupported or mismatched shape";
    case STR_ERR_DTYPE: return "unsupported element type";
    case STR_ERR_SINGULAR: return "normal-equation matrix not positive definite";
    case STR_ERR_NONFINITE: return "non-finite value in a slab";
    case STR_ERR_CAPACITY: return "temporal capacity exceeded";
    case STR_ERR_OOM: return "device allocation failed";
    case STR_ERR_CUDA: return "CUDA error";
    case STR_ERR_TIMEOUT: return "device wait timed out";
    case STR_ERR_STATE: return "call not valid in this state";
  }
  return "unknown status";
}

const char* str_last_error(void) { return g_last_error.c_str(); }

void str_destroy(str_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  for (void* p : c->owned) cudaFree(p);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  for (auto& e : c->pending) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  for (auto e : c->pool) cudaEventDestroy(e);
  forget_batch_graphs(c->uid);
  forget_wl_layouts(c->uid);
  if (c->ev_bfork) cudaEventDestroy(c->ev_bfork);
  if (c->ev_bjoin) cudaEventDestroy(c->ev_bjoin);
  if (c->bstream) { str_take_cross_wait(c->bstream); cudaStreamDestroy(c->bstream); }
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) { str_take_cross_wait(c->side); cudaStreamDestroy(c->side); }
  if (c->ev_fork2) cudaEventDestroy(c->ev_fork2);
  if (c->ev_join2) cudaEventDestroy(c->ev_join2);
  if (c->side2) { str_take_cross_wait(c->side2); cudaStreamDestroy(c->side2); }
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_sums) cudaFreeHost(c->h_sums);
  delete c;
}

// ---------------------------------------------------------------------------
// masked fit loss (stateless)
// ---------------------------------------------------------------------------
static str_status loss_setup(int N, const int64_t* dims, const int* ranks, str_dtype dtype,
                             const void* const* cores, const void* X, str_ctx* tmp) {
  if (!dims || !ranks || !cores || !X) return STR_ERR_INVALID_ARG;
  if (dtype != STR_F32 && dtype != STR_F64) return STR_ERR_DTYPE;
  if (N < 3 || N > STR_MAXN) return STR_ERR_SHAPE;
  for (int k = 0; k < N; ++k) {
    if (dims[k] < 1 || ranks[k] < 1 || ranks[k] > STR_MAXR || !cores[k]) return STR_ERR_SHAPE;
  }
  tmp->N = N;
  for (int k = 0; k < N; ++k) { tmp->I[k] = dims[k]; tmp->R[k] = ranks[k]; }
  tmp->R[N] = ranks[0];
  tmp->compute = dtype == STR_F64 ? 2 : 1;
  return STR_OK;
}

// Split of the modes into a prefix 1..k and a suffix k+1..N for the fused loss
// pass (1 <= k <= N-2, K = R_1 R_{k+1} <= 64): the one with the least work in the
// reduced MTTKRPs of the backward (a prefix of one core needs none).  0 = none.
static int loss_split(int N, const int64_t* dims, const int* R) {
  int best_k = 0;
  double best = 1e300;
  for (int k = 1; k <= N - 2; ++k) {
    const int K = R[0] * R[k];
    if (K > 64) continue;
    double rows = 1, cols = 1;
    for (int j = 0; j < k; ++j) rows *= (double)dims[j];
    for (int j = k; j < N; ++j) cols *= (double)dims[j];
    const double cost = ((k > 1 ? k * rows : 0.0) + (N - k) * cols + rows + cols) * K;
    if (cost < best) { best = cost; best_k = k; }
  }
  return best_k;
}

// Backward by one fused pass over X: Z (prefix side) and W (suffix side), then
// the gradient of each core as the MTTKRP of Z or W over a reduced trace
// problem in which a unit core stands for the other side's product:
//   prefix modes: tensor Z(i_1..i_k, c), cores G_1..G_k, U;
//   suffix modes: tensor W(c, i_{k+1}..i_N), cores V, G_{k+1}..G_N.
// tc: Z and W by the two tensor-core passes (FP32; pl unused), else by the SIMT
// fused pass with plan pl.
static str_status loss_bwd_fused(int N, const int64_t* dims, const str_ctx& t, const LossPlan& pl, bool tc,
                                 const void* const* cores_dev, const void* X_dev, const uint32_t* mask_bits,
                                 double grad_scale, void* const* grad_cores_dev, int64_t rows, int64_t cols,
                                 int kp, int K, size_t es, cudaStream_t s) {
  const int xt = es == 8 ? XT_F64 : XT_F32;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const int64_t nbl = tc ? 0 : (int64_t)pl.nrg * pl.ncg;
  size_t off[7];
  off[0] = 0;                                                          // loss partials
  off[1] = off[0] + al((size_t)nbl * 8);                              // Zpart
  off[2] = off[1] + (tc ? 0 : al((size_t)pl.ncg * rows * K * es));     // Wpart (nrg > 1)
  off[3] = off[2] + (!tc && pl.nrg > 1 ? al((size_t)pl.nrg * cols * K * es) : 0);  // Zt
  off[4] = off[3] + al((size_t)rows * K * es);                         // W
  off[5] = off[4] + al((size_t)cols * K * es);                         // U, V
  off[6] = off[5] + 2 * al((size_t)K * K * es);
  // the reduced MTTKRPs: arguments and the largest partial buffer, before any launch
  std::vector<MttkrpArgs> args;
  std::vector<size_t> part_off;
  size_t part_bytes = 0;
  for (int n = 0; n < N; ++n) {
    if (n < kp && kp == 1) { args.emplace_back(); part_off.push_back(0); continue; }
    MttkrpArgs a;
    a.xtype = xt;
    a.compute = t.compute;
    if (n < kp) {
      a.N = kp + 1;
      a.n = n;
      for (int k = 0; k < kp; ++k) { a.dim[k] = dims[k]; a.core[k] = cores_dev[k]; a.R[k] = t.R[k]; }
      a.dim[kp] = K;
      a.R[kp] = t.R[kp];
      a.R[kp + 1] = t.R[0];
    } else {
      a.N = N - kp + 1;
      a.n = n - kp + 1;
      a.dim[0] = K;
      a.R[0] = t.R[0];
      for (int k = kp; k < N; ++k) { a.dim[k - kp + 1] = dims[k]; a.core[k - kp + 1] = cores_dev[k]; a.R[k - kp + 1] = t.R[k]; }
      a.R[N - kp + 1] = t.R[0];
    }
    int64_t J = 1;
    for (int k = 0; k < a.N; ++k) if (k != a.n) J *= a.dim[k];
    a.nfib = J;
    // small reduced problems: at least 64 fibres per split, about two CTAs per SM
    const int64_t gx = (a.dim[a.n] + 63) / 64;
    const int64_t per = std::max<int64_t>(64, (J * gx + 303) / 304);
    a.fib_per_split = per;
    a.splits = (int)((J + per - 1) / per);
    part_off.push_back(part_bytes);   // each mode its own partials: the modes run concurrently
    part_bytes += al((size_t)a.splits * a.dim[a.n] * a.R[a.n] * a.R[a.n + 1] * es);
    args.push_back(a);
  }
  TRY(ws_grow(3, off[6]));
  // slot 2: the tensor-core passes' split tables and partials, then the reduced
  // MTTKRPs' partials (stream order separates the two uses)
  TRY(ws_grow(2, std::max(part_bytes + 64, tc ? loss_bwd_tc_ws_bytes(rows, cols, K) : (size_t)0)));
  char* b3 = (char*)g_loss_ws[3].p;
  void* Zpart = b3 + off[1];
  void* Zt = b3 + off[3];
  void* W = b3 + off[4];
  void* Wpart = !tc && pl.nrg > 1 ? (void*)(b3 + off[2]) : W;
  void* U = b3 + off[5];
  void* V = b3 + off[5] + al((size_t)K * K * es);
  STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, 0, kp - 1, 0, 0, g_loss_ws[0].p, s));
  STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, kp, N - 1, 0, 1, g_loss_ws[1].p, s));
  if (tc) {
    STR_CUDA_TRY(launch_loss_bwd_tc((const float*)g_loss_ws[0].p, (const float*)g_loss_ws[1].p, rows, cols, K,
                                    (const float*)X_dev, mask_bits, (float*)g_loss_ws[2].p, (float*)Zt, (float*)W,
                                    s));
  } else {
    STR_CUDA_TRY(launch_loss_pass(g_loss_ws[0].p, g_loss_ws[1].p, t.compute, rows, cols, K, X_dev, mask_bits, pl,
                                  true, (double*)(b3 + off[0]), Zpart, Wpart, s));
    STR_CUDA_TRY(launch_loss_reduce(Zpart, pl.ncg, rows, Wpart, pl.nrg, cols, K, t.compute, Zt, W, s));
  }
  STR_CUDA_TRY(launch_unit_cores(t.R[0], t.R[kp], t.compute, U, V, s));
  // the core gradients: mode n on the caller's stream (n = 0) or a side stream
  LossSide* ls = nullptr;
  TRY(loss_side(&ls));
  STR_CUDA_TRY(cudaEventRecord(ls->fork, s));
  bool used[kLossSide] = {};
  for (int n = 0; n < N; ++n) {
    const int side = n == 0 ? -1 : (n - 1) % kLossSide;
    cudaStream_t ss = side < 0 ? s : ls->st[side];
    if (side >= 0 && !used[side]) {
      STR_CUDA_TRY(wait_event(ss, ls->fork));
      used[side] = true;
    }
    if (n < kp && kp == 1) {
      STR_CUDA_TRY(launch_prefix1_grad(Zt, dims[0], K, grad_scale, t.compute, grad_cores_dev[0], ss));
      continue;
    }
    MttkrpArgs a = args[n];
    if (n < kp) { a.X = Zt; a.core[kp] = U; }
    else { a.X = W; a.core[0] = V; }
    a.partial = (char*)g_loss_ws[2].p + part_off[n];
    STR_CUDA_TRY(launch_mttkrp(a, ss));
    STR_CUDA_TRY(launch_reduce_partials_to(a.partial, t.compute, a.splits, a.dim[a.n] * a.R[a.n] * a.R[a.n + 1],
                                           -grad_scale, grad_cores_dev[n], xt, ss));
  }
  for (int i = 0; i < kLossSide; ++i)
    if (used[i]) {
      STR_CUDA_TRY(cudaEventRecord(ls->join[i], ls->st[i]));
      STR_CUDA_TRY(wait_event(s, ls->join[i]));
    }
  return STR_OK;
}

static str_status loss_fwd_body(int N, const int64_t* dims, const int* ranks, str_dtype dtype, const str_ctx& t,
                                const void* const* cores_dev, const void* X_dev, const uint32_t* mask_bits,
                                double* loss_dev, cudaStream_t s);
static str_status loss_bwd_body(int N, const int64_t* dims, const int* ranks, str_dtype dtype, const str_ctx& t,
                                const void* const* cores_dev, const void* X_dev, const uint32_t* mask_bits,
                                double grad_scale, void* const* grad_cores_dev, cudaStream_t s);

str_status tr_masked_loss_fwd(int N, const int64_t* dims, const int* ranks, str_dtype dtype,
                              const void* const* cores_dev, const void* X_dev, const uint32_t* mask_bits,
                              double* loss_dev, void* stream) {
  str_ctx t;
  TRY(loss_setup(N, dims, ranks, dtype, cores_dev, X_dev, &t));
  if (!loss_dev) return STR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  cudaStream_t s = (cudaStream_t)stream;
  bool capturing = false;
  TRY(ws_acquire(s, &capturing));
  const str_status st = loss_fwd_body(N, dims, ranks, dtype, t, cores_dev, X_dev, mask_bits, loss_dev, s);
  const str_status rs = ws_release(s, capturing);
  return st != STR_OK ? st : rs;
}

static str_status loss_fwd_body(int N, const int64_t* dims, const int* ranks, str_dtype dtype, const str_ctx& t,
                                const void* const* cores_dev, const void* X_dev, const uint32_t* mask_bits,
                                double* loss_dev, cudaStream_t s) {
  const int ks = loss_split(N, dims, t.R);
  const int kp = ks > 0 ? ks : N / 2;
  int64_t rows = 1, cols = 1;
  for (int k = 0; k < kp; ++k) rows *= dims[k];
  for (int k = kp; k < N; ++k) cols *= dims[k];
  const int K = ranks[0] * t.R[kp];
  const size_t es = dtype == STR_F64 ? 8 : 4;
  TRY(ws_grow(0, (size_t)rows * K * es));
  TRY(ws_grow(1, (size_t)cols * K * es));
  LossPlan pl;
  if (ks > 0 && t.compute == 1 && loss_fwd_tc_supported(rows, cols, K)) {
    // FP32: the tile reconstructions on the tensor cores, one pass over X
    const int nbl = loss_fwd_tc_blocks(rows, cols);
    TRY(ws_grow(2, (size_t)(nbl + 1) * 8 + 64));
    TRY(ws_grow(3, loss_fwd_tc_split_bytes(rows, cols)));
    STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, 0, kp - 1, 0, 0, g_loss_ws[0].p, s));
    STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, kp, N - 1, 0, 1, g_loss_ws[1].p, s));
    double* part = (double*)g_loss_ws[2].p;
    STR_CUDA_TRY(launch_loss_fwd_tc((const float*)g_loss_ws[0].p, (const float*)g_loss_ws[1].p, rows, cols, K,
                                    (const float*)X_dev, mask_bits, (float*)g_loss_ws[3].p, part, s));
    STR_CUDA_TRY(launch_sum_blocks(part, nbl, 1, part + nbl, 0.5, s));
    STR_CUDA_TRY(cudaMemcpyAsync(loss_dev, part + nbl, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return STR_OK;
  }
  if (ks > 0 && loss_pass_plan(t.compute, rows, cols, K, false, &pl)) {
    // one fused pass over X: per-CTA partial sums of r^2, summed in a fixed order
    const int64_t nbl = (int64_t)pl.nrg * pl.ncg;
    TRY(ws_grow(2, (size_t)nbl * 8 + 64));
    STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, 0, kp - 1, 0, 0, g_loss_ws[0].p, s));
    STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, kp, N - 1, 0, 1, g_loss_ws[1].p, s));
    double* part = (double*)g_loss_ws[2].p;
    STR_CUDA_TRY(launch_loss_pass(g_loss_ws[0].p, g_loss_ws[1].p, t.compute, rows, cols, K, X_dev, mask_bits, pl,
                                  false, part, nullptr, nullptr, s));
    STR_CUDA_TRY(launch_sum_blocks(part, nbl, 1, part + nbl, 0.5, s));
    STR_CUDA_TRY(cudaMemcpyAsync(loss_dev, part + nbl, sizeof(double), cudaMemcpyDeviceToDevice, s));
    return STR_OK;
  }
  TRY(ws_grow(2, (size_t)recon_blocks(rows, cols) * 16 + 64));
  STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, 0, kp - 1, 0, 0, g_loss_ws[0].p, s));
  STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, kp, N - 1, 0, 1, g_loss_ws[1].p, s));
  int64_t nb = 0;
  STR_CUDA_TRY(launch_recon(g_loss_ws[0].p, g_loss_ws[1].p, t.compute, rows, cols, K, RM_LOSS, X_dev,
                            xtype_of(dtype), mask_bits, nullptr, 0, (double*)g_loss_ws[2].p, &nb, s));
  STR_CUDA_TRY(launch_sum_blocks((double*)g_loss_ws[2].p, nb, 2, (double*)g_loss_ws[2].p + 2 * nb, 0.5, s));
  STR_CUDA_TRY(cudaMemcpyAsync(loss_dev, (double*)g_loss_ws[2].p + 2 * nb, sizeof(double), cudaMemcpyDeviceToDevice, s));
  return STR_OK;
}

str_status tr_masked_loss_bwd(int N, const int64_t* dims, const int* ranks, str_dtype dtype,
                              const void* const* cores_dev, const void* X_dev, const uint32_t* mask_bits,
                              double grad_scale, void* const* grad_cores_dev, void* stream) {
  str_ctx t;
  TRY(loss_setup(N, dims, ranks, dtype, cores_dev, X_dev, &t));
  if (!grad_cores_dev) return STR_ERR_INVALID_ARG;
  for (int k = 0; k < N; ++k) if (!grad_cores_dev[k]) return STR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_ws_mu);
  cudaStream_t s = (cudaStream_t)stream;
  bool capturing = false;
  TRY(ws_acquire(s, &capturing));
  const str_status st = loss_bwd_body(N, dims, ranks, dtype, t, cores_dev, X_dev, mask_bits, grad_scale,
                                      grad_cores_dev, s);
  const str_status rs = ws_release(s, capturing);
  return st != STR_OK ? st : rs;
}

static str_status loss_bwd_body(int N, const int64_t* dims, const int* ranks, str_dtype dtype, const str_ctx& t,
                                const void* const* cores_dev, const void* X_dev, const uint32_t* mask_bits,
                                double grad_scale, void* const* grad_cores_dev, cudaStream_t s) {
  const int ks = loss_split(N, dims, t.R);
  const int kp = ks > 0 ? ks : N / 2;
  int64_t rows = 1, cols = 1, count = 1;
  for (int k = 0; k < kp; ++k) rows *= dims[k];
  for (int k = kp; k < N; ++k) cols *= dims[k];
  count = rows * cols;
  const int K = ranks[0] * t.R[kp];
  const size_t es = dtype == STR_F64 ? 8 : 4;
  TRY(ws_grow(0, (size_t)rows * K * es));
  TRY(ws_grow(1, (size_t)cols * K * es));
  LossPlan pl{};
  if (ks > 0 && t.compute == 1 && loss_fwd_tc_supported(rows, cols, K))
    return loss_bwd_fused(N, dims, t, pl, true, cores_dev, X_dev, mask_bits, grad_scale, grad_cores_dev, rows, cols,
                          kp, K, es, s);
  if (ks > 0 && loss_pass_plan(t.compute, rows, cols, K, true, &pl))
    return loss_bwd_fused(N, dims, t, pl, false, cores_dev, X_dev, mask_bits, grad_scale, grad_cores_dev, rows, cols,
                          kp, K, es, s);
  TRY(ws_grow(3, (size_t)count * es));
  STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, 0, kp - 1, 0, 0, g_loss_ws[0].p, s));
  STR_CUDA_TRY(launch_chain_table(cores_dev, t.compute, t.R, N, dims, kp, N - 1, 0, 1, g_loss_ws[1].p, s));
  const int xt = xtype_of(dtype);
  STR_CUDA_TRY(launch_recon(g_loss_ws[0].p, g_loss_ws[1].p, t.compute, rows, cols, K, RM_RESID, X_dev, xt,
                            mask_bits, g_loss_ws[3].p, xt, nullptr, nullptr, s));
  // dL/dG_n = -(M .* residual)_[n] G^{!=n}_[2]: dense MTTKRP of the residual
  for (int n = 0; n < N; ++n) {
    MttkrpArgs a;
    a.X = g_loss_ws[3].p;
    a.xtype = xt;
    a.N = N;
    a.n = n;
    for (int k = 0; k < N; ++k) { a.dim[k] = dims[k]; a.core[k] = cores_dev[k]; }
    for (int k = 0; k <= N; ++k) a.R[k] = t.R[k];
    a.compute = t.compute;
    int64_t J = 1;
    for (int k = 0; k < N; ++k) if (k != n) J *= dims[k];
    a.nfib = J;
    int64_t per = 0;
    a.splits = mttkrp_plan_splits(a, &per);
    a.fib_per_split = per;
    const int RR = t.R[n] * t.R[n + 1];
    // partials share slot 2 (grown to fit)
    TRY(ws_grow(2, (size_t)a.splits * dims[n] * RR * es));
    a.partial = g_loss_ws[2].p;
    STR_CUDA_TRY(launch_mttkrp(a, s));
    STR_CUDA_TRY(launch_reduce_partials_to(a.partial, t.compute, a.splits, dims[n] * RR, -grad_scale,
                                           grad_cores_dev[n], xt, s));
  }
  return STR_OK;
}

}  // extern "C"
