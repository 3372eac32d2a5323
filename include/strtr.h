/*
 * strtr.h -- C ABI of the GB300 streaming tensor-ring (STR / rSTR) library.
 *
 * The library tracks the tensor-ring (TR) decomposition of a tensor that grows
 * along its last (temporal) mode, following Yu & Li, "Tracking Tensor Ring
 * Decompositions of Streaming Tensors": STR (Alg. 4) and rSTR (Alg. 5 with
 * the uniform, leverage-based and KSRFT schedules of Algs. 7-9).  Every step of
 * an update runs in this library's CUDA kernels; the caller supplies device
 * memory and a CUDA stream.
 *
 * Conventions shared by every call
 * --------------------------------
 * - Order N >= 3.  Modes 1..N-1 are spatial with fixed sizes I_1..I_{N-1};
 *   mode N is time.  TR-ranks R_1..R_N, R_{N+1} = R_1, 1 <= R_n <= 16 and
 *   R_n R_{n+1} <= 160.
 * - Tensors are dense with the paper's linear index (Sec. 2): element
 *   (i_1, .., i_N) sits at offset i_1 + I_1 (i_2 + I_2 (i_3 + ...)), i.e. i_1
 *   fastest.  A torch tensor of shape (t, I_{N-1}, .., I_1) is such a buffer.
 * - Core n is stored as the unfolding G_{n(2)} (Sec. 2, TR-ALS) in row-major
 *   order: element G_n(r_n, i_n, r_{n+1}) at offset
 *       i_n * R_n R_{n+1} + r_{n+1} * R_n + r_n.
 * - Pointers are device pointers unless a field or argument says "host".
 *   Input buffers are borrowed for the duration of the call on the given
 *   stream; the library keeps no reference to them.  Work is enqueued on
 *   `stream` (a cudaStream_t; NULL = the legacy default stream).
 * - Every call returns a str_status.  STR_OK = 0.  Unless a call says
 *   otherwise, a failing call leaves the context unchanged.
 * - Thread safety: one context must not be used by two host threads at once.
 */
#ifndef STRTR_H
#define STRTR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct str_ctx str_ctx;

typedef enum {
  STR_OK = 0,
  STR_ERR_INVALID_ARG = 1,  /* NULL pointer, bad enum, negative size */
  STR_ERR_SHAPE = 2,        /* order, dims or ranks outside the supported range */
  STR_ERR_DTYPE = 3,        /* unsupported element type for this call */
  STR_ERR_SINGULAR = 4,     /* a normal-equation matrix had a pivot too small to factor or invert */
  STR_ERR_NONFINITE = 5,    /* NaN/Inf found in a slab (only when check_finite is on) */
  STR_ERR_CAPACITY = 6,     /* the temporal core would exceed t_capacity rows */
  STR_ERR_OOM = 7,          /* device allocation failed */
  STR_ERR_CUDA = 8,         /* a CUDA runtime call failed; see str_last_error() */
  STR_ERR_TIMEOUT = 9,      /* a bounded device wait gave up */
  STR_ERR_STATE = 10        /* call not valid in the context's state */
} str_status;

typedef enum { STR_BF16 = 0, STR_F32 = 1, STR_F64 = 2 } str_dtype;

typedef enum {
  STR_SKETCH_NONE = -1,     /* exact STR (Alg. 4) */
  STR_SKETCH_UNIFORM = 0,   /* rSTR-U (Alg. 7) */
  STR_SKETCH_LEVERAGE = 1,  /* rSTR-L (Alg. 8) */
  STR_SKETCH_KSRFT = 2      /* rSTR-K (Alg. 9) */
} str_sketch;

/* A dense tensor in the linear layout above. */
typedef struct {
  const void* data;       /* element (0,..,0); 16-byte aligned recommended */
  str_dtype dtype;        /* STR_BF16, STR_F32 or STR_F64 */
  int order;              /* N */
  const int64_t* dims;    /* host array of N sizes I_1..I_{N-1}, t */
  int on_host;            /* 0 = device memory; 1 = host memory (copied in by the call) */
} str_tensor;

typedef struct {
  /* Precision of the slab-side arithmetic (subchain products, MTTKRP,
   * sampled products, DFT mixing): STR_F64 or STR_F32 (FP32 accumulate).
   * Gram tensors, Q_n, P_n accumulation and every solve are FP64. */
  str_dtype compute;
  int sweeps;              /* >= 1; passes over each slab per update (1 = Alg. 4) */
  int rescale;             /* rSTR: 1 = apply the sketch rescaling D (Eq. sampDS), 0 = omit it */
  int64_t t_capacity;      /* maximum temporal rows kept in G_N (default 65536) */
  int init_max_it;         /* str_init: TR-ALS-NE iterations (default 100, Sec. 4) */
  double init_tol;         /* str_init: stop when |change of rel. error| < tol (default 1e-8) */
  str_sketch sketch;       /* STR_SKETCH_NONE = STR; else the rSTR sketch fixed at init */
  int64_t m;               /* rSTR sketch size (rows drawn per mode) */
  uint64_t seed;           /* rSTR Philox key */
  uint32_t stream_id;      /* rSTR Philox stream word (independent streams of draws) */
  int check_finite;        /* 1 = scan each slab for NaN/Inf first (STR_ERR_NONFINITE) */
  int async_status;        /* 0 = each update synchronises and returns device errors
                            *     (state unchanged on error);
                            * 1 = no synchronisation; device errors surface at the next
                            *     call or str_sync() and then make the context sticky-failed */
  int profile;             /* 1 = time every kernel launch with CUDA events on the launch
                            *     stream (per-class totals in str_stats) */
  int mttkrp_path;         /* dense FP32-compute MTTKRP: 0 = tensor cores (tcgen05) where the
                            *     slab layout allows it, else SIMT; 1 = SIMT only */
  int graphs;              /* 1 (default) = str_update replays a captured CUDA graph of its
                            *     kernels once a slab shape has been seen; the slab is then
                            *     first copied to a library-owned buffer.  Not used while
                            *     profiling or on the legacy default stream (NULL).
                            *     0 = plain stream launches */
} str_options;

/* Fills *opt with the defaults listed above (compute F64, sweeps 1, rescale 1,
 * sketch NONE, m 1000, seed 0).  Returns STR_ERR_INVALID_ARG for NULL. */
str_status str_default_options(str_options* opt);

/*
 * str_init -- initialisation stage of Alg. 4 / Alg. 5.
 * Computes the initial cores of X0 by TR-ALS-NE (Alg. 2; stops per
 * opt->init_tol / init_max_it, Sec. 4) from the host FP64 initial guess
 * `guess` (N pointers, core n with I_n rows, the temporal one with t_init
 * rows), then P_n = X0_[n] G^{!=n}_[2] and Q_n = (H^{!=n})_<2> (the
 * initialisation of Alg. 4) or their sketched forms (Alg. 5, draws at tau = 0).
 *   out    : receives the new context (owns all device state); *out = NULL on error
 *   X0     : initial tensor I_1 x .. x I_{N-1} x t_init (device or host)
 *   ranks  : host array R_1..R_N
 *   guess  : host array of N host pointers to FP64 cores in the core layout
 *   opt    : NULL = defaults
 */
str_status str_init(str_ctx** out, const str_tensor* X0, const int* ranks,
                    const double* const* guess, const str_options* opt, void* stream);

/*
 * str_init_cores -- as str_init, but takes the initial cores as given (host
 * FP64, N pointers in the core layout, the temporal core with t_init rows) and
 * only builds P_n, Q_n from X0 (Alg. 4; Alg. 5).
 * X0 may be NULL: then P_n = 0 and Q_n = 0 (no history) and t_init = the
 * temporal core's row count `t_init`.
 */
str_status str_init_cores(str_ctx** out, int N, const int64_t* dims, const int* ranks,
                          int64_t t_init, const double* const* cores, const str_tensor* X0,
                          const str_options* opt, void* stream);

/*
 * str_update -- one time step of STR (Alg. 4): the temporal core's
 * new rows G_N^new = X^new_[N] G^{!=N}_[2] (H^{!=N}_<2>)^dagger are appended,
 * then for n = 1..N-1: P_n += X^new_[n] (G^{!=n}_new)_[2], Q_n += (H^{!=n}_new)_<2>,
 * G_{n(2)} = P_n Q_n^dagger.  With opt.sweeps = s > 1 the step is repeated s
 * times from the same P_n, Q_n (each sweep recomputes G_N^new with the latest
 * cores).  X_new: I_1 x .. x I_{N-1} x t_new, t_new >= 1, any dtype.
 * Works on any context (also one initialised for rSTR).
 */
str_status str_update(str_ctx* ctx, const str_tensor* X_new, void* stream);

/*
 * rstr_update -- one time step of rSTR (Alg. 5) with the draw schedule of
 * Alg. 7 (uniform), Alg. 8 (leverage) or Alg. 9 (KSRFT).  `type`, `m` and
 * `seed` must equal the values the context was initialised with
 * (STR_ERR_STATE otherwise).  Sample indices come from the Philox4x64-10
 * contract: key (seed, 0), counter (s, k, tau, purpose<<32 | stream_id).
 */
str_status rstr_update(str_ctx* ctx, const str_tensor* X_new, str_sketch type, int64_t m,
                       uint64_t seed, void* stream);

/*
 * str_update_batch -- updates `count` independent contexts with one slab each.
 * randomized = 0: str_update semantics; 1: rstr_update with each context's own
 * sketch settings.  On error no context is changed (sync mode).
 * Work-list form (randomized = 0, every context of order 3 with FP32 slab
 * arithmetic, one sweep, R_n R_{n+1} <= 160, not profiling): one fixed sequence
 * of about 30 launches per step updates every context together, each launch
 * covering all of them (core Grams, ring products, FP32 inverses, the dense
 * SIMT MTTKRP, split reductions, refined solves, appends); the sequence is
 * captured into a CUDA graph when the same batch recurs on a non-default
 * stream, and the staging chunk and solve rows per block are autotuned once per
 * shape signature by timing candidates (the first call of a new shape
 * signature synchronises).  Results are bit-identical to one str_update per
 * context wherever that update takes the SIMT MTTKRP (FP64 slabs, mttkrp_path
 * = 1, or slab layouts the tensor-core path does not take); otherwise they
 * differ by FP32 rounding.  Status words of all contexts are read with one
 * synchronisation per call.
 * Otherwise, on a non-default stream every context's update runs as one branch,
 * forked from `stream` and joined back to it, so the updates run concurrently;
 * for randomized = 0 a batch that recurs (same contexts, slab shapes and buffer
 * parities) is captured once into a CUDA graph and replayed (rSTR steps take
 * the step number as a launch argument and are not captured).  Slabs are
 * staged at each context's own device address (a device-to-device copy).  On
 * the legacy default stream the updates run one after another on `stream`.
 * These forms are bit-identical to one str_update (or rstr_update) per context.
 */
str_status str_update_batch(str_ctx* const* ctxs, const str_tensor* const* X_new, int count,
                            int randomized, void* stream);

/*
 * tr_reconstruct -- writes TR(G) (Sec. 1) for temporal rows [t0, t1) into `out`
 * (device, I_1 x .. x I_{N-1} x (t1-t0), dtype STR_F32 or STR_F64).
 */
str_status tr_reconstruct(const str_ctx* ctx, int64_t t0, int64_t t1, void* out, str_dtype dtype,
                          void* stream);

/*
 * tr_fit_error -- relative error ||X - TR(G)||_F / ||X||_F (Sec. 4) over the
 * temporal rows [t0, t0 + t) that X covers, by the direct residual with FP64
 * sums.  Synchronises the stream; *rel_err is a host double.
 */
str_status tr_fit_error(const str_ctx* ctx, const str_tensor* X, int64_t t0, double* rel_err,
                        void* stream);

/* Copies core n (1-based) to host FP64 in the core layout; the temporal core
 * (n = N) has str_num_time_rows() rows.  Synchronises. */
str_status str_get_core(const str_ctx* ctx, int n, double* host_out);
/* Number of temporal rows currently held (t_init + all appended rows). */
int64_t str_num_time_rows(const str_ctx* ctx);
/* Copies P_n (I_n x R_nR_{n+1}) and Q_n (R_nR_{n+1} square), n = 1..N-1, to host FP64. */
str_status str_get_pq(const str_ctx* ctx, int n, double* host_P, double* host_Q);
/* rSTR: copies idxs(:,k) (m zero-based int64 indices) and, for rSTR-L, p_k
 * (host_p may be NULL) of mode k (1-based).  Synchronises. */
str_status str_get_samples(const str_ctx* ctx, int k, int64_t* host_idxs, double* host_p);

/* Serialises the whole state (shapes, options, cores, P_n, Q_n, step counter,
 * sample indices, leverage distributions) into `buf`.  If buf is NULL, *len
 * receives the required size.  str_load rebuilds a context from such a buffer;
 * updates after a load are bit-identical to an uninterrupted run. */
str_status str_save(const str_ctx* ctx, void* buf, size_t* len);
str_status str_load(str_ctx** out, const void* buf, size_t len, void* stream);

/* kernel classes of the per-class profile counters */
enum {
  STR_K_MTTKRP = 0,   /* slab MTTKRP: tensor-core stage 1, or the SIMT kernel (sampled, FP64) */
  STR_K_REDUCE = 1,   /* fixed-order split reduction into P_n */
  STR_K_GRAM = 2,     /* core Gram and ring contraction */
  STR_K_FACTOR = 3,   /* factorisation or inverse of Q_n (with the fused ring product) */
  STR_K_SOLVE = 4,    /* triangular row solves, leverage scores */
  STR_K_SKETCH = 5,   /* draws, sign flips, weighted sampled Gram */
  STR_K_DFT = 6,      /* KSRFT mixing / unmixing */
  STR_K_OTHER = 7,    /* conversions, reconstruction, checks */
  STR_K_CONTRACT = 8, /* tensor-core MTTKRP stage 2: contraction with the chain tables */
  STR_K_CLASSES = 9
};

typedef struct {
  int64_t steps;            /* updates committed */
  int64_t time_rows;        /* temporal rows held */
  int64_t kernel_launches;  /* kernels launched by the last update */
  int64_t device_bytes;     /* device memory owned by the context */
  double min_pivot_ratio;   /* pivot / diagonal ratio (min over pivots) of the last factorisation of
                             * the last update's solves (0 for a pivot too small to use) */
  int64_t class_launches[STR_K_CLASSES];  /* with opt.profile: launches per class */
  double class_ms[STR_K_CLASSES];         /* with opt.profile: summed event time per class */
  int64_t fp64_fallbacks;   /* FP32 slab arithmetic: row blocks (CTAs) of the refined solves, since
                             * the context was created, that took the FP64 fallback because Q_n was
                             * too ill-conditioned for the FP32 inverse (pivot / diagonal ratio
                             * below 2^-13, or a first refinement correction above 1e-3 of the
                             * solution); their rows are solved with an FP64 inverse and one FP64
                             * refinement step.  Orders R_n R_{n+1} > 128 have no fallback. */
} str_stats;
/* Fills *stats.  The profile counters cover the launches since the previous
 * str_get_stats call (they are reset by it); reading them waits for those
 * launches to finish. */
str_status str_get_stats(const str_ctx* ctx, str_stats* stats);

/* Waits for the context's queued work and reports a pending device error. */
str_status str_sync(str_ctx* ctx);

const char* str_status_string(str_status s);
/* Text of the last CUDA error seen by this thread (empty if none). */
const char* str_last_error(void);
void str_destroy(str_ctx* ctx);

/*
 * Masked TR fit loss (no counterpart in the paper; used for gradient-based
 * fitting):  L = 1/2 sum_i M(i) (X(i) - TR(G)(i))^2, with M(i) = bit i of
 * mask_bits (1 = observed; NULL = all observed), bit b of word w covering
 * linear index 32 w + b.  Cores and X are device arrays of `dtype` (STR_F32 or
 * STR_F64); dims has N entries (the last one is the temporal size).
 *   tr_masked_loss_fwd writes L (FP64) to the device double *loss_dev.
 *   tr_masked_loss_bwd writes grad_scale * dL/dG_n into grad_cores_dev[n]
 *   (device, core layout, same dtype): dL/dG_{n(2)} = -(M .* (X - TR(G)))_[n] G^{!=n}_[2]
 *   (with M == 1 this equals G_{n(2)} Q_n - P_n of Eq. partial).
 * Both recompute the subchains; nothing is stored between them.  With the
 * modes split into a prefix and a suffix such that K = R_1 R_{k+1} <= 64, the
 * loss takes one pass over X (and the mask), and the backward forms the sums of
 * the masked residual against the suffix and prefix products, from which every
 * core gradient follows as a small MTTKRP; otherwise the residual is formed
 * in a scratch buffer first.  FP32: the forward reconstructs each 128 x 128 tile
 * of X on the tensor cores (TF32 with a 3-term split), and the backward takes
 * two passes over X, each reconstructing a tile, forming the residual and
 * contracting it on the tensor cores without writing it to memory; FP64: one
 * fused pass gives both sums.  The backward's per-core MTTKRPs run on
 * library-owned streams, forked from and joined back into `stream` by events
 * (under stream capture they become branches of the captured graph).  A device
 * wait that gives up makes the loss or the gradients NaN.  Results are reduced
 * in a fixed order
 * (deterministic for a given shape).  Scratch is library-owned (grow-only,
 * shared by all calls of the process): a host lock serialises the enqueueing,
 * and each call's stream first waits for the previous call's last use of the
 * scratch (a library event), so calls issued on different streams do not
 * overlap on the GPU.  Under stream capture that wait is not recorded and the
 * caller must order captured loss calls against others itself.
 */
str_status tr_masked_loss_fwd(int N, const int64_t* dims, const int* ranks, str_dtype dtype,
                              const void* const* cores_dev, const void* X_dev,
                              const uint32_t* mask_bits, double* loss_dev, void* stream);
str_status tr_masked_loss_bwd(int N, const int64_t* dims, const int* ranks, str_dtype dtype,
                              const void* const* cores_dev, const void* X_dev,
                              const uint32_t* mask_bits, double grad_scale,
                              void* const* grad_cores_dev, void* stream);

/*
 * tr_masked_loss_fwd_noalloc -- the paper has no counterpart; this is a service
 * entry point of the library.  Same arguments and result as
 * tr_masked_loss_fwd, but it allocates no device memory, for callers that
 * cannot call cudaMalloc: code whose framework allocator owns all device
 * memory (a raw cudaMalloc bypasses its budget and can fail once it has taken
 * the free memory), and latency-critical loops that cannot take cudaMalloc's
 * device synchronisation.
 * Its scratch is one fixed 32 MiB array in device global memory (held by every
 * GPU that loads the library until the process exits).  A problem whose
 * scratch does not fit, or whose 64 x 64 output blocks exceed the grid limits,
 * returns STR_ERR_SHAPE before launching anything (str_last_error() says why).
 * The modes are split into a prefix 1..N/2 and a suffix; the value agrees with
 * tr_masked_loss_fwd (which may split elsewhere) to rounding.  All calls share that array: calls that
 * overlap on the GPU (other streams or host threads) race.  The first call on
 * each device looks up the array's address with that device current; make it
 * before any stream capture.
 */
str_status tr_masked_loss_fwd_noalloc(int N, const int64_t* dims, const int* ranks,
                                      str_dtype dtype, const void* const* cores_dev,
                                      const void* X_dev, const uint32_t* mask_bits,
                                      double* loss_dev, void* stream);

/*
 * str_fma_probe -- measurement utility; the paper has no counterpart.  Enqueues
 * one kernel of `ctas` blocks of 256 threads in which every thread runs
 * `iters` rounds of 32 fused multiply-adds of `dtype` (STR_F32 or STR_F64) in
 * eight independent chains, and writes one sum per block to `out` (device,
 * `ctas` elements of dtype, caller-owned).  *flop (host) receives the launch's
 * floating-point operations, 64 * iters * 256 * ctas.  Timing the launch with
 * CUDA events on `stream` gives the FMA pipe's rate, the denominator of the
 * roofline for work on the FP32 or FP64 pipes.  STR_ERR_INVALID_ARG for NULL
 * pointers or non-positive sizes, STR_ERR_DTYPE for other types.
 */
str_status str_fma_probe(str_dtype dtype, int ctas, int64_t iters, void* out, double* flop, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* STRTR_H */
