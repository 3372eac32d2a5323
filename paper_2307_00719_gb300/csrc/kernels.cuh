// Internal kernel launchers of the STR / rSTR library (not part of the C ABI).
#pragma once
#include "common.cuh"

// element-storage codes for slabs / intermediates
enum XType : int { XT_BF16 = 0, XT_F32 = 1, XT_F64 = 2, XT_C32 = 3, XT_C64 = 4 };

// ---------------------------------------------------------------------------
// MTTKRP with an on-the-fly subchain:
//   out[split][i_n][c] = sum_{fibres f in split} w_f * X_[n](i_n, f) * S_f(c)
// S_f(c = a + R_n b) = [G_{n+1}(i_{n+1}) ... G_{n-1}(i_{n-1})](b, a)   (Def. subchain)
// Fibres are either every fibre of the slab (dense) or the sampled rows
// idxs(s, k) (Alg. 3).  Complex mode multiplies by conj(S) (KSRFT, Sec. 3.3).
// ---------------------------------------------------------------------------
struct MttkrpArgs {
  const void* X = nullptr;
  int xtype = XT_F32;
  int N = 0, n = 0;                       // order, mode (0-based)
  int64_t dim[STR_MAXN] = {};             // slab sizes I_1..I_{N-1}, t
  const void* core[STR_MAXN] = {};        // compute-type cores, [i][R_{k+1}][R_k]
  int R[STR_MAXN + 1] = {};               // R_1..R_N, R[N] = R[0]
  int64_t nfib = 0;                       // dense: J_n; sampled: m
  const int32_t* idxs = nullptr;          // sampled: idxs[k * m + s]
  int64_t m = 0;
  const double* p[STR_MAXN] = {};         // leverage: w_s = wscale / prod_{k!=n} p_k(idx_k(s))
  int leverage = 0;
  double wscale = 1.0;                    // weight multiplier
  void* partial = nullptr;                // [splits][I_n][RR] compute-type elements
  int splits = 1;
  int64_t fib_per_split = 0;
  void* gs_out = nullptr;                 // sampled: G_S[s][c] (compute type)
  double* ws_out = nullptr;               // sampled: w_s
  int compute = 2;                        // 1 = f32, 2 = f64
  int cplx = 0;
};
int mttkrp_plan_splits(const MttkrpArgs& a, int64_t* fib_per_split);
cudaError_t launch_mttkrp(const MttkrpArgs& a, cudaStream_t s);

// out[i] = (base ? base[i] : 0) + scale * sum_s partial[s][i]   (FP64 sums, fixed order)
// complex partials -> complex FP64 out (interleaved), base ignored.
cudaError_t launch_reduce_partials(const void* partial, int compute, int cplx, int splits,
                                   int64_t count, const double* base, double scale,
                                   double* out, cudaStream_t s);
// same, writing compute-type float output (for gradients) with scale
cudaError_t launch_reduce_partials_to(const void* partial, int compute, int splits, int64_t count,
                                      double scale, void* out, int out_type, cudaStream_t s);

// ---------------------------------------------------------------------------
// Gram of a core unfolding A = G_{(2)} (I x RR):  M = A^T A and its
// transfer-matrix permutation E[(a + Ra a'), (b + Rb b')] = M[a + Ra b, a' + Ra b'].
// ---------------------------------------------------------------------------
cudaError_t launch_core_gram(const double* G, int64_t I, int Ra, int Rb, double* M, double* E,
                             cudaStream_t s);
// C = A(MxK) B(KxN), FP64.  If perm_Ra > 0 the result W (rows (b + Rb b'), cols
// (a + Ra a')) is scattered into Q[(a + Ra b), (a' + Ra b')] = base + W (ring epilogue).
// ring-product GEMM with the permuting epilogue, fused with the FP32 sweep
// inverse of its result (Qout = base + perm(A B); Qf = FP32 copy; W32 = Qf^{-1});
// counter: one device word, zero between launches
cudaError_t launch_gemm64_factor(const double* A, const double* B, double* Qout, int M, int K, int N, int Ra,
                                 int Rb, const double* base, float* Qf, float* Qlo, float* W32, unsigned* counter,
                                 int* status, double* pivot_ratio, cudaStream_t s);
cudaError_t launch_gemm64(const double* A, const double* B, double* C, int M, int K, int N,
                          int perm_Ra, int perm_Rb, const double* base, cudaStream_t s, float* Qhi = nullptr,
                          float* Qlo = nullptr);

// ---------------------------------------------------------------------------
// FP64 LDL^T of an SPD matrix (one CTA, register-blocked): unit lower L and 1/d, pivot check ->
// status.  Rows: out_row = p_row Q^{-1} by substitution; leverage mode: lev[r] = p Q^{-1} p^T / n.
// ---------------------------------------------------------------------------
cudaError_t launch_chol_factor(const double* Q, int n, double* L, double* invdiag, int* status,
                               double* pivot_ratio, cudaStream_t s);
cudaError_t launch_chol_solve(const double* L, const double* invdiag, int n, const double* P,
                              int64_t rows, double* out64, float* out32, double* lev,
                              cudaStream_t s);
cudaError_t launch_fill(double* p, int64_t count, double v, cudaStream_t s);
// FP32 LDL^T factor of Q + FP32 row solves refined `iters` times with FP64 residuals
// (two launches; L32 n x n, invd32 n)
// right-hand side still in split partials: P = base + sum_k part[k] (part: splits x rows x n)
struct PartialSum {
  const float* part = nullptr;
  int splits = 0;
  const double* base = nullptr;   // may be null
  double* pout = nullptr;         // where P is stored
};
// FP32 sweep inverse W32 = Q^{-1} (factor) and the refined solve out = P Q^{-1} (apply);
// with ps, P is formed from the partials inside the apply kernel (and stored to ps->pout)
cudaError_t launch_factor_mixed(const double* Q, int n, float* W32, int* status, double* pivot_ratio,
                                cudaStream_t s);
cudaError_t launch_apply_mixed(const float* W32, const double* Q, int n, const double* P, int64_t rows,
                               int iters, double* out64, float* out32, const PartialSum* ps, cudaStream_t s);
// refined solve with Q as an FP32 pair (n <= 64, even); Q (FP64) -> pair
bool apply_df_supported(int n);
// one refined solve out = P Q^{-1} (FP32 inverse W, Q as an FP32 pair) with the
// FP64 fallback for an ill-conditioned Q (Q64, pivot_ratio, fallbacks)
struct ApplyDF {
  const float* W = nullptr;
  const float* Qh = nullptr;
  const float* Ql = nullptr;
  int n = 0;
  int64_t rows = 0;
  const double* P = nullptr;   // right-hand sides when ps.part is null
  PartialSum ps;
  double* out64 = nullptr;
  float* out32 = nullptr;
  int* status = nullptr;
  const double* Q64 = nullptr;          // FP64 Q for the fallback (null: no fallback)
  const double* pivot_ratio = nullptr;  // written by the FP32 inverse (null: not checked)
  unsigned* fallbacks = nullptr;        // CTAs that took the FP64 fallback (counter)
};
// Q64 (FP64 Q), pivot_ratio (from the FP32 inverse) and fallbacks (counter): the
// FP64 fallback for an ill-conditioned Q (Q64 null = none)
cudaError_t launch_apply_df(const float* W32, const float* Qh, const float* Ql, int n, const double* P, int64_t rows,
                            double* out64, float* out32, const PartialSum* ps, int* status, cudaStream_t s,
                            const double* Q64, const double* pivot_ratio, unsigned* fallbacks);
cudaError_t launch_leverage_dot(const double* G, const double* X, int64_t rows, int n, double* p, cudaStream_t s);
cudaError_t launch_split_pair(const double* Q, int64_t count, float* hi, float* lo, cudaStream_t s);

cudaError_t launch_solve_mixed(const double* Q, int n, const double* P, int64_t rows, int iters,
                               float* L32, float* invd32, double* out64, float* out32, int* status,
                               double* pivot_ratio, cudaStream_t s);

// ---------------------------------------------------------------------------
// sketches
// ---------------------------------------------------------------------------
cudaError_t launch_draw_indices(int32_t* out, int64_t m, int64_t I, uint64_t seed, int k,
                                uint64_t tau, uint32_t stream_id, const double* p, cudaStream_t s);
cudaError_t launch_signs(double* d, int64_t I, uint64_t seed, int k, uint64_t tau,
                         uint32_t stream_id, cudaStream_t s);
// out[c][c'] = base + sum_s w_s Re(g_s[c] conj(g_s[c']))  (FP64 accumulate; sample splits
// reduced in a fixed order; `part` holds 64 x RR x RR doubles)
cudaError_t launch_weighted_gram(const void* gs, int compute, int cplx, const double* w,
                                 int64_t m, int RR, const double* base, double* out, double* part,
                                 cudaStream_t s);
// unitary DFT with sign pre-multiply along mode `mode` of a tensor with dims[N]:
// out(.., k, ..) = sum_i F(k, i) d_i in(.., i, ..),  F(k,i) = exp(-2 pi i k i / L) / sqrt(L)
cudaError_t launch_dft_mode(const void* in, int in_type, void* out, int out_cplx_compute, int N,
                            const int64_t* dims, int mode, const double* d, cudaStream_t s);
// out[k][c] = base[k][c] + Re( d_k * sum_i conj(F(i, k)) Y[i][c] )  (unmix rows, Y complex FP64)
cudaError_t launch_unmix_rows(const double* Y, int64_t L, int RR, const double* d,
                              const double* base, double* out, cudaStream_t s);

// ---------------------------------------------------------------------------
// utilities
// ---------------------------------------------------------------------------
cudaError_t launch_convert(const void* in, int in_type, void* out, int out_type, int64_t count,
                           cudaStream_t s);
cudaError_t launch_check_finite(const void* X, int xtype, int64_t count, int* status,
                                cudaStream_t s);

// ---------------------------------------------------------------------------
// reconstruction / fit error / masked loss (TR format, Sec. 1)
//   Xhat[row + rows*col] = sum_c Lm[row][c] Rm[col][c]
// ---------------------------------------------------------------------------
// table[j][a + Rf * b] = [G_{k0}(i_{k0}) ... G_{k1}(i_{k1})](a, b)   (transpose=0)
// table[j][a + Rl * b] = [..](b, a)  with Rl the last right rank    (transpose=1)
// j runs over (i_{k0}, .., i_{k1}) with i_{k0} fastest.  core k0 may start at row t_off.
cudaError_t launch_chain_table(const void* const* cores, int compute, const int* R, int N,
                               const int64_t* dims, int k0, int k1, int64_t row_off_last,
                               int transpose, void* table, cudaStream_t s);
enum ReconMode : int { RM_WRITE = 0, RM_FIT = 1, RM_LOSS = 2, RM_RESID = 3 };
cudaError_t launch_recon(const void* Lm, const void* Rm, int compute, int64_t rows, int64_t cols,
                         int K, int mode, const void* X, int xtype, const uint32_t* mask,
                         void* out, int out_type, double* block_sums, int64_t* nblocks,
                         cudaStream_t s);
cudaError_t launch_sum_blocks(const double* block_sums, int64_t nblocks, int width, double* out,
                              double scale, cudaStream_t s);
int recon_blocks(int64_t rows, int64_t cols);
// fused masked-loss pass (one read of X): loss partials [nrg][ncg]; with bwd also
// Zpart [ncg][rows][K] (sum over columns of r Rm) and Wpart [nrg][cols][K] (sum
// over rows of r Lm); K <= 64
struct LossPlan {
  int RG = 64, nrg = 1, ncg = 1;
  int64_t cb_per = 1;
  size_t smem = 0;
};
bool loss_pass_plan(int compute, int64_t rows, int64_t cols, int K, bool bwd, LossPlan* pl);
// masked-loss forward on the tensor cores (FP32 tables and X, K <= 64): per-CTA
// partial sums of M (X - Lm Rm^T)^2 in loss_part[loss_fwd_tc_blocks()]; `split`
// holds loss_fwd_tc_split_bytes() of TF32-split tables
bool loss_fwd_tc_supported(int64_t rows, int64_t cols, int K);
size_t loss_fwd_tc_split_bytes(int64_t rows, int64_t cols);
int loss_fwd_tc_blocks(int64_t rows, int64_t cols);
cudaError_t launch_loss_fwd_tc(const float* Lm, const float* Rm, int64_t rows, int64_t cols, int K, const float* X,
                               const uint32_t* mask, float* split, double* loss_part, cudaStream_t s);
// masked-loss backward contractions on the tensor cores (same support as the
// forward): Zt[k][row] = sum_c R(row, c) Rm[c][k] and W[c][k] = sum_row R(row, c)
// Lm[row][k] of R = M .* (X - Lm Rm^T), by two passes over X; ws holds
// loss_bwd_tc_ws_bytes() (split tables and per-CTA partials)
size_t loss_bwd_tc_ws_bytes(int64_t rows, int64_t cols, int K);
// the driver's cuTensorMapEncodeTiled, resolved once through the runtime (null if absent)
void* str_tensor_map_encoder();
cudaError_t launch_loss_bwd_tc(const float* Lm, const float* Rm, int64_t rows, int64_t cols, int K, const float* X,
                               const uint32_t* mask, float* ws, float* Zt, float* W, cudaStream_t s);
cudaError_t launch_loss_pass(const void* Lm, const void* Rm, int compute, int64_t rows, int64_t cols, int K,
                             const void* X, const uint32_t* mask, const LossPlan& pl, bool bwd,
                             double* loss_part, void* Zpart, void* Wpart, cudaStream_t s);
// Zt[c][row] = sum of the column-group partials; W = sum of the row-group partials
// (skipped when nrg == 1: the pass wrote W itself)
cudaError_t launch_loss_reduce(const void* Zpart, int ncg, int64_t rows, const void* Wpart, int nrg, int64_t cols,
                               int K, int compute, void* Zt, void* W, cudaStream_t s);
// unit cores U, V (K x K each, core layout) of the reduced trace problems
cudaError_t launch_unit_cores(int R1, int Rk, int compute, void* U, void* V, cudaStream_t s);
cudaError_t launch_prefix1_grad(const void* Zt, int64_t I, int K, double scale, int compute, void* grad,
                                cudaStream_t s);

// ---------------------------------------------------------------------------
// tensor-core dense MTTKRP (k_tc.cu): stage 1 Y = X x_k G_k on tcgen05,
// stage 2 contraction of Y with the chain tables of the other cores
// ---------------------------------------------------------------------------
struct Stage2Args {
  const float* Y = nullptr;    // M x (R_k R_{k+1}), row m = i_lo + Jlo (i_n + dn i_hi)
  const float* TA = nullptr;   // [i_hi][R_{n+1} x R_k]  (nullptr = identity)
  const float* TB = nullptr;   // [i_lo (k = 0) or i_hi (k = 1)][R_{k+1} x R_n]  (nullptr = identity)
  int Rk = 0, Rk1 = 0, Rn = 0, Rn1 = 0;
  int k = 0;
  int64_t dn = 0, Jlo = 1, Jhi = 1;
  float* partial = nullptr;    // [splits][dn][R_n R_{n+1}]
  int splits = 1;
  int64_t per = 1;             // combinations per split
};
bool tc_supported(int K, int xtype, const void* base);
size_t stage1_smem_bytes(int Npad);
cudaError_t launch_prep_b(const double* G, int K, int N, int Kpad, int Npad, float* Bhi, float* Blo,
                          cudaStream_t s);
cudaError_t launch_transpose01(const void* in, void* out, int xtype, int d0, int d1, int64_t rest,
                               cudaStream_t s);
cudaError_t launch_stage1_tc(const void* Xa, int xtype, int64_t M, int K, const float* Bhi,
                             const float* Blo, int Kpad, int N, int Npad, float* Y, int* status,
                             cudaStream_t s);
// sampled MTTKRP on the tensor cores: rows of G_S (+ weights, + split GEMM operand
// B^T [Npad][Kpad], zero-filled by the caller), the gathered fibres A [I_n][Kpad],
// and the split-K GEMM (partials [splits][M][N])
cudaError_t launch_sampled_rows(const MttkrpArgs& a, int Kpad, float* Bhi, float* Blo, cudaStream_t s);
cudaError_t launch_gather_fibres(const MttkrpArgs& a, int Kpad, void* A, cudaStream_t s);
// complex samples (KSRFT): B operands of Re P and Im P, A = [Re X_S | Im X_S] over
// K' = 2 Kpad, and the pairwise sum of the two split-K partial sets into complex FP64
cudaError_t launch_sampled_rows_cplx(const MttkrpArgs& a, int Kpad, float* Brh, float* Brl, float* Bih, float* Bil,
                                     cudaStream_t s);
cudaError_t launch_gather_fibres_cplx(const MttkrpArgs& a, int Kpad, float* A, cudaStream_t s);
cudaError_t launch_reduce_cplx_pair(const float* Pre, const float* Pim, int splits, int64_t count, double* out,
                                    cudaStream_t s);
cudaError_t launch_gemm_tc_splitk(const void* A, int xtype, int64_t M, int Kpad, const float* Bhi,
                                  const float* Blo, int N, int Npad, int splits, float* Y, int* status,
                                  cudaStream_t s);
int gemm_tc_splitk_count(int Kpad, int splits);
int stage2_plan_splits(const Stage2Args& a, int64_t* per);
cudaError_t launch_stage2(const Stage2Args& a, cudaStream_t s);

// ---------------------------------------------------------------------------
// work lists for batched updates of many independent streams: each launch
// covers every stream; block b runs item b, which names a job (one stream's
// problem) and the tile of it this block computes.  Jobs and items live in
// device memory (built once per batch layout).
// ---------------------------------------------------------------------------
struct GramJob {                 // E = transfer form of G_{(2)}^T G_{(2)} (core_gram)
  const double* G = nullptr;
  int64_t I = 0;
  int Ra = 0, Rb = 0;
  double* E = nullptr;
  int chunk = 1;                 // rows staged per pass (core_gram_chunk)
};
int core_gram_chunk(int64_t I, int RR);
int core_gram_blocks(int RR);
cudaError_t launch_core_gram_batch(const GramJob* jobs, const int2* items, int nitems, cudaStream_t s);

struct GemmJob {                 // C = A B (M x K x N), ring epilogue when pRa > 0
  const double* A = nullptr;
  const double* B = nullptr;
  double* C = nullptr;
  int M = 0, K = 0, N = 0, pRa = 0, pRb = 0;
  const double* base = nullptr;
  float* Qf = nullptr;
  float* Qlo = nullptr;
};
cudaError_t launch_gemm64_batch(const GemmJob* jobs, const int4* items, int nitems, int Kmax, cudaStream_t s);

struct SweepJob {                // W = Q^{-1} by the FP32 sweep (order <= 128)
  const double* Q = nullptr;
  int n = 0;
  float* W = nullptr;
  int* status = nullptr;
  double* pivot_ratio = nullptr;
};
cudaError_t launch_sweep_batch(const SweepJob* jobs, int njobs, cudaStream_t s);

// dense SIMT MTTKRP jobs of one register-block class (mttkrp_class): item =
// (job, row block, split, stream); the job's slab is xptrs[stream] (the slab
// pointer changes every step, the jobs do not)
int mttkrp_class(const MttkrpArgs& a);
size_t mttkrp_smem_bytes(const MttkrpArgs& a, int BK);
int mttkrp_rows_per_block(const MttkrpArgs& a);
cudaError_t launch_mttkrp_batch(const MttkrpArgs* jobs, const int4* items, const void* const* xptrs, int nitems,
                                int cls, int xtype, int BK, size_t smem, cudaStream_t s);
// out[i] = *ptrs[i] for i < n
cudaError_t launch_gather_ints(const int* const* ptrs, int n, int* out, cudaStream_t s);

struct ReduceJob {               // out = base + sum of FP32 split partials (reduce order of launch_reduce_partials)
  const float* partial = nullptr;
  int splits = 1;
  int64_t count = 0;
  const double* base = nullptr;
  double* out = nullptr;
};
cudaError_t launch_reduce_batch(const ReduceJob* jobs, const int2* items, int nitems, cudaStream_t s);

// refined solves, all of order <= nmax (<= 128): item = (job, block, blocks of the job)
cudaError_t launch_apply_df_batch(const ApplyDF* jobs, const int4* items, int nitems, int nmax, cudaStream_t s);

struct RefineJob {               // out = P Q^{-1} for orders 129..160: FP32 inverse W, FP64 residual
  const float* W = nullptr;
  const double* Q = nullptr;
  int n = 0;
  const double* P = nullptr;
  int64_t rows = 0;
  int iters = 1;
  int q_in_smem = 0;
  double* out64 = nullptr;
  float* out32 = nullptr;
  PartialSum ps;
};
int refine_q_in_smem(int n);
size_t refine_smem(int n, int q_in_smem);
cudaError_t launch_refine_batch(const RefineJob* jobs, const int4* items, int nitems, int nmax, size_t smem,
                                cudaStream_t s);

struct CopyJob {                 // dst = src, bytes (16-byte aligned: both multiples of 16 or plain)
  const void* src = nullptr;
  void* dst = nullptr;
  int64_t bytes = 0;
};
cudaError_t launch_copy_batch(const CopyJob* jobs, const int2* items, int nitems, cudaStream_t s);
