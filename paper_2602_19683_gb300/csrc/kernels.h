// Host-visible declarations of the device kernels (internal to libgp).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace gpk {

// Task kinds of the persistent DAG kernel (int4 {kind, p, q, r}).
enum TaskKind {
  TASK_POTRF = 0,   // (J)        L_JJ = Chol(K_JJ)                      Sec. 3.2 POTRF
  TASK_TRSM = 1,    // (I, J)     L_IJ = K_IJ L_JJ^{-T}                  Sec. 3.2 TRSM
  TASK_UPD = 2,     // (I, K, J)  K_IK -= L_IJ L_KJ^T (SYRK when I == K) Sec. 3.2 SYRK/GEMM
  TASK_VTRSM = 3,   // (J, c)     V_Jc = L_JJ^{-1} V_Jc                  Eq. (3), L V = K_{X,Xs}
  TASK_VGEMM = 4,   // (I, J, c)  V_Ic -= L_IJ V_Jc
  TASK_WSYRK = 5,   // (a, b, J)  S_ab -= V_Ja^T V_Jb                    Eq. (3), cov = K_{Xs,Xs} - V^T V
  TASK_FSOLVE = 6,  // (J)        b_J = L_JJ^{-1} b_J                    Eq. (2), L beta = y
  TASK_FGEMV = 7,   // (I, J, ch) b_I[ch] -= L_IJ[ch,:] b_J
  TASK_BSOLVE = 8,  // (J)        b_J = L_JJ^{-T} b_J                    Eq. (2), L^T alpha = beta
  TASK_BGEMV = 9,   // (J, I, ch) b_J[ch] -= L_IJ[:,ch]^T b_I
  // Reverse sweep of the tiled Cholesky (the adjoint of Fig. 1's algorithm, for the NLML gradient):
  // Lbar -> Kbar tile by tile, columns J = Mt-1 .. 0. Bt holds Lbar, then Abar (the adjoint of K's
  // stored lower entries; a diagonal tile holds Abar + Abar^T).
  TASK_RUPD = 10,   // (P, K, J)  Lbar_PJ -= Abar~_PK L_KJ    (reverse of step J's SYRK/GEMM updates)
  TASK_RTRSM = 11,  // (P, J)     Abar_PJ = Lbar_PJ L_JJ^{-1} (reverse of TRSM(P, J))
  TASK_RDIAG = 12,  // (P, J)     Lbar_JJ -= tril(Abar_PJ^T L_PJ)
  TASK_RPOTRF = 13,  // (J)       Abar_JJ = sym(L^{-T} Phi(L^T Lbar_JJ) L^{-1})  (reverse of POTRF(J))
  // Inverse of a factored diagonal tile, kept for the vector solves of Eq. (2) (each diagonal-block
  // solve becomes a matrix-vector product; not a step of the paper, which solves by substitution).
  TASK_TRTRI = 14,   // (J)        Linv_J = L_JJ^{-1} (FP64)
  // Grouped covariance products of the mixed mode on the tensor cores (one pass over the output tile
  // for several J; never part of a batched launch):
  TASK_VGEMM_G = 15,  // (I, c, J0 | J1 << 16)  V_Ic -= sum_{J0 <= J < J1} L_IJ V_Jc
  TASK_WSYRK_G = 16,  // (a, b, J0 | J1 << 16)  S_ab -= sum_{J0 <= J < J1} V_Ja^T V_Jb
  // Vector solves with the stored inverses, each diagonal block split into 32-row chunks that run in
  // parallel (a second vector, xvec, holds the forward result so no chunk overwrites what another reads):
  TASK_FSOLVE_C = 17,  // (J, ch)  xvec_J[ch] = Linv_J[ch, :] bvec_J
  TASK_BSOLVE_C = 18,  // (J, ch)  bvec_J[ch] = (Linv_J^T)[ch, :] xvec_J
  // Two vertically adjacent tiles of one column updated together (mixed mode on the tensor cores,
  // tile edge 128): both products read the same L_KJ, loaded once per k chunk.
  TASK_UPD2 = 19  // (I, K, J0 | J1 << 16)  K_IK and K_{I+1,K} -= sum_{J0 <= J < J1} L_{I(+1),J} L_KJ^T
};

// One GP of a batch: its inputs, outputs, hyperparameters and workspace (all device pointers).
struct GpDesc {
  const double* X;    // n x D
  const double* y;    // n
  const double* Xs;   // m x D
  double* mean;       // m (output)
  double* cov;        // m x m (output, may be null)
  double* Kt;         // packed lower tiles
  double* V;          // Mt*T x ldv
  double* S;          // Mc*T x lds
  double* bvec;       // Mt*T
  int* cK;            // counters: lower tiles
  int* cV;            // V tiles
  int* cS;            // lower S tiles
  int* cF;            // forward chunks
  int* cB;            // backward chunks
  int* dF;            // forward solve done
  int* dB;            // backward solve done
  long long n, m, ldv, lds;
  double l, v, s2;
  int D, T, Mt, Mc, nch, pad;
  long long* QX;      // fixed-point coordinates of X and Xs under the GP's scale fx (se_kernel.cuh)
  long long* QXs;
  FxScale* fx;
};

// Partial sums of the reverse sweep's diagonal adjoint: RDIAG(P, J) accumulates into partial
// (P - J - 1) mod kAdjParts of column J, so the sum over P runs as kAdjParts parallel chains.
constexpr int kAdjParts = 8;

// Batched task encoding: kind | (gp index << 4) in the first component.
constexpr int kBatchKindBits = 5;  // kinds 0..16 fit below the GP index

struct DagArgs {
  double* Kt;       // packed lower tiles (T x T row-major each), tile (I,J) at I(I+1)/2 + J
  int T, Mt;        // tile edge, tiles per dimension
  double* V;        // Mt*T x ldv row-major (right-hand side K_{X,Xs}, overwritten by V)
  long long ldv;
  int Mc;           // column tiles of V and of S
  double* S;        // Mc*T x lds row-major, lower tiles hold K_{Xs,Xs} - V^T V on exit
  long long lds;
  double* bvec;     // Mt*T vector: y on entry, beta then alpha
  double* Linv;     // Mt x T x T: inverses of the diagonal tiles of L (null: solves by substitution)
  double* xvec;     // Mt*T vector of the chunked solves (forward result; non-null: FSOLVE_C/BSOLVE_C graph,
                    // whose per-block completion counters dF/dB count chunks up to nch)
  uint8_t* Pk;      // mixed mode: packed tensor-core operands of the panel tiles L_IJ (I > J), same tile
                    // index as Kt, T*T*8 bytes each (null: operands staged from FP64 per update)
  uint8_t* PV;      // mixed mode: packed operands of the blocks V_Jc (transposed), (J*Mc + c)*T*T*8 bytes
  uint8_t* PLinv;   // mixed mode, T = 128: packed FP32 inverses of the diagonal tiles, J*T*T*8 bytes (null:
                    // the later panel TRSMs and the V solves run as FP32 substitutions)
  int nch;          // T / 32 (row chunks of the vector tasks)
  int* cK;          // per lower K tile: updates applied (J+1 once final)
  int* cV;          // per V tile
  int* cS;          // per lower S tile
  int* cF;          // per (tile row, chunk): forward updates applied
  int* cB;          // per (tile row, chunk): backward updates applied
  int* dF;          // per tile row: forward solve done
  int* dB;          // per tile row: backward solve done
  double* Bt;       // adjoint tiles (same packing as Kt)
  double* Wt;       // per-diagonal-tile FP64 workspace of the reverse POTRF (Mt x T x T)
  double* Pt;       // partial sums of the diagonal adjoints (Mt x kAdjParts x T x T), zeroed per launch
  int* rc;          // per lower tile: reverse updates applied to Lbar_PJ
  int* fa;          // per lower tile: Abar final
  int* rd;          // per (diagonal tile, part): reverse diagonal updates applied
  const GpDesc* descs;  // batched launch: per-GP views (null otherwise)
  const int4* tasks;
  int ntasks;
  DevStatus* st;
  long long timeout_ns;
  int withhold_task;  // test hook (-1 = off): this task's completion is never published
  int use_umma;       // mixed mode: trailing updates on the tensor cores (tcgen05)
  int prec;           // precision form of the tensor-core products (GP_FP32 = 3xTF32, GP_TF32, GP_BF16,
                      // GP_BF16X3, GP_BF16X6, GP_FP64_OZAKI; gp.h)
  int pkb;            // bytes per value of a packed operand of that form (8, 8, 2, 4, 6, 14)
  int eL, eV;         // GP_FP64_OZAKI: scale exponents of the packed panel tiles of L and of the blocks of V
                      // (|L_ij| <= 2^(eL-1), |V_ij| <= 2^(eV-1): L's rows have norm sqrt(K_ii), V's columns
                      // norm <= sqrt(v))
  int* PLinvExp;      // GP_FP64_OZAKI: scale exponent of each packed diagonal-tile inverse (per tile J)
  long long* trace;   // optional: per task {CTA, t_taken, t_ready, t_done} (%globaltimer ns), 4 x int64
};

// Covariance assembly (Eq. 1). Q / QA, QB / QXs, QX: the points' fixed-point coordinates under the common
// scale fx (launch_fx_prepare over every point set of the call, then launch_fx_quantize per set; null:
// the FP64 distance). With a usable scale the squared distances are exact integer sums (se_kernel.cuh).
cudaError_t launch_exp_neg(const double* x, long long n, double* out, int sms, cudaStream_t st);
// The assembly's fixed-point squared distance sum_d (qa_d - qb_d)^2 2^-twoF, run on the host by the same
// integer routines (se_kernel.cuh).
double fx_sqdist_host(const long long* qa, const long long* qb, int D, int twoF);
cudaError_t launch_fx_prepare(const double* A, long long na, const double* B, long long nb, int D, double l, FxScale* out,
                              int sms, cudaStream_t st);
cudaError_t launch_fx_quantize(const double* X, long long cnt, const FxScale* fx, long long* Q, int sms, cudaStream_t st);
cudaError_t launch_assemble_tiles(const double* X, long long n, int D, double l, double v, double s2, double* Kt, int T,
                                  int Mt, cudaStream_t st, const long long* Q = nullptr, const FxScale* fx = nullptr);
cudaError_t launch_assemble_dense(const double* A, long long na, const double* B, long long nb, int D, double l,
                                  double v, double diag_add, double* out, long long ld, long long rows_pad,
                                  long long cols_pad, cudaStream_t st, const long long* QA = nullptr,
                                  const long long* QB = nullptr, const FxScale* fx = nullptr);
cudaError_t launch_mean_gemv(const double* Xs, long long m, const double* X, long long n, int D, double l, double v,
                             const double* alpha, double* mean, cudaStream_t st, const long long* QXs = nullptr,
                             const long long* QX = nullptr, const FxScale* fx = nullptr);
cudaError_t launch_var_from_v(const double* V, long long ldv, long long nrows, double v, double diag_add, double* var,
                              long long m, cudaStream_t st);
cudaError_t launch_cov_copy(const double* S, long long lds, double* cov, long long m, cudaStream_t st);
cudaError_t launch_factor_rows(const double* Kt, int T, long long n, long long row0, long long nrows, double* out,
                               cudaStream_t st);
cudaError_t launch_logdet(const double* Kt, int T, long long n, double* out, cudaStream_t st);
// Blocked triangular solves with the factor in FP32 (trsv.cu), the correction solves of the refined
// precision forms: b <- L^{-T} L^{-1} b on the packed lower FP32 tiles Lt (edge T = 128 or 256, Mt tile rows)
// with the FP32 diagonal-tile inverses Linv and the chain's matrices M, P (launch_chain_mats); b (FP64) holds the right-hand side on entry and the solution
// on exit, xb (FP64) receives the forward result; front (2 ints) must be zero on entry. One persistent
// CTA per SM (grid, capped at Mt). withhold >= 0: test hook, that forward block is never published (its
// dependants' bounded waits expire with GP_ERR_TIMEOUT). trace (optional, Mt(Mt+1) items): per item
// {CTA, start, ready, done} times and {kind, I, J, 0}, the layout of the persistent kernel's trace; the
// slot counter is st->next_task (zero on entry). trsv32_smem_bytes returns the dynamic shared memory of a
// launch (and its stages), or -1 when the solve does not fit this kernel (T, or too many tile rows per CTA).
int trsv32_smem_bytes(int T, int Mt, int grid, int* stages);
// The solve kernel's item sequence of CTA c out of G (capped at Mt), computed on the host by the same
// iterator the kernel runs: {kind, I, J} triples (kinds 0-7: forward tile, chain step, y product, first
// block; backward the same); returns the count (out may be null), -1 on invalid arguments.
long long trsv32_items(int Mt, int G, int c, int* out, long long cap);
cudaError_t launch_trsv32(const float* Lt, const float* Linv, const float* M, const float* P, double* b, double* xb,
                          int* front, int T, int Mt, int grid, DevStatus* st, long long timeout_ns, int withhold,
                          long long* trace, int4* trace_items, cudaStream_t stream);
// The chain's matrices of the FP32 solve, once per factor (Mt T^2 floats each): M_I = L_II^-1 L_{I,I-1}
// (I >= 1) and P_J = L_{J+1,J} L_JJ^-1 (J <= Mt - 2), from the FP32 tiles and inverses. T = 128 or 256.
cudaError_t launch_chain_mats(const float* Lt, const float* Linv, float* M, float* P, int T, int Mt, cudaStream_t stream);
// dst[i] = (float)src[i] for i < n (the FP32 copy of the factor and of its diagonal-tile inverses).
cudaError_t launch_to_f32(const double* src, float* dst, long long n, int sms, cudaStream_t stream);
cudaError_t launch_dag(const DagArgs& a, int grid, bool mixed, cudaStream_t st, bool reverse = false,
                       bool batch = false);
int dag_max_ctas_per_sm_batch(bool mixed, int use_umma);
// Test hook: C (128 x 128) (-)= A B^T (A, B: 128 x K row-major FP64) through the packed products of
// precision form prec, in one CTA, reps times; work: 2 half_bytes of device memory for the operands.
cudaError_t launch_debug_product(int prec, const double* A, const double* B, double* C, int K, int store, int lower,
                                 uint8_t* work, size_t half_bytes, int reps, DevStatus* st, long long timeout_ns,
                                 cudaStream_t stream);
// Allows the dynamic shared memory of the tensor-core path (once per device).
cudaError_t dag_enable_umma();
// Batched pre/post work, one CTA per work item {kind, gp, a, b}:
//   pre:  0 = K tile a rows [b*32, +32); 1 = K_{X,Xs} rows [a, a+8); 2 = K_{Xs,Xs} rows [a, a+8);
//         3 = rhs vector (y, zero padded)
//   post: 0 = mean rows [a, a+8) (fused K_{Xs,X} alpha); 1 = covariance rows [a, a+8) copied/mirrored
// One CTA per GP: the GP's common fixed-point scale over X and Xs, then both sets quantised.
cudaError_t launch_batch_fx(const GpDesc* descs, int B, cudaStream_t st);
cudaError_t launch_batch_pre(const int4* items, int nitems, const GpDesc* descs, bool noisy_prior, cudaStream_t st);
cudaError_t launch_batch_post(const int4* items, int nitems, const GpDesc* descs, cudaStream_t st);
int dag_max_ctas_per_sm(bool mixed, int use_umma);
// r = y - K alpha from packed lower FP64 tiles; norms = {||r||_2^2, ||y||_2^2, ||r||_inf, ||K||_inf,
// ||alpha||_inf, ||y||_inf} (||K||_inf only with with_knorm, else 0). partial needs 6 * Mt * (T/32) doubles.
cudaError_t launch_residual(const double* Kt, int T, int Mt, long long n, const double* y, const double* alpha,
                            double* r, double* partial, double* norms, cudaStream_t st, bool with_knorm);
cudaError_t launch_axpy(double* alpha, const double* d, long long n, cudaStream_t st);
// NaN/Inf in a[0..cnt) -> GP_ERR_NONFINITE in the status word, info = base + first index + 1.
cudaError_t launch_scan_nonfinite(const double* a, long long cnt, long long base, DevStatus* status,
                                  cudaStream_t st);
// beta = L^T alpha from the factor tiles (so that beta = L^{-1} y when alpha = K^{-1} y).
cudaError_t launch_beta(const double* Lt, int T, int Mt, const double* alpha, double* beta, cudaStream_t st);
// Lbar of the NLML w.r.t. L: -alpha beta^T on the lower triangle plus diag(1/L_ii), i, j < n.
cudaError_t launch_init_lbar(const double* Lt, double* Bt, int T, int Mt, long long n, const double* alpha,
                             const double* beta, cudaStream_t st);
// Partials of sum over stored lower entries of Abar_ij dK_ij/d(l, v, s2), dK recomputed from X; then
// out[0..3) = the three sums. partial needs 3 * Mt(Mt+1)/2 * (T/32) doubles.
cudaError_t launch_grad_contract(const double* Bt, int T, int Mt, const double* X, long long n, int D, double l,
                                 double v, double* partial, double* out, cudaStream_t st,
                                 const long long* Q = nullptr, const FxScale* fx = nullptr);
// GMRES-based refinement: out[i] = <V_i, w> (i < k, rows of V with leading dimension ldv); w += sign * sum_j
// h_j V_j (h on the device); dst = a * src; and the diagonal shift diag(K) += tau of the packed tiles.
cudaError_t launch_multi_dot(const double* V, long long ldv, int k, const double* w, long long n, double* out,
                             cudaStream_t st);
cudaError_t launch_multi_axpy(double* w, const double* V, long long ldv, const double* h, int k, double sign,
                              long long n, cudaStream_t st);
cudaError_t launch_scale_copy(double* dst, const double* src, double a, long long n, cudaStream_t st);
cudaError_t launch_add_diag(double* Kt, int T, long long n, double tau, cudaStream_t st);
// out[0] = sum_{i<n} a_i b_i (one CTA).
cudaError_t launch_dot(const double* a, const double* b, long long n, double* out, cudaStream_t st);

}  // namespace gpk
