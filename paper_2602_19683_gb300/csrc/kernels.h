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
  TASK_BGEMV = 9    // (J, I, ch) b_J[ch] -= L_IJ[:,ch]^T b_I
};

struct DagArgs {
  double* Kt;       // packed lower tiles (T x T row-major each), tile (I,J) at I(I+1)/2 + J
  int T, Mt;        // tile edge, tiles per dimension
  double* V;        // Mt*T x ldv row-major (right-hand side K_{X,Xs}, overwritten by V)
  long long ldv;
  int Mc;           // column tiles of V and of S
  double* S;        // Mc*T x lds row-major, lower tiles hold K_{Xs,Xs} - V^T V on exit
  long long lds;
  double* bvec;     // Mt*T vector: y on entry, beta then alpha
  int nch;          // T / 32 (row chunks of the vector tasks)
  int* cK;          // per lower K tile: updates applied (J+1 once final)
  int* cV;          // per V tile
  int* cS;          // per lower S tile
  int* cF;          // per (tile row, chunk): forward updates applied
  int* cB;          // per (tile row, chunk): backward updates applied
  int* dF;          // per tile row: forward solve done
  int* dB;          // per tile row: backward solve done
  const int4* tasks;
  int ntasks;
  DevStatus* st;
  long long timeout_ns;
  int withhold_task;  // test hook (-1 = off): this task's completion is never published
};

cudaError_t launch_assemble_tiles(const double* X, long long n, int D, double l, double v, double s2, double* Kt, int T,
                                  int Mt, cudaStream_t st);
cudaError_t launch_assemble_dense(const double* A, long long na, const double* B, long long nb, int D, double l,
                                  double v, double diag_add, double* out, long long ld, long long rows_pad,
                                  long long cols_pad, cudaStream_t st);
cudaError_t launch_mean_gemv(const double* Xs, long long m, const double* X, long long n, int D, double l, double v,
                             const double* alpha, double* mean, cudaStream_t st);
cudaError_t launch_cov_copy(const double* S, long long lds, double* cov, long long m, cudaStream_t st);
cudaError_t launch_factor_rows(const double* Kt, int T, long long n, long long row0, long long nrows, double* out,
                               cudaStream_t st);
cudaError_t launch_logdet(const double* Kt, int T, long long n, double* out, cudaStream_t st);
cudaError_t launch_dag(const DagArgs& a, int grid, bool mixed, cudaStream_t st);
int dag_max_ctas_per_sm(bool mixed);
// r = y - K alpha from packed lower FP64 tiles; norms[0] = ||r||^2, norms[1] = ||y||^2.
// partial needs 2 * Mt * (T/32) doubles.
cudaError_t launch_residual(const double* Kt, int T, int Mt, long long n, const double* y, const double* alpha,
                            double* r, double* partial, double* norms, cudaStream_t st);
cudaError_t launch_axpy(double* alpha, const double* d, long long n, cudaStream_t st);

}  // namespace gpk
