/* FP64 CPU oracle for exact GP prediction (TEST INFRASTRUCTURE, not the product path).
 *
 * Plain, slow, obviously correct C: every quantity is computed from its definition in the paper
 * (Sec. 3.1 "Gaussian Process Regression", Eqs. (1)-(3); Sec. 3.2 "Tiled Algorithms") or from the
 * textbook definition it cites (Rasmussen & Williams 2006, Ch. 2 and Sec. 5.4, for the marginal
 * likelihood and its gradient). No BLAS/LAPACK, no blocking beyond the tiled algorithm the paper
 * itself states. OpenMP only splits independent rows/tiles across threads; every sum is still a
 * plain left-to-right loop.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may call this code. It shares
 * nothing with the CUDA library.
 *
 * Conventions: all matrices are dense, row-major, double precision. Hyperparameters follow the
 * textbook squared-exponential form k(a,b) = v*exp(-|a-b|^2/(2 l^2)) + [same training index]*s2.
 * The paper prints the exponent as -(1/(2 l)) * sum_d (a_d-b_d)^2 (Eq. 1); the two agree when the
 * paper's lengthscale equals l^2, and are identical at the paper's l = 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;

/* ---------------------------------------------------------------- Eq. (1): the SE kernel */

/* Squared distance by direct differences, summed over d = 0..D-1 in order. */
static double sqdist(const double* a, const double* b, int D) {
  double r2 = 0.0;
  for (int d = 0; d < D; ++d) {
    double t = a[d] - b[d];
    r2 += t * t;
  }
  return r2;
}

/* Noise-free part of Eq. (1): v * exp(-r2 / (2 l^2)). */
static double se(double r2, double l, double v) { return v * exp(-r2 / (2.0 * l * l)); }

/* K = K_{X,X} (n x n, both triangles): Eq. (1) with the delta term on the diagonal (Sec. 3.1). */
void oracle_assemble_K(const double* X, i64 n, int D, double l, double v, double s2, double* K) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < n; ++i)
    for (i64 j = 0; j < n; ++j)
      K[i * n + j] = se(sqdist(X + i * D, X + j * D, D), l, v) + (i == j ? s2 : 0.0);
}

/* Cross-covariance K_{A,B} (na x nb): Eq. (1) between two different point sets, so the delta
 * (same-index) term never applies, even where a test point coincides with a training point. */
void oracle_assemble_cross(const double* A, i64 na, const double* B, i64 nb, int D, double l, double v,
                           double* out) {
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < na; ++i)
    for (i64 j = 0; j < nb; ++j) out[i * nb + j] = se(sqdist(A + i * D, B + j * D, D), l, v);
}

/* Prior test covariance K_{Xs,Xs} (m x m). Eq. (3) uses it without saying whether the noise term
 * is present; s2_diag is added on the diagonal (0 gives the latent-function covariance). */
void oracle_assemble_prior(const double* Xs, i64 m, int D, double l, double v, double s2_diag, double* out) {
  oracle_assemble_cross(Xs, m, Xs, m, D, l, v, out);
  for (i64 i = 0; i < m; ++i) out[i * m + i] += s2_diag;
}

/* Selected entries k(A[ia[t]], B[ib[t]]) + (same[t] ? s2 : 0), for sampled checks at large n. */
void oracle_kernel_entries(const double* A, const double* B, int D, double l, double v, double s2, i64 cnt,
                           const i64* ia, const i64* ib, const int32_t* same, double* out) {
#pragma omp parallel for schedule(static)
  for (i64 t = 0; t < cnt; ++t)
    out[t] = se(sqdist(A + ia[t] * D, B + ib[t] * D, D), l, v) + (same[t] ? s2 : 0.0);
}

/* Rows `rows[t]` of K_{X,X} times a vector: out[t] = sum_j k(x_rows[t], x_j) w_j, the kernel entries
 * recomputed from X (used to form residuals y - K alpha without storing K). */
void oracle_kernel_rows_matvec(const double* X, i64 n, int D, double l, double v, double s2, i64 cnt,
                               const i64* rows, const double* w, double* out) {
#pragma omp parallel for schedule(static)
  for (i64 t = 0; t < cnt; ++t) {
    i64 i = rows[t];
    double acc = 0.0;
    for (i64 j = 0; j < n; ++j) acc += (se(sqdist(X + i * D, X + j * D, D), l, v) + (i == j ? s2 : 0.0)) * w[j];
    out[t] = acc;
  }
}

/* ---------------------------------------------------------------- Cholesky, K = L L^T (Sec. 3.1) */

/* Unblocked right-looking Cholesky in place on the lower triangle of the n x n row-major A: for
 * each column j, L_jj = sqrt(A_jj), L_ij = A_ij / L_jj below it, then the rank-1 update
 * A_ik -= L_ij L_kj of the trailing lower triangle. The strict upper triangle is set to zero.
 * Returns 0, or the 1-based column whose pivot is not positive (LAPACK convention). */
int oracle_cholesky(double* A, i64 n) {
  for (i64 j = 0; j < n; ++j) {
    double d = A[j * n + j];
    if (!(d > 0.0)) return (int)(j + 1);
    double ljj = sqrt(d);
    A[j * n + j] = ljj;
    for (i64 i = j + 1; i < n; ++i) A[i * n + j] /= ljj;
#pragma omp parallel for schedule(static) if (n - j > 256)
    for (i64 k = j + 1; k < n; ++k) {
      double lkj = A[k * n + j];
      for (i64 i = k; i < n; ++i) A[i * n + k] -= A[i * n + j] * lkj;
    }
  }
  for (i64 i = 0; i < n; ++i)
    for (i64 j = i + 1; j < n; ++j) A[i * n + j] = 0.0;
  return 0;
}

/* Tile (I,J) of the n x n row-major matrix, tile edge T; the last tile row/column may be short. */
typedef struct {
  double* p;
  i64 ld, rows, cols;
} tile_t;

static tile_t tile_at(double* A, i64 n, i64 T, i64 I, i64 J) {
  tile_t t;
  t.p = A + I * T * n + J * T;
  t.ld = n;
  t.rows = (I * T + T <= n) ? T : n - I * T;
  t.cols = (J * T + T <= n) ? T : n - J * T;
  return t;
}

/* POTRF: L_JJ <- Chol(K_JJ), unblocked right-looking on one diagonal tile. Returns 0 or the
 * 1-based column within the tile. */
static int tile_potrf(tile_t a) {
  for (i64 j = 0; j < a.rows; ++j) {
    double d = a.p[j * a.ld + j];
    if (!(d > 0.0)) return (int)(j + 1);
    double ljj = sqrt(d);
    a.p[j * a.ld + j] = ljj;
    for (i64 i = j + 1; i < a.rows; ++i) a.p[i * a.ld + j] /= ljj;
    for (i64 k = j + 1; k < a.rows; ++k)
      for (i64 i = k; i < a.rows; ++i) a.p[i * a.ld + k] -= a.p[i * a.ld + j] * a.p[k * a.ld + j];
  }
  return 0;
}

/* TRSM: L_IJ <- K_IJ L_JJ^{-T}, i.e. solve X L_JJ^T = K_IJ row by row (forward substitution on
 * each row of the panel tile). */
static void tile_trsm(tile_t l, tile_t b) {
  for (i64 r = 0; r < b.rows; ++r) {
    double* x = b.p + r * b.ld;
    for (i64 c = 0; c < b.cols; ++c) {
      double s = x[c];
      for (i64 k = 0; k < c; ++k) s -= x[k] * l.p[c * l.ld + k];
      x[c] = s / l.p[c * l.ld + c];
    }
  }
}

/* GEMM / SYRK: C <- C - A B^T (SYRK is the case A == B on a diagonal tile, lower half only). */
static void tile_update(tile_t c, tile_t a, tile_t b, int lower_only) {
  for (i64 i = 0; i < c.rows; ++i)
    for (i64 k = 0; k < (lower_only ? i + 1 : c.cols); ++k) {
      double s = 0.0;
      for (i64 t = 0; t < a.cols; ++t) s += a.p[i * a.ld + t] * b.p[k * b.ld + t];
      c.p[i * c.ld + k] -= s;
    }
}

/* The paper's tiled right-looking Cholesky (Sec. 3.2, Fig. 1): for J = 0..M-1, POTRF on the
 * diagonal tile, TRSM on every tile below it, then SYRK on the diagonal tiles and GEMM on the
 * off-diagonal tiles of the trailing lower triangle. Same arithmetic order per entry as the figure;
 * the independent TRSM and update tasks of one step run on OpenMP threads. Tiles of size T, the last
 * one ragged when T does not divide n. Returns 0 or the 1-based failing column. */
int oracle_cholesky_tiled(double* A, i64 n, i64 T) {
  if (T <= 0) T = n;
  i64 M = (n + T - 1) / T;
  for (i64 J = 0; J < M; ++J) {
    int info = tile_potrf(tile_at(A, n, T, J, J));
    if (info) return (int)(J * T + info);
#pragma omp parallel for schedule(dynamic)
    for (i64 I = J + 1; I < M; ++I) tile_trsm(tile_at(A, n, T, J, J), tile_at(A, n, T, I, J));
#pragma omp parallel for schedule(dynamic)
    for (i64 p = 0; p < (M - J - 1) * (M - J - 1); ++p) {
      i64 I = J + 1 + p / (M - J - 1), Kc = J + 1 + p % (M - J - 1);
      if (Kc > I) continue;
      tile_update(tile_at(A, n, T, I, Kc), tile_at(A, n, T, I, J), tile_at(A, n, T, Kc, J), Kc == I);
    }
  }
  for (i64 i = 0; i < n; ++i)
    for (i64 j = i + 1; j < n; ++j) A[i * n + j] = 0.0;
  return 0;
}

/* ---------------------------------------------------------------- Eq. (2): predictive mean */

/* Forward substitution L x = b for nrhs right-hand sides stored as columns of the n x nrhs b. */
void oracle_forward(const double* L, i64 n, const double* b, i64 nrhs, double* x) {
#pragma omp parallel for schedule(static)
  for (i64 c = 0; c < nrhs; ++c)
    for (i64 i = 0; i < n; ++i) {
      double s = b[i * nrhs + c];
      for (i64 k = 0; k < i; ++k) s -= L[i * n + k] * x[k * nrhs + c];
      x[i * nrhs + c] = s / L[i * n + i];
    }
}

/* Backward substitution L^T x = b (one right-hand side). */
void oracle_backward(const double* L, i64 n, const double* b, double* x) {
  for (i64 i = n - 1; i >= 0; --i) {
    double s = b[i];
    for (i64 k = i + 1; k < n; ++k) s -= L[k * n + i] * x[k];
    x[i] = s / L[i * n + i];
  }
}

/* Eq. (2) by the paper's recipe: L beta = y, L^T alpha = beta, mean = K_{Xs,X} alpha. */
void oracle_predict_mean(const double* L, i64 n, const double* y, const double* Kxs, i64 m, double* alpha,
                         double* mean) {
  double* beta = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  oracle_forward(L, n, y, 1, beta);
  oracle_backward(L, n, beta, alpha);
  free(beta);
#pragma omp parallel for schedule(static)
  for (i64 i = 0; i < m; ++i) {
    double s = 0.0;
    for (i64 j = 0; j < n; ++j) s += Kxs[i * n + j] * alpha[j];
    mean[i] = s;
  }
}

/* ---------------------------------------------------------------- Eq. (3): predictive covariance */

/* Eq. (3) by the paper's recipe: solve L V = K_{X,Xs} (V is n x m), W = V^T V, cov = K_{Xs,Xs} - W.
 * Kxs is K_{Xs,X} (m x n); its transpose is the right-hand side. Every entry of cov is computed on
 * its own (both triangles), so symmetry of the result is a real check. V (n x m) is returned. */
void oracle_predict_cov(const double* L, i64 n, const double* Kxs, const double* Kss, i64 m, double* V,
                        double* cov) {
  double* rhs = (double*)malloc(sizeof(double) * (size_t)(n * m > 0 ? n * m : 1));
  for (i64 i = 0; i < n; ++i)
    for (i64 c = 0; c < m; ++c) rhs[i * m + c] = Kxs[c * n + i];
  oracle_forward(L, n, rhs, m, V);
  free(rhs);
#pragma omp parallel for schedule(static)
  for (i64 a = 0; a < m; ++a)
    for (i64 b = 0; b < m; ++b) {
      double w = 0.0;
      for (i64 k = 0; k < n; ++k) w += V[k * m + a] * V[k * m + b];
      cov[a * m + b] = Kss[a * m + b] - w;
    }
}

/* ---------------------------------------------------------------- marginal likelihood (R&W 2006) */

/* log det K = 2 sum_i log L_ii. */
double oracle_logdet(const double* L, i64 n) {
  double s = 0.0;
  for (i64 i = 0; i < n; ++i) s += log(L[i * n + i]);
  return 2.0 * s;
}

/* Negative log marginal likelihood: 1/2 y^T alpha + 1/2 log det K + n/2 log(2 pi) (R&W Eq. 2.30). */
double oracle_nlml(const double* L, i64 n, const double* y, const double* alpha) {
  double q = 0.0;
  for (i64 i = 0; i < n; ++i) q += y[i] * alpha[i];
  return 0.5 * q + 0.5 * oracle_logdet(L, n) + 0.5 * (double)n * log(2.0 * 3.14159265358979323846);
}

/* K^{-1} = L^{-T} L^{-1}: the triangular inverse Li = L^{-1} by forward substitution on the
 * identity, then Kinv_ij = sum_k Li_ki Li_kj. */
void oracle_kinv(const double* L, i64 n, double* Kinv) {
  double* Li = (double*)calloc((size_t)(n * n > 0 ? n * n : 1), sizeof(double));
#pragma omp parallel for schedule(dynamic)
  for (i64 c = 0; c < n; ++c)
    for (i64 i = c; i < n; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (i64 k = c; k < i; ++k) s -= L[i * n + k] * Li[k * n + c];
      Li[i * n + c] = s / L[i * n + i];
    }
#pragma omp parallel for schedule(dynamic)
  for (i64 i = 0; i < n; ++i)
    for (i64 j = 0; j < n; ++j) {
      double s = 0.0;
      for (i64 k = (i > j ? i : j); k < n; ++k) s += Li[k * n + i] * Li[k * n + j];
      Kinv[i * n + j] = s;
    }
  free(Li);
}

/* Gradient of the NLML w.r.t. (l, v, s2) (R&W Eq. 5.9 with the sign of the negative):
 * d nlml / d theta = 1/2 sum_ij (K^{-1} - alpha alpha^T)_ij dK_ij/dtheta, with
 * dK/dl = v exp(-r2/(2l^2)) r2 / l^3, dK/dv = exp(-r2/(2l^2)), dK/ds2 = I. */
void oracle_nlml_grad(const double* X, i64 n, int D, double l, double v, const double* Kinv, const double* alpha,
                      double grad[3]) {
  double gl = 0.0, gv = 0.0, gs = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : gl, gv, gs)
  for (i64 i = 0; i < n; ++i) {
    double al = 0.0, av = 0.0;
    for (i64 j = 0; j < n; ++j) {
      double r2 = sqdist(X + i * D, X + j * D, D);
      double e = exp(-r2 / (2.0 * l * l));
      double kbar = Kinv[i * n + j] - alpha[i] * alpha[j];
      al += kbar * v * e * r2 / (l * l * l);
      av += kbar * e;
    }
    gl += al;
    gv += av;
    gs += Kinv[i * n + i] - alpha[i] * alpha[i];
  }
  grad[0] = 0.5 * gl;
  grad[1] = 0.5 * gv;
  grad[2] = 0.5 * gs;
}
