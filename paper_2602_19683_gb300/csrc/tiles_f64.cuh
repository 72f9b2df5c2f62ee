// CTA-level FP64 tile operations of the tiled Cholesky (Sec. 3.2: POTRF, TRSM, SYRK, GEMM) and of
// the triangular solves of Eqs. (2)-(3). Every function is executed by all kThreads threads of one
// CTA and reads operands that other CTAs may have written through L2-only loads.
//
// On GB300 the FP64 pipe issues about two FMAs per clock per SM (measured: 1.19 TFLOP/s FP64 FFMA,
// 1.05 TFLOP/s for the FP64 mma.sync path), so these routines are FP64-issue bound at any sane
// memory layout: the design goal is no wasted FMAs and enough independent FMA chains per warp, and
// the FMA path is plain FFMA rather than DMMA.
#pragma once
#include "common.cuh"

namespace gpk {

// Operand layouts of C -= op(A) op(B), with op(A) M x K and op(B) K x N.
enum { A_MK = 0, A_KM = 1 };  // A_MK: A[m*lda + k]; A_KM: A[k*lda + m]
enum { B_NK = 0, B_KN = 1 };  // B_NK: B[n*ldb + k] (C -= A B^T); B_KN: B[k*ldb + n]

constexpr int GBM = 64, GBN = 64, GBK = 16, GPAD = 4;

struct __align__(16) GemmSmem {  // read with 16-byte vector loads
  double a[2][GBK][GBM + GPAD];
  double b[2][GBK][GBN + GPAD];
};

template <int LA>
__device__ __forceinline__ void gemm_load_a(double (&r)[4], const double* A, int lda, int m0, int k0, int M, int K) {
  const int t = threadIdx.x;
  if (LA == A_MK) {  // 64 rows x 16 k: thread -> (m = t/4, k = 4*(t%4) .. +3)
    const int m = m0 + t / 4, k = k0 + 4 * (t % 4);
#pragma unroll
    for (int q = 0; q < 4; ++q) r[q] = (m < M && k + q < K) ? ldcg(A + (size_t)m * lda + k + q) : 0.0;
  } else {  // 16 k x 64 m: thread -> (k = t/16, m = 4*(t%16) .. +3)
    const int k = k0 + t / 16, m = m0 + 4 * (t % 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) r[q] = (k < K && m + q < M) ? ldcg(A + (size_t)k * lda + m + q) : 0.0;
  }
}

template <int LA>
__device__ __forceinline__ void gemm_store_a(GemmSmem& s, int buf, const double (&r)[4]) {
  const int t = threadIdx.x;
  if (LA == A_MK) {
    const int m = t / 4, k = 4 * (t % 4);
#pragma unroll
    for (int q = 0; q < 4; ++q) s.a[buf][k + q][m] = r[q];
  } else {
    const int k = t / 16, m = 4 * (t % 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) s.a[buf][k][m + q] = r[q];
  }
}

template <int LB>
__device__ __forceinline__ void gemm_load_b(double (&r)[4], const double* B, int ldb, int n0, int k0, int N, int K) {
  const int t = threadIdx.x;
  if (LB == B_NK) {
    const int n = n0 + t / 4, k = k0 + 4 * (t % 4);
#pragma unroll
    for (int q = 0; q < 4; ++q) r[q] = (n < N && k + q < K) ? ldcg(B + (size_t)n * ldb + k + q) : 0.0;
  } else {
    const int k = k0 + t / 16, n = n0 + 4 * (t % 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) r[q] = (k < K && n + q < N) ? ldcg(B + (size_t)k * ldb + n + q) : 0.0;
  }
}

template <int LB>
__device__ __forceinline__ void gemm_store_b(GemmSmem& s, int buf, const double (&r)[4]) {
  const int t = threadIdx.x;
  if (LB == B_NK) {
    const int n = t / 4, k = 4 * (t % 4);
#pragma unroll
    for (int q = 0; q < 4; ++q) s.b[buf][k + q][n] = r[q];
  } else {
    const int k = t / 16, n = 4 * (t % 16);
#pragma unroll
    for (int q = 0; q < 4; ++q) s.b[buf][k][n + q] = r[q];
  }
}

// C[M x N] -= op(A) op(B). lower: only entries with (row + diag_off) >= col are written (and output
// blocks entirely above that line are skipped). Ends with __syncthreads().
template <int LA, int LB>
__device__ void cta_gemm_sub(double* C, int ldc, const double* A, int lda, const double* B, int ldb, int M, int N,
                             int K, bool lower, int diag_off, GemmSmem& s) {
  const int t = threadIdx.x, ty = t / 16, tx = t % 16;
  const int nbm = (M + GBM - 1) / GBM, nbn = (N + GBN - 1) / GBN;
  const int nk = (K + GBK - 1) / GBK;
  for (int blk = 0; blk < nbm * nbn; ++blk) {
    const int m0 = (blk / nbn) * GBM, n0 = (blk % nbn) * GBN;
    if (lower && n0 > m0 + GBM - 1 + diag_off) continue;  // block strictly above the diagonal
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    double ra[4], rb[4];
    gemm_load_a<LA>(ra, A, lda, m0, 0, M, K);
    gemm_load_b<LB>(rb, B, ldb, n0, 0, N, K);
    gemm_store_a<LA>(s, 0, ra);
    gemm_store_b<LB>(s, 0, rb);
    __syncthreads();
    for (int kc = 0; kc < nk; ++kc) {
      const int cur = kc & 1;
      if (kc + 1 < nk) {
        gemm_load_a<LA>(ra, A, lda, m0, (kc + 1) * GBK, M, K);
        gemm_load_b<LB>(rb, B, ldb, n0, (kc + 1) * GBK, N, K);
      }
#pragma unroll
      for (int k = 0; k < GBK; ++k) {
        const double2 a01 = *reinterpret_cast<const double2*>(&s.a[cur][k][ty * 4]);
        const double2 a23 = *reinterpret_cast<const double2*>(&s.a[cur][k][ty * 4 + 2]);
        const double2 b01 = *reinterpret_cast<const double2*>(&s.b[cur][k][tx * 4]);
        const double2 b23 = *reinterpret_cast<const double2*>(&s.b[cur][k][tx * 4 + 2]);
        const double av[4] = {a01.x, a01.y, a23.x, a23.y};
        const double bv[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
      }
      if (kc + 1 < nk) {
        gemm_store_a<LA>(s, cur ^ 1, ra);
        gemm_store_b<LB>(s, cur ^ 1, rb);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + ty * 4 + i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int n = n0 + tx * 4 + j;
        if (n >= N || (lower && n > m + diag_off)) continue;
        double* c = C + (size_t)m * ldc + n;
        *c = ldcg(c) - acc[i][j];
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- 32-wide triangular kernels

// Smem copy of a 32 x 32 lower-triangular diagonal block with its reciprocal diagonal.
struct Tri32 {
  double l[32][33];
  double inv[32];
};

// Loads the lower triangle of L[0..32) x [0..32) (already factored) into smem.
__device__ __forceinline__ void tri32_load(Tri32& s, const double* L, int ldl) {
  for (int e = threadIdx.x; e < 32 * 32; e += kThreads) {
    const int i = e / 32, j = e % 32;
    s.l[i][j] = (j <= i) ? ldcg(L + (size_t)i * ldl + j) : 0.0;
  }
  __syncthreads();
  if (threadIdx.x < 32) s.inv[threadIdx.x] = 1.0 / s.l[threadIdx.x][threadIdx.x];
  __syncthreads();
}

// Square root of a positive pivot d and its reciprocal, for the serial chain of a diagonal block
// (one thread computes them while the CTA waits): an FP32 reciprocal-square-root seed refined by two
// Newton-Raphson steps in FP64, r <- r (3 - d r^2) / 2, each of which doubles the correct bits (about
// 2^-22 -> 2^-44 -> below FP64 rounding); then sqrt(d) = d r. About ten FP64 operations instead of an
// FP64 square root and a division, whose longer dependent sequences cost microseconds per pivot on
// this GPU's FP64 pipe. Pivots outside the FP32 range take the library square root and division.
__device__ __forceinline__ void pivot_sqrt_rcp(double d, double& s, double& r) {
  if (d > 1e-30 && d < 1e30) {
    double y = (double)rsqrtf((float)d);
    const double h = 0.5 * d;
    y = y * fma(-h * y, y, 1.5);
    y = y * fma(-h * y, y, 1.5);
    r = y;
    s = d * y;
  } else {
    s = sqrt(d);
    r = 1.0 / s;
  }
}

// CTA-parallel right-looking Cholesky of a 32 x 32 block B (smem, leading dimension ld): step j, thread
// 0 takes the pivot, 31 threads scale column j, and all 8 warps share the rank-1 update of the trailing
// triangle (thread t: row j+1+t/8, columns j+1+(t%8), +8, ...), so every SM sub-partition's FP64 unit
// works (a single warp would reach only a quarter of the SM's FP64 rate). inv receives 1/L_jj.
// Returns 0 or the 1-based failing column (same in every thread).
__device__ int cta_potrf32_par(double* B, int ld, double* inv, int* flag) {
  const int t = threadIdx.x;
  for (int j = 0; j < 32; ++j) {
    if (t == 0) {
      const double d = B[j * ld + j];
      if (!(d > 0.0)) {
        *flag = j + 1;
      } else {
        double ljj, rj;
        pivot_sqrt_rcp(d, ljj, rj);
        B[j * ld + j] = ljj;
        inv[j] = rj;
      }
    }
    __syncthreads();
    if (*flag) return *flag;
    if (t > j && t < 32) B[t * ld + j] *= inv[j];
    __syncthreads();
    const int i = j + 1 + (t >> 3);
    if (i < 32) {
      const double lij = B[i * ld + j];
      for (int k = j + 1 + (t & 7); k <= i; k += 8) B[i * ld + k] = fma(-lij, B[k * ld + j], B[i * ld + k]);
    }
    __syncthreads();
  }
  return 0;
}

// Warp-level right-looking Cholesky of a 32 x 32 block whose row `lane` is held in registers r[0..32)
// (lower part significant). col[32] is a smem column buffer; inv receives the reciprocal diagonal.
// Statically indexed inner loops keep everything in registers. Returns 0 or the 1-based failing
// column (same in every lane).
__device__ __forceinline__ int warp_potrf32_regs(double (&r)[32], double* col, double* inv) {
  const int i = threadIdx.x & 31;
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const double d = __shfl_sync(0xffffffffu, r[j], j);
    if (!(d > 0.0)) return j + 1;  // uniform: every lane saw the same pivot (also catches NaN)
    const double ljj = sqrt(d), ij = 1.0 / ljj;
    if (i == j) {
      r[j] = ljj;
      inv[j] = ij;
    }
    if (i > j) r[j] *= ij;
    col[i] = r[j];  // column j of L (rows > j significant)
    __syncwarp();
#pragma unroll
    for (int k = j + 1; k < 32; ++k)
      if (k <= i) r[k] = fma(-r[j], col[k], r[k]);
    __syncwarp();
  }
  return 0;
}

// Unblocked Cholesky of the 32 x 32 diagonal block at A (in place, lower; upper zeroed), by warp 0
// with lane i owning row i: right-looking column by column. Leaves the factor in s. Returns 0 or
// the 1-based failing column (same value in every thread).
// kRegs: rows in registers (warp_potrf32_regs; for kernels with registers to spare); otherwise the
// rows stay in smem and lane i updates row i element by element (fits the 128-register FP64 kernel).
template <bool kRegs>
__device__ int cta_potrf32(double* A, int lda, Tri32& s, int* shared_flag) {
  const int t = threadIdx.x;
  __shared__ double col[32];
  if (t == 0) *shared_flag = 0;
  if constexpr (kRegs) {
    (void)col;
    for (int e = t; e < 32 * 32; e += kThreads) {
      const int i = e / 32, j = e % 32;
      s.l[i][j] = (j <= i) ? ldcg(A + (size_t)i * lda + j) : 0.0;
    }
    __syncthreads();
    cta_potrf32_par(&s.l[0][0], 33, s.inv, shared_flag);
  } else {
    for (int e = t; e < 32 * 32; e += kThreads) {
      const int i = e / 32, j = e % 32;
      s.l[i][j] = (j <= i) ? ldcg(A + (size_t)i * lda + j) : 0.0;
    }
    __syncthreads();
    if (t < 32) {
      const int i = t;
      int fail = 0;
      for (int j = 0; j < 32; ++j) {
        const double d = s.l[j][j];
        if (!(d > 0.0)) {
          fail = j + 1;
          break;
        }
        const double ljj = sqrt(d);
        const double inv = 1.0 / ljj;
        __syncwarp();
        if (i == j) {
          s.l[j][j] = ljj;
          s.inv[j] = inv;
        }
        if (i > j) s.l[i][j] *= inv;
        __syncwarp();
        if (i > j) {
          const double lij = s.l[i][j];
          for (int k = j + 1; k <= i; ++k) s.l[i][k] = fma(-lij, s.l[k][j], s.l[i][k]);
        }
        __syncwarp();
      }
      if (i == 0) *shared_flag = fail;
    }
  }
  __syncthreads();
  const int fail = *shared_flag;
  if (fail == 0) {
    for (int e = t; e < 32 * 32; e += kThreads) {
      const int i = e / 32, j = e % 32;
      A[(size_t)i * lda + j] = (j <= i) ? s.l[i][j] : 0.0;
    }
  }
  __syncthreads();
  return fail;
}

// B[rows x 32] <- B L^{-T} with L the 32 x 32 lower block in s: each thread solves whole rows
// (x_c = (b_c - sum_{k<c} x_k L_ck) / L_cc).
__device__ void cta_trsm_rows32(const Tri32& s, double* B, int ldb, int rows) {
  for (int r = threadIdx.x; r < rows; r += kThreads) {
    double x[32];
    double* row = B + (size_t)r * ldb;
#pragma unroll
    for (int c = 0; c < 32; ++c) x[c] = ldcg(row + c);
#pragma unroll
    for (int c = 0; c < 32; ++c) {  // four independent chains: the FP64 FMA latency is long
      double a0 = x[c], a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
      for (int k = 0; k < c; ++k) {
        const double v = -x[k];
        if ((k & 3) == 0) a0 = fma(v, s.l[c][k], a0);
        if ((k & 3) == 1) a1 = fma(v, s.l[c][k], a1);
        if ((k & 3) == 2) a2 = fma(v, s.l[c][k], a2);
        if ((k & 3) == 3) a3 = fma(v, s.l[c][k], a3);
      }
      x[c] = ((a0 + a1) + (a2 + a3)) * s.inv[c];
    }
#pragma unroll
    for (int c = 0; c < 32; ++c) row[c] = x[c];
  }
  __syncthreads();
}

// B[32 x ncols] <- L^{-1} B with L the 32 x 32 lower block in s: each thread solves whole columns.
__device__ void cta_trsm_cols32(const Tri32& s, double* B, int ldb, int ncols) {
  for (int c = threadIdx.x; c < ncols; c += kThreads) {
    double x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = ldcg(B + (size_t)i * ldb + c);
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      double acc = x[i];
#pragma unroll
      for (int k = 0; k < i; ++k) acc = fma(-s.l[i][k], x[k], acc);
      x[i] = acc * s.inv[i];
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) B[(size_t)i * ldb + c] = x[i];
  }
  __syncthreads();
}

struct __align__(16) TileSmem {
  GemmSmem g;
  Tri32 tri;
  int flag;
};

// POTRF of the nb x nb diagonal tile A (nb a multiple of 32), blocked right-looking with 32-wide
// strips: factor the strip's diagonal block, TRSM the rows below it, SYRK-update the trailing
// lower triangle. Upper triangle zeroed. Returns 0 or the 1-based failing column within the tile.
template <bool kRegs>
__device__ int cta_potrf(double* A, int lda, int nb, TileSmem& s) {
  for (int k0 = 0; k0 < nb; k0 += 32) {
    const int fail = cta_potrf32<kRegs>(A + (size_t)k0 * lda + k0, lda, s.tri, &s.flag);
    if (fail) return k0 + fail;
    const int rest = nb - k0 - 32;
    if (rest > 0) {
      cta_trsm_rows32(s.tri, A + (size_t)(k0 + 32) * lda + k0, lda, rest);
      double* P = A + (size_t)(k0 + 32) * lda + k0;  // rest x 32 panel
      cta_gemm_sub<A_MK, B_NK>(A + (size_t)(k0 + 32) * lda + k0 + 32, lda, P, lda, P, lda, rest, rest, 32, true, 0,
                               s.g);
    }
    // zero the strip's part above the diagonal block (columns k0+32.. of rows k0..k0+32)
    for (int e = threadIdx.x; e < 32 * rest; e += kThreads) {
      const int i = e / rest, j = e % rest;
      A[(size_t)(k0 + i) * lda + k0 + 32 + j] = 0.0;
    }
    __syncthreads();
  }
  return 0;
}

// POTRF of an nb x nb diagonal tile (nb <= 128, a multiple of 32) held entirely in shared memory
// (sm: nb x (nb + 1) doubles, inv: 32 doubles): coalesced load, 32-wide right-looking strips (warp 0
// factors the strip's diagonal block, one thread per row solves the rows below it, all threads update
// the trailing lower triangle), coalesced store with the upper triangle zeroed. Same arithmetic as
// cta_potrf, without the global-memory round trips that make the critical path latency-bound.
// Returns 0 or the 1-based failing column.
__device__ int cta_potrf_smem(double* A, int lda, int nb, double* sm, double* inv, int* flag) {
  const int ld = nb + 1, t = threadIdx.x;
  // coalesced double2 loads, eight in flight per thread (the tile is L2-resident: latency, not
  // bandwidth, decides how long this takes)
  const int npair = nb / 2;
  for (int e0 = 0; e0 < nb * npair; e0 += 8 * kThreads) {
    double2 d[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * kThreads + t;
      if (e < nb * npair) d[q] = __ldcg(reinterpret_cast<const double2*>(A + (size_t)(e / npair) * lda) + e % npair);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = e0 + q * kThreads + t;
      if (e < nb * npair) {
        const int i = e / npair, j = 2 * (e % npair);
        sm[i * ld + j] = (j <= i) ? d[q].x : 0.0;
        sm[i * ld + j + 1] = (j + 1 <= i) ? d[q].y : 0.0;
      }
    }
  }
  if (t == 0) *flag = 0;
  __syncthreads();
  for (int k0 = 0; k0 < nb; k0 += 32) {
    {
      const int fail = cta_potrf32_par(sm + (size_t)k0 * ld + k0, ld, inv, flag);
      if (fail) return k0 + fail;
    }
    for (int r = k0 + 32 + t; r < nb; r += kThreads) {  // rows below: x L_kk^T = row
      double* row = sm + (size_t)r * ld + k0;
      double x[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) x[c] = row[c];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        const double* lc = sm + (size_t)(k0 + c) * ld + k0;
        double a0 = x[c], a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
        for (int k = 0; k < c; ++k) {
          if ((k & 3) == 0) a0 = fma(-x[k], lc[k], a0);
          if ((k & 3) == 1) a1 = fma(-x[k], lc[k], a1);
          if ((k & 3) == 2) a2 = fma(-x[k], lc[k], a2);
          if ((k & 3) == 3) a3 = fma(-x[k], lc[k], a3);
        }
        x[c] = ((a0 + a1) + (a2 + a3)) * inv[c];
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) row[c] = x[c];
    }
    __syncthreads();
    const int m = nb - k0 - 32;  // trailing lower triangle, entries (i, j), j <= i, enumerated directly
    for (int e = t; e < m * (m + 1) / 2; e += kThreads) {
      int i = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while (i * (i + 1) / 2 > e) --i;
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      const int j = e - i * (i + 1) / 2;
      const double* ri = sm + (size_t)(k0 + 32 + i) * ld + k0;
      const double* rj = sm + (size_t)(k0 + 32 + j) * ld + k0;
      double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
      for (int c = 0; c < 32; c += 4) {
        a0 = fma(ri[c], rj[c], a0);
        a1 = fma(ri[c + 1], rj[c + 1], a1);
        a2 = fma(ri[c + 2], rj[c + 2], a2);
        a3 = fma(ri[c + 3], rj[c + 3], a3);
      }
      sm[(size_t)(k0 + 32 + i) * ld + k0 + 32 + j] -= (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
  }
  for (int e = t; e < nb * nb; e += kThreads) {
    const int i = e / nb, j = e % nb;
    A[(size_t)i * lda + j] = (j <= i) ? sm[(size_t)i * ld + j] : 0.0;
  }
  __syncthreads();
  return 0;
}

// TRSM from the right: B[rows x nb] <- B L^{-T}, L the nb x nb lower factor (Sec. 3.2 TRSM,
// L_IJ = K_IJ L_JJ^{-T}). Right-looking over 32-wide column strips.
__device__ void cta_trsm_right(const double* L, int ldl, double* B, int ldb, int rows, int nb, TileSmem& s) {
  for (int k0 = 0; k0 < nb; k0 += 32) {
    tri32_load(s.tri, L + (size_t)k0 * ldl + k0, ldl);
    cta_trsm_rows32(s.tri, B + k0, ldb, rows);
    const int rest = nb - k0 - 32;
    if (rest > 0)
      cta_gemm_sub<A_MK, B_NK>(B + k0 + 32, ldb, B + k0, ldb, L + (size_t)(k0 + 32) * ldl + k0, ldl, rows, rest, 32,
                               false, 0, s.g);
  }
}

// TRSM from the left: B[nb x ncols] <- L^{-1} B (Eq. 3's L V = K_{X,Xs}, one tile row at a time).
__device__ void cta_trsm_left(const double* L, int ldl, double* B, int ldb, int nb, int ncols, TileSmem& s) {
  for (int k0 = 0; k0 < nb; k0 += 32) {
    tri32_load(s.tri, L + (size_t)k0 * ldl + k0, ldl);
    cta_trsm_cols32(s.tri, B + (size_t)k0 * ldb, ldb, ncols);
    const int rest = nb - k0 - 32;
    if (rest > 0)
      cta_gemm_sub<A_MK, B_KN>(B + (size_t)(k0 + 32) * ldb, ldb, L + (size_t)(k0 + 32) * ldl + k0, ldl,
                               B + (size_t)k0 * ldb, ldb, rest, ncols, 32, false, 0, s.g);
  }
}

// TRSM from the right with L not transposed: B[rows x nb] <- B L^{-1} (G L = B, columns solved from
// the last: g_c = (b_c - sum_{k>c} g_k L_kc) / L_cc). Used by the Cholesky adjoint.
__device__ void cta_trsm_right_N(const double* L, int ldl, double* B, int ldb, int rows, int nb, TileSmem& s) {
  for (int k0 = nb - 32; k0 >= 0; k0 -= 32) {
    tri32_load(s.tri, L + (size_t)k0 * ldl + k0, ldl);
    for (int r = threadIdx.x; r < rows; r += kThreads) {
      double x[32];
      double* row = B + (size_t)r * ldb + k0;
#pragma unroll
      for (int c = 0; c < 32; ++c) x[c] = ldcg(row + c);
#pragma unroll
      for (int c = 31; c >= 0; --c) {
        double acc = x[c];
#pragma unroll
        for (int k = c + 1; k < 32; ++k) acc = fma(-x[k], s.tri.l[k][c], acc);
        x[c] = acc * s.tri.inv[c];
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) row[c] = x[c];
    }
    __syncthreads();
    if (k0 > 0)  // B[:, 0:k0] -= G[:, k0:k0+32] L[k0:k0+32, 0:k0]
      cta_gemm_sub<A_MK, B_KN>(B, ldb, B + k0, ldb, L + (size_t)k0 * ldl, ldl, rows, k0, 32, false, 0, s.g);
  }
}

// TRSM from the left with L transposed: B[nb x ncols] <- L^{-T} B (rows solved from the bottom:
// x_i = (b_i - sum_{k>i} L_ki x_k) / L_ii). Used by the Cholesky adjoint.
__device__ void cta_trsm_left_T(const double* L, int ldl, double* B, int ldb, int nb, int ncols, TileSmem& s) {
  for (int k0 = nb - 32; k0 >= 0; k0 -= 32) {
    tri32_load(s.tri, L + (size_t)k0 * ldl + k0, ldl);
    for (int c = threadIdx.x; c < ncols; c += kThreads) {
      double x[32];
#pragma unroll
      for (int i = 0; i < 32; ++i) x[i] = ldcg(B + (size_t)(k0 + i) * ldb + c);
#pragma unroll
      for (int i = 31; i >= 0; --i) {
        double acc = x[i];
#pragma unroll
        for (int k = i + 1; k < 32; ++k) acc = fma(-s.tri.l[k][i], x[k], acc);
        x[i] = acc * s.tri.inv[i];
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) B[(size_t)(k0 + i) * ldb + c] = x[i];
    }
    __syncthreads();
    if (k0 > 0)  // B[0:k0, :] -= L[k0:k0+32, 0:k0]^T X
      cta_gemm_sub<A_KM, B_KN>(B, ldb, L + (size_t)k0 * ldl, ldl, B + (size_t)k0 * ldb, ldb, k0, ncols, 32, false, 0,
                               s.g);
  }
}

// ---------------------------------------------------------------- vector solves (Eq. 2)

// b[0..nb) <- L^{-1} b (forward substitution with one diagonal tile). Each 32-row strip: its 32 x 32
// diagonal block is staged in smem, warp 0 solves it (lane i owns row i), then all threads update the
// rows below with the strip's columns.
__device__ void cta_trsv_lower(const double* L, int ldl, double* b, int nb, double* xs /*smem[32]*/, Tri32& tri) {
  const int t = threadIdx.x;
  for (int k0 = 0; k0 < nb; k0 += 32) {
    tri32_load(tri, L + (size_t)k0 * ldl + k0, ldl);
    if (t < 32) {
      double bi = ldcg(b + k0 + t);
      for (int j = 0; j < 32; ++j) {
        const double xj = __shfl_sync(0xffffffffu, bi * tri.inv[j], j);
        if (t == j) bi = xj;
        if (t > j) bi = fma(-tri.l[t][j], xj, bi);
      }
      xs[t] = bi;
      b[k0 + t] = bi;
    }
    __syncthreads();
    for (int r = k0 + 32 + t; r < nb; r += kThreads) {
      const double* Lr = L + (size_t)r * ldl + k0;
      double acc = ldcg(b + r);
#pragma unroll 8
      for (int j = 0; j < 32; ++j) acc = fma(-ldcg(Lr + j), xs[j], acc);
      b[r] = acc;
    }
    __syncthreads();
  }
}

// b[0..nb) <- L^{-T} b (backward substitution with one diagonal tile), strips from the bottom.
__device__ void cta_trsv_lower_T(const double* L, int ldl, double* b, int nb, double* xs, Tri32& tri) {
  const int t = threadIdx.x;
  for (int k0 = nb - 32; k0 >= 0; k0 -= 32) {
    tri32_load(tri, L + (size_t)k0 * ldl + k0, ldl);
    if (t < 32) {
      double bi = ldcg(b + k0 + t);
      for (int j = 31; j >= 0; --j) {
        const double xj = __shfl_sync(0xffffffffu, bi * tri.inv[j], j);
        if (t == j) bi = xj;
        if (t < j) bi = fma(-tri.l[j][t], xj, bi);
      }
      xs[t] = bi;
      b[k0 + t] = bi;
    }
    __syncthreads();
    for (int r = t; r < k0; r += kThreads) {  // rows above: b_r -= sum_j L[k0+j][r] x_j
      double acc = ldcg(b + r);
#pragma unroll 8
      for (int j = 0; j < 32; ++j) acc = fma(-ldcg(L + (size_t)(k0 + j) * ldl + r), xs[j], acc);
      b[r] = acc;
    }
    __syncthreads();
  }
}

// b[0..nb) <- Linv b, Linv the lower-triangular inverse of a diagonal tile (upper triangle zero): the
// diagonal-block solve as a matrix-vector product, without the substitution's serial chain. b is
// staged in smem (xs, nb doubles). Each warp takes eight rows at a time; lanes stride the columns
// (coalesced row segments), so up to 8 x (nb / 32) loads per lane are in flight together.
__device__ void cta_trsv_inv(const double* Linv, int ld, double* b, int nb, double* xs) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  for (int i = t; i < nb; i += kThreads) xs[i] = ldcg(b + i);
  __syncthreads();
  for (int r0 = 8 * w; r0 < nb; r0 += 8 * (kThreads / 32)) {
    const double* L0 = Linv + (size_t)r0 * ld;
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
#pragma unroll 4
    for (int c = lane; c <= r0 + 7; c += 32) {
      const double x = xs[c];
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = fma(ldcg(L0 + (size_t)q * ld + c), x, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (lane < 8) {
      double v = acc[0];
#pragma unroll
      for (int q = 1; q < 8; ++q) v = (lane == q) ? acc[q] : v;
      b[r0 + lane] = v;
    }
  }
  __syncthreads();
}

// b[0..nb) <- Linv^T b (the diagonal-block solve of L^T x = b). Per 32-column strip: warps split the
// rows at or below the strip, lanes own its columns; partial sums are reduced through red[8][32].
__device__ void cta_trsv_inv_T(const double* Linv, int ld, double* b, int nb, double* xs, double (*red)[32]) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  for (int i = t; i < nb; i += kThreads) xs[i] = ldcg(b + i);
  __syncthreads();
  for (int c0 = 0; c0 < nb; c0 += 32) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int r = c0 + w;
    constexpr int W = kThreads / 32;
    for (; r + 3 * W < nb; r += 4 * W) {
      a0 = fma(ldcg(Linv + (size_t)r * ld + c0 + lane), xs[r], a0);
      a1 = fma(ldcg(Linv + (size_t)(r + W) * ld + c0 + lane), xs[r + W], a1);
      a2 = fma(ldcg(Linv + (size_t)(r + 2 * W) * ld + c0 + lane), xs[r + 2 * W], a2);
      a3 = fma(ldcg(Linv + (size_t)(r + 3 * W) * ld + c0 + lane), xs[r + 3 * W], a3);
    }
    for (; r < nb; r += W) a0 = fma(ldcg(Linv + (size_t)r * ld + c0 + lane), xs[r], a0);
    red[w][lane] = (a0 + a1) + (a2 + a3);
    __syncthreads();
    if (t < 32) {
      double acc = 0.0;
#pragma unroll
      for (int q = 0; q < W; ++q) acc += red[q][t];
      b[c0 + t] = acc;
    }
    __syncthreads();
  }
}

// Linv <- L^{-1} for a factored nb x nb diagonal tile: the identity solved in place from the left.
// Entries above the diagonal stay exactly zero.
__device__ void cta_trtri(const double* L, int ldl, double* Linv, int nb, TileSmem& s);

// b[r] -= sum_c A[r][c] x[c] for r in [0, rows) (kSet: b[r] = sum ...): each warp takes four rows at a
// time, lanes over columns, so the loads of the four rows are in flight together.
template <bool kSet = false>
__device__ void cta_gemv_sub(const double* A, int lda, const double* x, double* b, int rows, int cols) {
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  for (int r0 = 4 * w; r0 < rows; r0 += 4 * (kThreads / 32)) {
    const int nr = rows - r0 < 4 ? rows - r0 : 4;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 4
    for (int c = lane; c < cols; c += 32) {
      const double xv = ldcg(x + c);
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (q < nr) acc[q] = fma(ldcg(A + (size_t)(r0 + q) * lda + c), xv, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    }
    if (lane < nr) {
      const double v = lane == 0 ? acc[0] : lane == 1 ? acc[1] : lane == 2 ? acc[2] : acc[3];
      b[r0 + lane] = kSet ? v : ldcg(b + r0 + lane) - v;
    }
  }
  __syncthreads();
}

// b[c] -= sum_r A[r][c] x[r] for c in [0, cols) with cols <= 32 (kSet: b[c] = sum ...): warps split the
// rows, lanes own columns, partial sums reduced through smem (red[8][32]).
template <bool kSet = false>
__device__ void cta_gemv_T_sub(const double* A, int lda, const double* x, double* b, int rows, int cols,
                               double (*red)[32]) {
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  double a0 = 0.0, a1 = 0.0;
  if (lane < cols) {
    constexpr int W = kThreads / 32;
    int r = w;
#pragma unroll 2
    for (; r + W < rows; r += 2 * W) {
      a0 = fma(ldcg(A + (size_t)r * lda + lane), ldcg(x + r), a0);
      a1 = fma(ldcg(A + (size_t)(r + W) * lda + lane), ldcg(x + r + W), a1);
    }
    if (r < rows) a0 = fma(ldcg(A + (size_t)r * lda + lane), ldcg(x + r), a0);
  }
  red[w][lane] = a0 + a1;
  __syncthreads();
  if (threadIdx.x < cols) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < kThreads / 32; ++q) s += red[q][threadIdx.x];
    b[threadIdx.x] = kSet ? s : ldcg(b + threadIdx.x) - s;
  }
  __syncthreads();
}

__device__ void cta_trtri(const double* L, int ldl, double* Linv, int nb, TileSmem& s) {
  const size_t nn = (size_t)nb * nb;
  for (size_t e = threadIdx.x; e < nn; e += kThreads) Linv[e] = (e / nb == e % nb) ? 1.0 : 0.0;
  __syncthreads();
  cta_trsm_left(L, ldl, Linv, nb, nb, nb, s);
}

}  // namespace gpk
