// FP32-arithmetic variants of the tile operations, used by the mixed-precision factorization: the
// trailing SYRK/GEMM updates (Sec. 3.2) and the panel TRSMs after the first block column run in FP32
// with FP32 accumulation, on tiles stored in FP64 (each operand is rounded to FP32 when staged in
// shared memory; each result is subtracted from / stored to the FP64 tile).
#pragma once
#include "tiles_f64.cuh"

namespace gpk {

constexpr int SBM = 128, SBN = 128, SBK = 16, SPAD = 4;

struct __align__(16) GemmSmemF32 {  // read with 16-byte vector loads
  float a[2][SBK][SBM + SPAD];
  float b[2][SBK][SBN + SPAD];
};

// 128 x 16 (or 16 x 128) operand chunk: 8 consecutive elements per thread.
template <int L>
__device__ __forceinline__ void g32_load(double (&r)[8], const double* P, int ld, int x0, int k0, int X, int K) {
  const int t = threadIdx.x;
  if (L == 0) {  // P[x*ld + k]: x = t/2, k = 8*(t%2)..+7
    const int x = x0 + t / 2, k = k0 + 8 * (t % 2);
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = (x < X && k + q < K) ? ldcg(P + (size_t)x * ld + k + q) : 0.0;
  } else {  // P[k*ld + x]: k = t/16, x = 8*(t%16)..+7
    const int k = k0 + t / 16, x = x0 + 8 * (t % 16);
#pragma unroll
    for (int q = 0; q < 8; ++q) r[q] = (k < K && x + q < X) ? ldcg(P + (size_t)k * ld + x + q) : 0.0;
  }
}

template <int L>
__device__ __forceinline__ void g32_store(float (*s)[SBM + SPAD], const double (&r)[8]) {
  const int t = threadIdx.x;
  if (L == 0) {
    const int x = t / 2, k = 8 * (t % 2);
#pragma unroll
    for (int q = 0; q < 8; ++q) s[k + q][x] = f64_to_f32_rn(r[q]);
  } else {
    const int k = t / 16, x = 8 * (t % 16);
#pragma unroll
    for (int q = 0; q < 8; ++q) s[k][x + q] = f64_to_f32_rn(r[q]);
  }
}

// C[M x N] (FP64) -= op(A) op(B) computed in FP32 (layouts as in cta_gemm_sub; A_MK/B_NK = 0,
// A_KM/B_KN = 1). 128 x 128 output blocks, 8 x 8 per thread. Ends with __syncthreads().
template <int LA, int LB>
__device__ void cta_gemm_sub_f32(double* C, int ldc, const double* A, int lda, const double* B, int ldb, int M, int N,
                                 int K, bool lower, GemmSmemF32& s) {
  const int t = threadIdx.x, ty = t / 16, tx = t % 16;
  const int nbm = (M + SBM - 1) / SBM, nbn = (N + SBN - 1) / SBN;
  const int nk = (K + SBK - 1) / SBK;
  for (int blk = 0; blk < nbm * nbn; ++blk) {
    const int m0 = (blk / nbn) * SBM, n0 = (blk % nbn) * SBN;
    if (lower && n0 > m0 + SBM - 1) continue;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    double ra[8], rb[8];
    g32_load<LA>(ra, A, lda, m0, 0, M, K);
    g32_load<LB>(rb, B, ldb, n0, 0, N, K);
    g32_store<LA>(s.a[0], ra);
    g32_store<LB>(s.b[0], rb);
    __syncthreads();
    for (int kc = 0; kc < nk; ++kc) {
      const int cur = kc & 1;
      if (kc + 1 < nk) {
        g32_load<LA>(ra, A, lda, m0, (kc + 1) * SBK, M, K);
        g32_load<LB>(rb, B, ldb, n0, (kc + 1) * SBK, N, K);
      }
#pragma unroll
      for (int k = 0; k < SBK; ++k) {
        // rows ty*4 + {0..3} and 64 + ty*4 + {0..3}; columns likewise with tx (conflict-free float4s)
        const float4 a0 = *reinterpret_cast<const float4*>(&s.a[cur][k][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&s.a[cur][k][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&s.b[cur][k][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&s.b[cur][k][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      if (kc + 1 < nk) {
        g32_store<LA>(s.a[cur ^ 1], ra);
        g32_store<LB>(s.b[cur ^ 1], rb);
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int n = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + j - 4);
        if (n >= N || (lower && n > m)) continue;
        double* c = C + (size_t)m * ldc + n;
        *c = ldcg(c) - f32_to_f64(acc[i][j]);
      }
    }
    __syncthreads();
  }
}

struct Tri32F {
  float l[32][33];
  float inv[32];
};

__device__ __forceinline__ void tri32f_load(Tri32F& s, const double* L, int ldl) {
  for (int e = threadIdx.x; e < 32 * 32; e += kThreads) {
    const int i = e / 32, j = e % 32;
    s.l[i][j] = (j <= i) ? f64_to_f32_rn(ldcg(L + (size_t)i * ldl + j)) : 0.f;
  }
  __syncthreads();
  if (threadIdx.x < 32) s.inv[threadIdx.x] = 1.f / s.l[threadIdx.x][threadIdx.x];
  __syncthreads();
}

// B[rows x 32] <- B L^{-T} in FP32 (rows of FP64 storage). Blocks of 256 rows are staged through
// smem (the FP32 GEMM buffers, 256 x 33 floats) with coalesced loads and stores: a warp moves two
// 32-value row segments per instruction, then each thread solves one row from smem.
__device__ void cta_trsm_rows32_f32(const Tri32F& s, double* B, int ldb, int rows, float (*stage)[33]) {
  const int t = threadIdx.x, kp = t & 15, rr = t >> 4;
  for (int r0 = 0; r0 < rows; r0 += kThreads) {
    const int nr = rows - r0 < kThreads ? rows - r0 : kThreads;
    for (int r = rr; r < nr; r += kThreads / 16) {
      const double2 d = __ldcg(reinterpret_cast<const double2*>(B + (size_t)(r0 + r) * ldb) + kp);
      stage[r][2 * kp] = f64_to_f32_rn(d.x);
      stage[r][2 * kp + 1] = f64_to_f32_rn(d.y);
    }
    __syncthreads();
    if (t < nr) {
      float x[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) x[c] = stage[t][c];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        float acc = x[c];
#pragma unroll
        for (int k = 0; k < c; ++k) acc = fmaf(-x[k], s.l[c][k], acc);
        x[c] = acc * s.inv[c];
      }
#pragma unroll
      for (int c = 0; c < 32; ++c) stage[t][c] = x[c];
    }
    __syncthreads();
    for (int r = rr; r < nr; r += kThreads / 16)
      reinterpret_cast<double2*>(B + (size_t)(r0 + r) * ldb)[kp] =
          make_double2(f32_to_f64(stage[r][2 * kp]), f32_to_f64(stage[r][2 * kp + 1]));
    __syncthreads();
  }
}

// B[32 x ncols] <- L^{-1} B in FP32.
__device__ void cta_trsm_cols32_f32(const Tri32F& s, double* B, int ldb, int ncols) {
  for (int c = threadIdx.x; c < ncols; c += kThreads) {
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) x[i] = f64_to_f32_rn(ldcg(B + (size_t)i * ldb + c));
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      float acc = x[i];
#pragma unroll
      for (int k = 0; k < i; ++k) acc = fmaf(-s.l[i][k], x[k], acc);
      x[i] = acc * s.inv[i];
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) B[(size_t)i * ldb + c] = f32_to_f64(x[i]);
  }
  __syncthreads();
}

struct __align__(16) TileSmemF32 {
  GemmSmemF32 g;  // also the 256 x 33 float staging area of the row solves
  Tri32F tri;
};
static_assert(sizeof(GemmSmemF32) >= 256 * 33 * sizeof(float), "row-solve staging must fit the GEMM buffers");

__device__ void cta_trsm_right_f32(const double* L, int ldl, double* B, int ldb, int rows, int nb, TileSmemF32& s) {
  for (int k0 = 0; k0 < nb; k0 += 32) {
    tri32f_load(s.tri, L + (size_t)k0 * ldl + k0, ldl);
    cta_trsm_rows32_f32(s.tri, B + k0, ldb, rows, reinterpret_cast<float(*)[33]>(&s.g));
    const int rest = nb - k0 - 32;
    if (rest > 0)
      cta_gemm_sub_f32<0, 0>(B + k0 + 32, ldb, B + k0, ldb, L + (size_t)(k0 + 32) * ldl + k0, ldl, rows, rest, 32,
                             false, s.g);
  }
}

__device__ void cta_trsm_left_f32(const double* L, int ldl, double* B, int ldb, int nb, int ncols, TileSmemF32& s) {
  for (int k0 = 0; k0 < nb; k0 += 32) {
    tri32f_load(s.tri, L + (size_t)k0 * ldl + k0, ldl);
    cta_trsm_cols32_f32(s.tri, B + (size_t)k0 * ldb, ldb, ncols);
    const int rest = nb - k0 - 32;
    if (rest > 0)
      cta_gemm_sub_f32<0, 1>(B + (size_t)(k0 + 32) * ldb, ldb, L + (size_t)(k0 + 32) * ldl + k0, ldl,
                             B + (size_t)k0 * ldb, ldb, rest, ncols, 32, false, s.g);
  }
}

}  // namespace gpk
