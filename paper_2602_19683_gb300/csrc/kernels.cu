// Device kernels of the GP hot path: covariance assembly (Eq. 1), the persistent task-DAG kernel that
// runs the tiled Cholesky (Sec. 3.2, Fig. 1) and the tiled solves of Eqs. (2)-(3), and the fused
// cross-covariance GEMV of the predictive mean.
#include <climits>

#include "bslice.cuh"
#include "kernels.h"
#include "se_kernel.cuh"

namespace gpk {

// ---------------------------------------------------------------- tensor-core forms

// Packs an R x Kd FP64 block (Op[r][k] = src[r ld + k], or src[k ld + r] when trans) in the operand
// format of precision form `prec` (scale exponent e for the fixed-point digits of GP_FP64_OZAKI).
__device__ __noinline__ void form_pack(int prec, const double* src, int ld, bool trans, int R, int Kd, uint8_t* dst,
                                       int e) {
  switch (prec) {
    case GP_BF16: cta_pack_bs<1, false, kBsKcFloat>(src, ld, trans, R, Kd, dst, 0); break;
    case GP_BF16X3: cta_pack_bs<2, false, kBsKcFloat>(src, ld, trans, R, Kd, dst, 0); break;
    case GP_BF16X6: cta_pack_bs<3, false, kBsKcFloat>(src, ld, trans, R, Kd, dst, 0); break;
    case GP_FP64_OZAKI: cta_pack_bs<kOzSlices, true, kBsKcFixed>(src, ld, trans, R, Kd, dst, e); break;
    default: cta_pack_operand(src, ld, trans, R, Kd, dst); break;  // GP_FP32 (3xTF32), GP_TF32
  }
}

// Packs an FP32 nb x nb matrix in shared memory (leading dimension ldx) in the form's operand format.
__device__ __noinline__ void form_pack_f32(int prec, const float* Xs, int ldx, int nb, uint8_t* dst) {
  switch (prec) {
    case GP_BF16: cta_pack_bs_f32<1>(Xs, ldx, nb, dst); break;
    case GP_BF16X3: cta_pack_bs_f32<2>(Xs, ldx, nb, dst); break;
    case GP_BF16X6: cta_pack_bs_f32<3>(Xs, ldx, nb, dst); break;
    default: cta_pack_tf32_f32(Xs, ldx, nb, dst); break;
  }
}

// C (T x T tile, ldc) -= (kStore: =) sum_j A_j B_j^T from packed operands of precision form `prec`.
// The BF16-slice forms take T = 128; eA, eB: scale exponents of the fixed-point form.
// Fixed-point operands with a per-tile scale (single-tile products: kStore) take the fixed-point unit
// kOzLsbTile; the norm-bounded panel and V operands of the updates kOzLsbBounded.
template <bool kStore>
__device__ __noinline__ bool form_product(UmmaState& u, BsPipe& bp, int prec, double* C, int ldc, const PkPairs& pr,
                                          int T, bool lower, int eA, int eB, DevStatus* st, long long to,
                                          long long where) {
  constexpr int lsb = kStore ? kOzLsbTile : kOzLsbBounded;
  switch (prec) {
    case GP_BF16: return bs_block_sub<1, false, kStore>(u, bp, C, ldc, pr, T, 0, 0, lower, 0, 0, 0, st, to, where);
    case GP_BF16X3: return bs_block_sub<2, false, kStore>(u, bp, C, ldc, pr, T, 0, 0, lower, 0, 0, 0, st, to, where);
    case GP_BF16X6: return bs_block_sub<3, false, kStore>(u, bp, C, ldc, pr, T, 0, 0, lower, 0, 0, 0, st, to, where);
    case GP_FP64_OZAKI:
      return bs_block_sub<kOzSlices, true, kStore>(u, bp, C, ldc, pr, T, 0, 0, lower, eA, eB, lsb, st, to, where);
    case GP_TF32: return umma_pk_gemm_sub<kStore, 1>(u, C, ldc, pr, T, T, T, lower, st, to, where);
    default: return umma_pk_gemm_sub<kStore, 3>(u, C, ldc, pr, T, T, T, lower, st, to, where);
  }
}

// ---------------------------------------------------------------- Eq. (1)

template <int D>
__device__ __forceinline__ double sqdist_t(const double* __restrict__ a, const double* __restrict__ b, int Dr) {
  double r2 = 0.0;
  if (D > 0) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const double t = __ldg(a + d) - __ldg(b + d);
      r2 = fma(t, t, r2);
    }
  } else {
    for (int d = 0; d < Dr; ++d) {
      const double t = __ldg(a + d) - __ldg(b + d);
      r2 = fma(t, t, r2);
    }
  }
  return r2;
}

// r^2 = |a - b|^2 from fixed-point coordinates (exact, rounded once); D > 0.
template <int D>
__device__ __forceinline__ double fx_sqdist(const long long* qa, const long long (&qb)[D], int twoF) {
  U128 acc{0ull, 0ull};
#pragma unroll
  for (int d = 0; d < D; ++d) fx_add_sq(acc, __ldg(qa + d), qb[d]);
  return fx_to_double(acc, twoF);
}

// The same with the dimension known at run time (both coordinate rows read from memory).
__device__ __forceinline__ double fx_sqdist_rt(const long long* qa, const long long* qb, int D, int twoF) {
  U128 acc{0ull, 0ull};
  for (int d = 0; d < D; ++d) fx_add_sq(acc, __ldg(qa + d), __ldg(qb + d));
  return fx_to_double(acc, twoF);
}

// The scale rule shared by the single-GP and batched preparations: F = 57 - floor(log2 S) for the largest
// |coordinate| S; usable when every coordinate is finite, S <= 64 l, D <= 256 and F is in range.
__device__ __forceinline__ FxScale fx_decide(double S, int nonfinite, int D, double l) {
  FxScale r{0, 0};
  if (!nonfinite && D <= 256) {
    if (S == 0.0) {
      r.usable = 1;
    } else {
      r.F = 57 - ilogb(S);
      r.usable = (S <= 64.0 * l && r.F <= 511 && r.F >= -448) ? 1 : 0;
    }
  }
  return r;
}

// Quantisation of one launch family: S = max |coordinate| over A (na x D) and B (nb x D), reduced by
// many CTAs into out->smax / out->nonfinite (zeroed beforehand), then fx_decide_kernel sets F and
// usable (fx_decide).
__global__ void __launch_bounds__(kThreads) fx_reduce_kernel(const double* __restrict__ A, long long na,
                                                             const double* __restrict__ B, long long nb, int D,
                                                             FxScale* out) {
  double mx = 0.0;
  int nonfinite = 0;
  const long long total = (na + nb) * D;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const double x = e < na * D ? A[e] : B[e - na * D];
    if (!(fabs(x) <= 1.7976931348623157e308)) nonfinite = 1;
    else mx = fmax(mx, fabs(x));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nonfinite |= __shfl_xor_sync(0xffffffffu, nonfinite, o);
  }
  if (threadIdx.x % 32 == 0) {
    if (mx > 0.0) atomicMax(&out->smax, (unsigned long long)__double_as_longlong(mx));
    if (nonfinite) atomicOr(&out->nonfinite, 1);
  }
}

__global__ void fx_decide_kernel(int D, double l, FxScale* out) {
  const FxScale r = fx_decide(__longlong_as_double((long long)out->smax), out->nonfinite, D, l);
  out->F = r.F;
  out->usable = r.usable;
}

// Q[e] = round(X[e] 2^F) (nothing when the scale is not usable).
__global__ void fx_quantize_kernel(const double* __restrict__ X, long long cnt, const FxScale* __restrict__ fx,
                                   long long* __restrict__ Q) {
  const FxScale f = *fx;
  if (!f.usable) return;
  const double scale = ldexp(1.0, f.F);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x)
    Q[e] = __double2ll_rn(X[e] * scale);
}

// Lower tiles of K: tile blockIdx.x (packed index), rows [blockIdx.y*32, +32) of it. Entries outside
// the n x n matrix form the identity padding. With usable fixed-point coordinates Q (D > 0) the
// distances are the exact integer ones; a thread keeps its column's coordinates in registers while its
// column stays the same.
template <int D>
__global__ void __launch_bounds__(kThreads) assemble_tiles_kernel(const double* __restrict__ X, long long n, int Dr,
                                                                  double neg_half_inv_l2, double v, double s2,
                                                                  double* __restrict__ Kt, int T,
                                                                  const long long* __restrict__ Q,
                                                                  const FxScale* __restrict__ fx) {
  const long long t = blockIdx.x;
  long long I = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > t) --I;
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  const long long J = t - I * (I + 1) / 2;
  double* tile = Kt + (size_t)t * T * T;
  const int r0 = blockIdx.y * 32;
  const bool use_fx = D > 0 && Q != nullptr && fx->usable;
  const int twoF = use_fx ? 2 * fx->F : 0;
  long long qj[D > 0 ? D : 1];
  long long jcached = -1;
  for (int e = threadIdx.x; e < 32 * T; e += kThreads) {
    const int r = r0 + e / T, c = e % T;
    const long long i = I * T + r, j = J * T + c;
    double val;
    if (i < n && j < n) {
      double r2;
      if (D > 0 && use_fx) {
        if (j != jcached) {
#pragma unroll
          for (int d = 0; d < (D > 0 ? D : 1); ++d) qj[d] = __ldg(Q + j * D + d);
          jcached = j;
        }
        r2 = fx_sqdist<(D > 0 ? D : 1)>(Q + i * D, qj, twoF);
      } else {
        r2 = sqdist_t<D>(X + i * Dr, X + j * Dr, Dr);
      }
      val = v * exp_neg(r2 * neg_half_inv_l2) + (i == j ? s2 : 0.0);
    } else {
      val = (i == j) ? 1.0 : 0.0;
    }
    tile[(size_t)r * T + c] = val;
  }
}

// Dense block out[i*ld + j], i < rows_pad, j < cols_pad: k(A_i, B_j) for i < na, j < nb (no noise:
// different point sets), plus diag_add on i == j when same_set, and 0 in the padding. QA, QB: the
// fixed-point coordinates of A and B under one common scale fx (or null).
template <int D>
__global__ void __launch_bounds__(kThreads) assemble_dense_kernel(const double* __restrict__ A, long long na,
                                                                  const double* __restrict__ B, long long nb, int Dr,
                                                                  double neg_half_inv_l2, double v, double diag_add,
                                                                  double* __restrict__ out, long long ld,
                                                                  long long rows_pad, long long cols_pad,
                                                                  const long long* __restrict__ QA,
                                                                  const long long* __restrict__ QB,
                                                                  const FxScale* __restrict__ fx) {
  const long long i = (long long)blockIdx.y * 8 + threadIdx.x / 32;
  if (i >= rows_pad) return;
  const bool use_fx = D > 0 && QA != nullptr && fx->usable && i < na;
  const int twoF = use_fx ? 2 * fx->F : 0;
  long long qi[D > 0 ? D : 1];
  if (use_fx) {
#pragma unroll
    for (int d = 0; d < (D > 0 ? D : 1); ++d) qi[d] = __ldg(QA + i * D + d);
  }
  for (long long j = (long long)blockIdx.x * 128 + (threadIdx.x % 32); j < cols_pad && j < (long long)(blockIdx.x + 1) * 128;
       j += 32) {
    double val = 0.0;
    if (i < na && j < nb) {
      const double r2 = (D > 0 && use_fx) ? fx_sqdist<(D > 0 ? D : 1)>(QB + j * D, qi, twoF)
                                          : sqdist_t<D>(A + i * Dr, B + j * Dr, Dr);
      val = v * exp_neg(r2 * neg_half_inv_l2) + (i == j ? diag_add : 0.0);
    }
    out[(size_t)i * ld + j] = val;
  }
}

// mean[i] = sum_{j<n} k(Xs_i, X_j) alpha_j, the kernel row recomputed on the fly (Eq. 2's last
// step fused with the assembly of K_{Xs,X}). 8 test points per CTA. QXs, QX: fixed-point coordinates
// under one common scale fx (or null).
template <int D>
__global__ void __launch_bounds__(kThreads) mean_gemv_kernel(const double* __restrict__ Xs, long long m,
                                                             const double* __restrict__ X, long long n, int Dr,
                                                             double neg_half_inv_l2, double v,
                                                             const double* __restrict__ alpha, double* __restrict__ mean,
                                                             const long long* __restrict__ QXs,
                                                             const long long* __restrict__ QX,
                                                             const FxScale* __restrict__ fx) {
  __shared__ double red[8][kThreads / 32];
  __shared__ long long qs[8][D > 0 ? D : 1];
  const long long i0 = (long long)blockIdx.x * 8;
  const bool use_fx = D > 0 && QX != nullptr && fx->usable;
  const int twoF = use_fx ? 2 * fx->F : 0;
  if (use_fx) {
    for (int e = threadIdx.x; e < 8 * (D > 0 ? D : 1); e += kThreads) {
      const int q = e / (D > 0 ? D : 1), d = e % (D > 0 ? D : 1);
      qs[q][d] = i0 + q < m ? QXs[(i0 + q) * (D > 0 ? D : 1) + d] : 0;
    }
    __syncthreads();
  }
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  for (long long j = threadIdx.x; j < n; j += kThreads) {
    const double aj = __ldg(alpha + j);
    if (D > 0 && use_fx) {
      long long qj[D > 0 ? D : 1];
#pragma unroll
      for (int d = 0; d < (D > 0 ? D : 1); ++d) qj[d] = __ldg(QX + j * (D > 0 ? D : 1) + d);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (i0 + q < m) {
          U128 sacc{0ull, 0ull};
#pragma unroll
          for (int d = 0; d < (D > 0 ? D : 1); ++d) fx_add_sq(sacc, qs[q][d], qj[d]);
          acc[q] = fma(v * exp_neg(fx_to_double(sacc, twoF) * neg_half_inv_l2), aj, acc[q]);
        }
      }
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (i0 + q < m) {
          const double r2 = sqdist_t<D>(Xs + (i0 + q) * Dr, X + j * Dr, Dr);
          acc[q] = fma(v * exp_neg(r2 * neg_half_inv_l2), aj, acc[q]);
        }
      }
    }
  }
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double s = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) red[q][w] = s;
  }
  __syncthreads();
  if (threadIdx.x < 8 && i0 + threadIdx.x < m) {
    double s = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[threadIdx.x][q];
    mean[i0 + threadIdx.x] = s;
  }
}

// cov[a*m + b] from the lower triangle of the padded work matrix S (both triangles written).
__global__ void cov_copy_kernel(const double* __restrict__ S, long long lds, double* __restrict__ cov, long long m) {
  for (long long a = blockIdx.y; a < m; a += gridDim.y)
    for (long long b = (long long)blockIdx.x * kThreads + threadIdx.x; b < m; b += (long long)gridDim.x * kThreads)
      cov[a * m + b] = (a >= b) ? S[a * lds + b] : S[b * lds + a];
}

// ---------------------------------------------------------------- persistent task-DAG kernel

__device__ __forceinline__ size_t tri(long long I, long long J) { return (size_t)(I * (I + 1) / 2 + J); }

// Waits (thread 0) for every dependency of task tk. Returns false on abort/time-out.
__device__ bool wait_deps(const DagArgs& a, int4 tk, int ti) {
  const int type = tk.x, p = tk.y, q = tk.z, r = tk.w;
  DevStatus* st = a.st;
  const long long to = a.timeout_ns;
  switch (type) {
    case TASK_POTRF:
      return wait_ge(a.cK + tri(p, p), p, st, to, ti);
    case TASK_TRSM:  // (I=p, J=q)
      return wait_ge(a.cK + tri(q, q), q + 1, st, to, ti) && wait_ge(a.cK + tri(p, q), q, st, to, ti);
    case TASK_UPD: {  // (I=p, K=q, J in [J0, J1)) with r = J0 | J1 << 16 (J1 = 0: the single column J0)
      const int J0 = r & 0xFFFF, J1 = (r >> 16) ? (r >> 16) : J0 + 1;
      for (int J = J0; J < J1; ++J)
        if (!wait_ge(a.cK + tri(p, J), J + 1, st, to, ti) || !wait_ge(a.cK + tri(q, J), J + 1, st, to, ti)) return false;
      return wait_ge(a.cK + tri(p, q), J0, st, to, ti);
    }
    case TASK_UPD2: {  // rows p and p + 1 of column q, J in [J0, J1)
      const int J0 = r & 0xFFFF, J1 = r >> 16;
      for (int J = J0; J < J1; ++J)
        if (!wait_ge(a.cK + tri(p, J), J + 1, st, to, ti) || !wait_ge(a.cK + tri(p + 1, J), J + 1, st, to, ti) ||
            !wait_ge(a.cK + tri(q, J), J + 1, st, to, ti))
          return false;
      return wait_ge(a.cK + tri(p, q), J0, st, to, ti) && wait_ge(a.cK + tri(p + 1, q), J0, st, to, ti);
    }
    // The solve tasks also wait for the factor tiles they read to be final (immediately true when the
    // factorisation ran in an earlier launch; needed when one launch runs a GP's whole pipeline).
    case TASK_VTRSM:  // (J=p, c=q)
      return wait_ge(a.cK + tri(p, p), p + 1, st, to, ti) && wait_ge(a.cV + (size_t)p * a.Mc + q, p, st, to, ti);
    case TASK_VGEMM:  // (I=p, J=q, c=r)
      return wait_ge(a.cK + tri(p, q), q + 1, st, to, ti) && wait_ge(a.cV + (size_t)q * a.Mc + r, q + 1, st, to, ti) &&
             wait_ge(a.cV + (size_t)p * a.Mc + r, q, st, to, ti);
    case TASK_VGEMM_G: {  // (I=p, c=q, J0 | J1 << 16)
      const int J0 = r & 0xFFFF, J1 = r >> 16;
      for (int J = J0; J < J1; ++J)
        if (!wait_ge(a.cK + tri(p, J), J + 1, st, to, ti) || !wait_ge(a.cV + (size_t)J * a.Mc + q, J + 1, st, to, ti))
          return false;
      return wait_ge(a.cV + (size_t)p * a.Mc + q, J0, st, to, ti);
    }
    case TASK_WSYRK_G: {  // (a=p, b=q, J0 | J1 << 16)
      const int J0 = r & 0xFFFF, J1 = r >> 16;
      for (int J = J0; J < J1; ++J)
        if (!wait_ge(a.cV + (size_t)J * a.Mc + p, J + 1, st, to, ti) || !wait_ge(a.cV + (size_t)J * a.Mc + q, J + 1, st, to, ti))
          return false;
      return wait_ge(a.cS + tri(p, q), J0, st, to, ti);
    }
    case TASK_WSYRK:  // (a=p, b=q, J=r)
      return wait_ge(a.cV + (size_t)r * a.Mc + p, r + 1, st, to, ti) &&
             wait_ge(a.cV + (size_t)r * a.Mc + q, r + 1, st, to, ti) && wait_ge(a.cS + tri(p, q), r, st, to, ti);
    case TASK_FSOLVE: {  // (J=p)
      if (!wait_ge(a.cK + tri(p, p), p + 1, st, to, ti)) return false;
      for (int ch = 0; ch < a.nch; ++ch)
        if (!wait_ge(a.cF + (size_t)p * a.nch + ch, p, st, to, ti)) return false;
      return true;
    }
    case TASK_FGEMV:  // (I=p, J=q, ch=r)
      return wait_ge(a.cK + tri(p, q), q + 1, st, to, ti) && wait_ge(a.dF + q, a.xvec ? a.nch : 1, st, to, ti) &&
             wait_ge(a.cF + (size_t)p * a.nch + r, q, st, to, ti);
    case TASK_FSOLVE_C: {  // (J=p, ch=q): every chunk of block J has all its updates
      if (!wait_ge(a.cK + tri(p, p), p + 1, st, to, ti)) return false;
      for (int ch = 0; ch < a.nch; ++ch)
        if (!wait_ge(a.cF + (size_t)p * a.nch + ch, p, st, to, ti)) return false;
      return true;
    }
    case TASK_BSOLVE_C: {  // (J=p, ch=q): forward block J done, every chunk of xvec_J has its updates
      if (!wait_ge(a.dF + p, a.nch, st, to, ti)) return false;
      for (int ch = 0; ch < a.nch; ++ch)
        if (!wait_ge(a.cB + (size_t)p * a.nch + ch, a.Mt - 1 - p, st, to, ti)) return false;
      return true;
    }
    case TASK_BSOLVE: {  // (J=p)
      if (!wait_ge(a.dF + p, 1, st, to, ti)) return false;
      for (int ch = 0; ch < a.nch; ++ch)
        if (!wait_ge(a.cB + (size_t)p * a.nch + ch, a.Mt - 1 - p, st, to, ti)) return false;
      return true;
    }
    case TASK_BGEMV:  // (J=p, I=q, ch=r)
      return wait_ge(a.cK + tri(q, p), p + 1, st, to, ti) && wait_ge(a.dB + q, a.xvec ? a.nch : 1, st, to, ti) &&
             wait_ge(a.dF + p, a.xvec ? a.nch : 1, st, to, ti) &&
             wait_ge(a.cB + (size_t)p * a.nch + r, a.Mt - 1 - q, st, to, ti);
    case TASK_RUPD: {  // (P=p, K=q, J=r); terms applied with K descending
      const int hi = p > q ? p : q, lo = p > q ? q : p;
      return wait_ge(a.fa + tri(hi, lo), 1, st, to, ti) && wait_ge(a.rc + tri(p, r), a.Mt - 1 - q, st, to, ti);
    }
    case TASK_RTRSM:  // (P=p, J=q)
      return wait_ge(a.rc + tri(p, q), a.Mt - 1 - q, st, to, ti);
    case TASK_RDIAG: {  // (P=p, J=q): k-th contribution of part (p - q - 1) % kAdjParts
      const int part = (p - q - 1) % kAdjParts, k = (p - q - 1) / kAdjParts;
      return wait_ge(a.fa + tri(p, q), 1, st, to, ti) && wait_ge(a.rd + (size_t)q * kAdjParts + part, k, st, to, ti);
    }
    case TASK_TRTRI:  // (J=p): the factored diagonal tile
      return wait_ge(a.cK + tri(p, p), p + 1, st, to, ti);
    case TASK_RPOTRF: {  // (J=p): every part complete
      for (int part = 0; part < kAdjParts; ++part) {
        const int cnt = (a.Mt - 1 - p - part + kAdjParts - 1) / kAdjParts;
        if (cnt > 0 && !wait_ge(a.rd + (size_t)p * kAdjParts + part, cnt, st, to, ti)) return false;
      }
      return true;
    }
  }
  return false;
}

// The persistent kernel: each CTA repeatedly takes the next task in dispatch order, waits (bounded)
// until the counters of the tiles it reads say their producers are done, runs the tile operation,
// and publishes its own tile's counter. kMixed selects FP32 arithmetic for the trailing updates,
// the panel TRSMs after the first block column and the covariance solve; POTRF, the first block
// column's TRSM and the vector solves stay FP64.
// A batched launch (kBatch) runs the tasks of many independent GPs: each task names its GP in the
// high bits of its kind, and the CTA takes that GP's pointers and sizes from the descriptor table.
template <bool kMixed, bool kRev, bool kBatch>
__global__ void __launch_bounds__(kThreads, kMixed ? 1 : 2) dag_kernel(DagArgs a0) {
  union __align__(16) TileScratch {
    TileSmem d;
    TileSmemF32 f;
  };
  static_assert(alignof(TileScratch) >= 16, "the tile routines read their scratch with 16-byte vector loads");
  // Tensor-core path of the mixed trailing updates: TMEM accumulator and mbarriers per CTA.
  constexpr bool kUmma = kMixed && !kRev;
  extern __shared__ __align__(1024) uint8_t dyn_smem[];
  TileScratch* up;
  if constexpr (kUmma) {
    // the tile routines' scratch aliases the tensor-core stages: a task uses one or the other
    up = reinterpret_cast<TileScratch*>(((uintptr_t)dyn_smem + 1023) & ~(uintptr_t)1023);
  } else {
    __shared__ TileScratch u_static;
    up = &u_static;
  }
  TileScratch& u = *up;
  if (((uintptr_t)up & 15) != 0) {  // guard: the layout above must keep the scratch 16-byte aligned
    if (threadIdx.x == 0) raise_error(a0.st, GP_ERR_CUDA, -1);
    return;
  }
  __shared__ int s_task;
  __shared__ int s_flag;
  __shared__ double s_red[kThreads / 32][32];
  TileSmem& s = u.d;
  __shared__ uint64_t s_bar[2 + 2 * kPkStages];
  __shared__ uint64_t s_bsbar[2 * kBsMaxStages];
  __shared__ uint32_t s_tmem;
  UmmaState um;
  BsPipe bp;
  const bool use_umma = kUmma && a0.use_umma;
  if (kUmma && use_umma) {
    if (threadIdx.x < 32) {
      tmem_alloc(&s_tmem, kUmmaTmemCols);
      tmem_relinquish();
    }
    if (threadIdx.x == 0) {
      for (int b = 0; b < 2 + 2 * kPkStages; ++b) mbar_init(&s_bar[b], 1);
      for (int b = 0; b < 2 * kBsMaxStages; ++b) mbar_init(&s_bsbar[b], 1);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    umma_fence_before();
    __syncthreads();
    umma_fence_after();
    um.smem = reinterpret_cast<uint8_t*>(((uintptr_t)dyn_smem + 1023) & ~(uintptr_t)1023);
    um.bar = s_bar;
    um.tmem = s_tmem;
    um.phase[0] = um.phase[1] = 0;
    um.pending[0] = um.pending[1] = 0;
    um.pfull = s_bar + 2;
    um.pempty = s_bar + 2 + kPkStages;
    for (int b = 0; b < kPkStages; ++b) um.fph[b] = um.eph[b] = um.fpend[b] = um.epend[b] = 0;
    bp.full = s_bsbar;
    bp.empty = s_bsbar + kBsMaxStages;
    for (int b = 0; b < kBsMaxStages; ++b) bp.fph[b] = bp.eph[b] = bp.fpend[b] = bp.epend[b] = 0;
  }
  while (true) {
    if (threadIdx.x == 0) s_task = ld_relaxed(&a0.st->abort) ? INT_MAX : (int)atomicAdd(&a0.st->next_task, 1ull);
    __syncthreads();
    const int ti = s_task;
    __syncthreads();
    if (ti >= a0.ntasks) break;
    int4 tk = a0.tasks[ti];
    DagArgs a = a0;
    long long gp_tag = 0;  // error detail: GP index in the high 32 bits for batched launches
    if constexpr (kBatch) {
      const int g = tk.x >> kBatchKindBits;
      tk.x &= (1 << kBatchKindBits) - 1;
      const GpDesc& d = a0.descs[g];
      a.Kt = d.Kt;
      a.T = d.T;
      a.Mt = d.Mt;
      a.V = d.V;
      a.ldv = d.ldv;
      a.Mc = d.Mc;
      a.S = d.S;
      a.lds = d.lds;
      a.bvec = d.bvec;
      a.nch = d.nch;
      a.cK = d.cK;
      a.cV = d.cV;
      a.cS = d.cS;
      a.cF = d.cF;
      a.cB = d.cB;
      a.dF = d.dF;
      a.dB = d.dB;
      gp_tag = (long long)g << 32;
    }
    const int T = a.T;
    const size_t TT = (size_t)T * T;
    bool aborted = false;
    bool ok = true;
    long long t_taken = 0;
    if (a0.trace && threadIdx.x == 0) t_taken = (long long)globaltimer();
    if (threadIdx.x == 0) ok = wait_deps(a, tk, ti);
    if (__syncthreads_or(!ok)) break;
    if (a0.trace && threadIdx.x == 0) {
      long long* rec = a0.trace + 4 * (size_t)ti;
      rec[0] = blockIdx.x;
      rec[1] = t_taken;
      rec[2] = (long long)globaltimer();
    }
    const int p = tk.y, q = tk.z, r = tk.w;
    if (ti == a.withhold_task) continue;  // test hook: this task's completion is never published
    if constexpr (!kRev) {
      switch (tk.x) {
      case TASK_POTRF: {
        const int fail = (kUmma && use_umma && T <= 128)
                             ? cta_potrf_smem(a.Kt + tri(p, p) * TT, T, T, reinterpret_cast<double*>(um.smem),
                                              &s_red[0][0], &s_flag)
                             : cta_potrf<kMixed>(a.Kt + tri(p, p) * TT, T, T, s);
        if (fail) {
          if (threadIdx.x == 0) raise_error(a.st, GP_ERR_NOT_PD, gp_tag + (long long)p * T + fail);
          aborted = true;
          break;
        }
        if (kUmma && use_umma && a.PLinv && T == kUmmaM) {
          uint8_t* dst = a.PLinv + (size_t)p * TT * a.pkb;
          if (a.prec == GP_FP64_OZAKI) {
            // FP64 inverse of the factored tile (also the vector solves' Linv), packed as fixed-point
            // digits at its own scale for the column's TRSMs and V solves
            __syncthreads();
            double* Li = a.Linv + (size_t)p * TT;
            cta_inverse_f64_smem(um.smem, T, Li);  // from the factor left in shared memory
            const int e = cta_scale_exp(Li, T, T, T, &s_flag);
            if (threadIdx.x == 0) a.PLinvExp[p] = e;
            form_pack(a.prec, Li, T, false, T, T, dst, e);
          } else {  // FP32 inverse from the factor left in shared memory, packed in the form's format
            const float* Xs = cta_inverse_f32_smem(um.smem, T);
            form_pack_f32(a.prec, Xs, T + 1, T, dst);
          }
        }
        cta_publish(a.cK + tri(p, p), p + 1);
        break;
      }
      case TASK_TRSM:
        if (kUmma && use_umma && (q > 0 || a.prec == GP_FP64_OZAKI) && a.PLinv && a.Pk && T == kUmmaM) {
          // L_IJ = K_IJ X_J^T on the tensor cores, X_J the packed inverse of L_JJ (K_IJ packed first,
          // in the slot that then receives L_IJ; the FP64-emulating form also for the first column)
          double* Kij = a.Kt + tri(p, q) * TT;
          uint8_t* Pij = a.Pk + tri(p, q) * TT * a.pkb;
          const bool oz = a.prec == GP_FP64_OZAKI;
          const int eK = oz ? cta_scale_exp(Kij, T, T, T, &s_flag) : 0;
          form_pack(a.prec, Kij, T, false, T, T, Pij, eK);
          PkPairs pr;
          pr.n = 1;
          pr.A[0] = Pij;
          pr.B[0] = a.PLinv + (size_t)q * TT * a.pkb;
          const int eX = oz ? __ldcg(a.PLinvExp + q) : 0;
          if (!form_product<true>(um, bp, a.prec, Kij, T, pr, T, false, eK, eX, a.st, a.timeout_ns, ti)) {
            aborted = true;
            break;
          }
        } else if (kMixed && q > 0)
          cta_trsm_right_f32(a.Kt + tri(q, q) * TT, T, a.Kt + tri(p, q) * TT, T, T, T, u.f);
        else
          cta_trsm_right(a.Kt + tri(q, q) * TT, T, a.Kt + tri(p, q) * TT, T, T, T, s);
        if (kUmma && a.Pk && T % kUmmaM == 0) {  // the panel tile in the operand format of its readers
          __syncthreads();
          form_pack(a.prec, a.Kt + tri(p, q) * TT, T, false, T, T, a.Pk + tri(p, q) * TT * a.pkb, a.eL);
        }
        cta_publish(a.cK + tri(p, q), q + 1);
        break;
      case TASK_UPD:    // K_IK -= sum_{J0 <= J < J1} L_IJ L_KJ^T (SYRK when I == K), J in increasing order
      case TASK_UPD2: {  // the same for tiles (I, K) and (I + 1, K) together
        const int J0 = r & 0xFFFF, J1 = (r >> 16) ? (r >> 16) : J0 + 1;
        const int rows = tk.x == TASK_UPD2 ? 2 : 1;
        if (rows == 2 && kUmma && use_umma && a.Pk && T == kUmmaM && J1 - J0 <= kUmmaMaxPairs &&
            a.prec == GP_FP32) {
          PkPairs2 pr;
          pr.n = J1 - J0;
          for (int J = J0; J < J1; ++J) {
            pr.A0[J - J0] = a.Pk + tri(p, J) * TT * a.pkb;
            pr.A1[J - J0] = a.Pk + tri(p + 1, J) * TT * a.pkb;
            pr.B[J - J0] = a.Pk + tri(q, J) * TT * a.pkb;
          }
          if (!umma_pk_block2_sub(um, a.Kt + tri(p, q) * TT, a.Kt + tri(p + 1, q) * TT, T, pr, T, p == q, a.st,
                                  a.timeout_ns, ti)) {
            aborted = true;
            break;
          }
        } else {
          for (int I = p; I < p + rows && !aborted; ++I) {  // one tile at a time
            double* C = a.Kt + tri(I, q) * TT;
            if (kUmma && use_umma && a.Pk && T % kUmmaM == 0 && J1 - J0 <= kUmmaMaxPairs) {
              PkPairs pr;
              pr.n = J1 - J0;
              for (int J = J0; J < J1; ++J) {
                pr.A[J - J0] = a.Pk + tri(I, J) * TT * a.pkb;
                pr.B[J - J0] = a.Pk + tri(q, J) * TT * a.pkb;
              }
              if (!form_product<false>(um, bp, a.prec, C, T, pr, T, I == q, a.eL, a.eL, a.st, a.timeout_ns, ti))
                aborted = true;
            } else if (kUmma && use_umma && T % kUmmaM == 0 && J1 - J0 <= kUmmaMaxPairs) {
              UmmaPairs pr;
              pr.n = J1 - J0;
              for (int J = J0; J < J1; ++J) {
                pr.A[J - J0] = a.Kt + tri(I, J) * TT;
                pr.B[J - J0] = a.Kt + tri(q, J) * TT;
              }
              if (!umma_gemm_sub(um, C, T, pr, T, T, T, T, T, I == q, a.st, a.timeout_ns, ti)) aborted = true;
            } else {
              for (int J = J0; J < J1; ++J) {
                if (kMixed)
                  cta_gemm_sub_f32<0, 0>(C, T, a.Kt + tri(I, J) * TT, T, a.Kt + tri(q, J) * TT, T, T, T, T, I == q,
                                         u.f.g);
                else
                  cta_gemm_sub<A_MK, B_NK>(C, T, a.Kt + tri(I, J) * TT, T, a.Kt + tri(q, J) * TT, T, T, T, T, I == q,
                                           0, s.g);
              }
            }
          }
          if (aborted) break;
        }
        cta_publish(a.cK + tri(p, q), J1);
        if (rows == 2) cta_publish(a.cK + tri(p + 1, q), J1);
        break;
      }
      case TASK_VTRSM: {
        double* B = a.V + (size_t)p * T * a.ldv + (size_t)q * T;
        if (kUmma && use_umma && a.PLinv && a.PV && T == kUmmaM) {
          // V_Jc = X_J V_Jc on the tensor cores (V_Jc packed transposed first, in the slot that then
          // receives the solved block)
          uint8_t* Pjc = a.PV + ((size_t)p * a.Mc + q) * TT * a.pkb;
          const bool oz = a.prec == GP_FP64_OZAKI;
          const int eB = oz ? cta_scale_exp(B, (int)a.ldv, T, T, &s_flag) : 0;
          form_pack(a.prec, B, (int)a.ldv, true, T, T, Pjc, eB);
          PkPairs pr;
          pr.n = 1;
          pr.A[0] = a.PLinv + (size_t)p * TT * a.pkb;
          pr.B[0] = Pjc;
          const int eX = oz ? __ldcg(a.PLinvExp + p) : 0;
          if (!form_product<true>(um, bp, a.prec, B, (int)a.ldv, pr, T, false, eX, eB, a.st, a.timeout_ns, ti)) {
            aborted = true;
            break;
          }
        } else if (kMixed)
          cta_trsm_left_f32(a.Kt + tri(p, p) * TT, T, B, (int)a.ldv, T, T, u.f);
        else
          cta_trsm_left(a.Kt + tri(p, p) * TT, T, B, (int)a.ldv, T, T, s);
        if (kUmma && a.PV && T % kUmmaM == 0) {  // V_Jc is final: its transposed operand for V and W
          __syncthreads();
          form_pack(a.prec, B, (int)a.ldv, true, T, T, a.PV + ((size_t)p * a.Mc + q) * TT * a.pkb, a.eV);
        }
        cta_publish(a.cV + (size_t)p * a.Mc + q, p + 1);
        break;
      }
      case TASK_VGEMM: {
        double* C = a.V + (size_t)p * T * a.ldv + (size_t)r * T;
        const double* B = a.V + (size_t)q * T * a.ldv + (size_t)r * T;
        if (kUmma && use_umma && a.Pk && a.PV && T % kUmmaM == 0) {  // V_Ic -= L_IJ V_Jc, packed operands
          PkPairs pr;
          pr.n = 1;
          pr.A[0] = a.Pk + tri(p, q) * TT * a.pkb;
          pr.B[0] = a.PV + ((size_t)q * a.Mc + r) * TT * a.pkb;
          if (!form_product<false>(um, bp, a.prec, C, (int)a.ldv, pr, T, false, a.eL, a.eV, a.st, a.timeout_ns, ti)) {
            aborted = true;
            break;
          }
        } else if (kMixed)
          cta_gemm_sub_f32<0, 1>(C, (int)a.ldv, a.Kt + tri(p, q) * TT, T, B, (int)a.ldv, T, T, T, false, u.f.g);
        else
          cta_gemm_sub<A_MK, B_KN>(C, (int)a.ldv, a.Kt + tri(p, q) * TT, T, B, (int)a.ldv, T, T, T, false, 0, s.g);
        cta_publish(a.cV + (size_t)p * a.Mc + r, q + 1);
        break;
      }
      case TASK_WSYRK: {
        double* C = a.S + (size_t)p * T * a.lds + (size_t)q * T;
        const double* Va = a.V + (size_t)r * T * a.ldv + (size_t)p * T;
        const double* Vb = a.V + (size_t)r * T * a.ldv + (size_t)q * T;
        if (kUmma && use_umma && a.PV && T % kUmmaM == 0) {  // S_ab -= V_Ja^T V_Jb, packed operands
          PkPairs pr;
          pr.n = 1;
          pr.A[0] = a.PV + ((size_t)r * a.Mc + p) * TT * a.pkb;
          pr.B[0] = a.PV + ((size_t)r * a.Mc + q) * TT * a.pkb;
          if (!form_product<false>(um, bp, a.prec, C, (int)a.lds, pr, T, p == q, a.eV, a.eV, a.st, a.timeout_ns, ti)) {
            aborted = true;
            break;
          }
        } else if (kMixed)
          cta_gemm_sub_f32<1, 1>(C, (int)a.lds, Va, (int)a.ldv, Vb, (int)a.ldv, T, T, T, p == q, u.f.g);
        else
          cta_gemm_sub<A_KM, B_KN>(C, (int)a.lds, Va, (int)a.ldv, Vb, (int)a.ldv, T, T, T, p == q, 0, s.g);
        cta_publish(a.cS + tri(p, q), r + 1);
        break;
      }
      case TASK_VGEMM_G:    // V_Ic -= sum_J L_IJ V_Jc (packed operands, one pass over V_Ic)
      case TASK_WSYRK_G: {  // S_ab -= sum_J V_Ja^T V_Jb
        const int J0 = r & 0xFFFF, J1 = r >> 16;
        if (!(kUmma && use_umma && a.PV && T % kUmmaM == 0 && J1 - J0 <= kUmmaMaxPairs &&
              (tk.x == TASK_WSYRK_G || a.Pk))) {  // the host schedules these only for that path
          if (threadIdx.x == 0) raise_error(a.st, GP_ERR_INVALID_ARG, ti);
          aborted = true;
          break;
        }
        PkPairs pr;
        pr.n = J1 - J0;
        double* C;
        int ldc;
        if (tk.x == TASK_VGEMM_G) {
          C = a.V + (size_t)p * T * a.ldv + (size_t)q * T;
          ldc = (int)a.ldv;
          for (int J = J0; J < J1; ++J) {
            pr.A[J - J0] = a.Pk + tri(p, J) * TT * a.pkb;
            pr.B[J - J0] = a.PV + ((size_t)J * a.Mc + q) * TT * a.pkb;
          }
        } else {
          C = a.S + (size_t)p * T * a.lds + (size_t)q * T;
          ldc = (int)a.lds;
          for (int J = J0; J < J1; ++J) {
            pr.A[J - J0] = a.PV + ((size_t)J * a.Mc + p) * TT * a.pkb;
            pr.B[J - J0] = a.PV + ((size_t)J * a.Mc + q) * TT * a.pkb;
          }
        }
        const bool wg = tk.x == TASK_WSYRK_G;
        if (!form_product<false>(um, bp, a.prec, C, ldc, pr, T, wg && p == q, wg ? a.eV : a.eL, a.eV, a.st,
                                 a.timeout_ns, ti)) {
          aborted = true;
          break;
        }
        if (tk.x == TASK_VGEMM_G)
          cta_publish(a.cV + (size_t)p * a.Mc + q, J1);
        else
          cta_publish(a.cS + tri(p, q), J1);
        break;
      }
      case TASK_FSOLVE:
        if (a.Linv)
          cta_trsv_inv(a.Linv + (size_t)p * TT, T, a.bvec + (size_t)p * T, T, &s.g.a[0][0][0]);
        else
          cta_trsv_lower(a.Kt + tri(p, p) * TT, T, a.bvec + (size_t)p * T, T, &s_red[0][0], s.tri);
        cta_publish(a.dF + p, 1);
        break;
      case TASK_FGEMV:  // b_I[ch] -= L_IJ[ch, :] x_J, x_J in xvec for the chunked solves
        cta_gemv_sub(a.Kt + tri(p, q) * TT + (size_t)r * 32 * T, T, (a.xvec ? a.xvec : a.bvec) + (size_t)q * T,
                     a.bvec + (size_t)p * T + r * 32, 32, T);
        cta_publish(a.cF + (size_t)p * a.nch + r, q + 1);
        break;
      case TASK_FSOLVE_C:  // xvec_J[ch] = Linv_J[ch rows, :] bvec_J
        cta_gemv_sub<true>(a.Linv + (size_t)p * TT + (size_t)q * 32 * T, T, a.bvec + (size_t)p * T,
                           a.xvec + (size_t)p * T + q * 32, 32, T);
        cta_publish_add(a.dF + p);
        break;
      case TASK_BSOLVE_C:  // bvec_J[ch] = sum_r Linv_J[r][ch cols] xvec_J[r]
        cta_gemv_T_sub<true>(a.Linv + (size_t)p * TT + q * 32, T, a.xvec + (size_t)p * T,
                             a.bvec + (size_t)p * T + q * 32, T, 32, s_red);
        cta_publish_add(a.dB + p);
        break;
      case TASK_BSOLVE:
        if (a.Linv)
          cta_trsv_inv_T(a.Linv + (size_t)p * TT, T, a.bvec + (size_t)p * T, T, &s.g.a[0][0][0], s_red);
        else
          cta_trsv_lower_T(a.Kt + tri(p, p) * TT, T, a.bvec + (size_t)p * T, T, &s_red[0][0], s.tri);
        cta_publish(a.dB + p, 1);
        break;
      case TASK_TRTRI:  // read by later launches only: nothing to publish
        if (!(kUmma && use_umma && a.PLinv && T == kUmmaM && a.prec == GP_FP64_OZAKI))  // else done by POTRF
          cta_trtri(a.Kt + tri(p, p) * TT, T, a.Linv + (size_t)p * TT, T, s);
        break;
      case TASK_BGEMV:  // b_J[ch] -= L_IJ[:, ch]^T x_I; chunked solves: xvec_J[ch] -= L_IJ[:, ch]^T bvec_I
        cta_gemv_T_sub(a.Kt + tri(q, p) * TT + (size_t)r * 32, T, a.bvec + (size_t)q * T,
                       (a.xvec ? a.xvec : a.bvec) + (size_t)p * T + r * 32, T, 32, s_red);
        cta_publish(a.cB + (size_t)p * a.nch + r, a.Mt - q);
        break;
      }
    } else {
      switch (tk.x) {
      case TASK_RUPD: {  // Lbar_PJ -= Abar~_PK L_KJ, Abar~ the symmetric adjoint (diagonal tiles hold Abar + Abar^T)
        double* C = a.Bt + tri(p, r) * TT;
        const double* Lkj = a.Kt + tri(q, r) * TT;
        if (p >= q) {
          if (kMixed)
            cta_gemm_sub_f32<0, 1>(C, T, a.Bt + tri(p, q) * TT, T, Lkj, T, T, T, T, false, u.f.g);
          else
            cta_gemm_sub<A_MK, B_KN>(C, T, a.Bt + tri(p, q) * TT, T, Lkj, T, T, T, T, false, 0, s.g);
        } else {
          if (kMixed)
            cta_gemm_sub_f32<1, 1>(C, T, a.Bt + tri(q, p) * TT, T, Lkj, T, T, T, T, false, u.f.g);
          else
            cta_gemm_sub<A_KM, B_KN>(C, T, a.Bt + tri(q, p) * TT, T, Lkj, T, T, T, T, false, 0, s.g);
        }
        cta_publish(a.rc + tri(p, r), a.Mt - q);
        break;
      }
      case TASK_RTRSM:  // Abar_PJ = Lbar_PJ L_JJ^{-1}
        cta_trsm_right_N(a.Kt + tri(q, q) * TT, T, a.Bt + tri(p, q) * TT, T, T, T, s);
        cta_publish(a.fa + tri(p, q), 1);
        break;
      case TASK_RDIAG: {  // part_(P-J-1)%parts of Lbar_JJ -= tril(Abar_PJ^T L_PJ)
        const int part = (p - q - 1) % kAdjParts;
        double* Cp = a.Pt + ((size_t)q * kAdjParts + part) * TT;
        if (kMixed)
          cta_gemm_sub_f32<1, 1>(Cp, T, a.Bt + tri(p, q) * TT, T, a.Kt + tri(p, q) * TT, T, T, T, T, true, u.f.g);
        else
          cta_gemm_sub<A_KM, B_KN>(Cp, T, a.Bt + tri(p, q) * TT, T, a.Kt + tri(p, q) * TT, T, T, T, T, true, 0, s.g);
        cta_publish(a.rd + (size_t)q * kAdjParts + part, (p - q - 1) / kAdjParts + 1);
        break;
      }
      case TASK_RPOTRF: {  // Abar_JJ (+ its transpose) from Lbar_JJ, W = -L^{-T} Phi(L^T Lbar) L^{-1}
        const double* L = a.Kt + tri(p, p) * TT;
        double* B = a.Bt + tri(p, p) * TT;
        double* W = a.Wt + (size_t)p * TT;
        for (size_t e = threadIdx.x; e < TT; e += kThreads) {  // Lbar_JJ = initial + sum of the parts
          double acc = ldcg(B + e);
          for (int part = 0; part < kAdjParts; ++part) acc += ldcg(a.Pt + ((size_t)p * kAdjParts + part) * TT + e);
          B[e] = acc;
          W[e] = 0.0;
        }
        __syncthreads();
        cta_gemm_sub<A_KM, B_KN>(W, T, L, T, B, T, T, T, T, true, 0, s.g);  // W = -tril(L^T Lbar)
        for (int i = threadIdx.x; i < T; i += kThreads) W[(size_t)i * T + i] *= 0.5;
        __syncthreads();
        cta_trsm_right_N(L, T, W, T, T, T, s);
        cta_trsm_left_T(L, T, W, T, T, T, s);
        for (size_t e = threadIdx.x; e < TT; e += kThreads) {
          const size_t i = e / T, j = e % T;
          B[e] = -(ldcg(W + i * T + j) + ldcg(W + j * T + i));
        }
        cta_publish(a.fa + tri(p, p), 1);
        break;
      }
      }
    }
    if (aborted) break;  // uniform across the CTA (set after a barrier-synchronised decision)
    if (a0.trace && threadIdx.x == 0) a0.trace[4 * (size_t)ti + 3] = (long long)globaltimer();
  }
  if (kUmma && use_umma) {
    umma_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(um.tmem, kUmmaTmemCols);
  }
}

// Test hook behind gp_debug_tile_product: one CTA packs A and B (128 x K FP64, row-major) in the operand
// format of precision form `prec` into `work` and forms C (128 x 128, ldc 128) -= A B^T (store: C =
// A B^T) with the same device routines as the persistent kernel, `reps` times (the product is timed
// by the caller). The fixed-point form takes each operand's own scale (cta_scale_exp).
__global__ void __launch_bounds__(kThreads, 1) debug_product_kernel(int prec, const double* A, const double* B,
                                                                    double* C, int K, int store, int lower,
                                                                    uint8_t* work, size_t half_bytes, int reps,
                                                                    DevStatus* st, long long timeout_ns) {
  extern __shared__ __align__(1024) uint8_t dyn_smem[];
  __shared__ uint64_t s_bar[2 + 2 * kPkStages];
  __shared__ uint64_t s_bsbar[2 * kBsMaxStages];
  __shared__ uint32_t s_tmem;
  __shared__ int s_flag;
  UmmaState um;
  BsPipe bp;
  if (threadIdx.x < 32) {
    tmem_alloc(&s_tmem, kUmmaTmemCols);
    tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2 + 2 * kPkStages; ++b) mbar_init(&s_bar[b], 1);
    for (int b = 0; b < 2 * kBsMaxStages; ++b) mbar_init(&s_bsbar[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  umma_fence_before();
  __syncthreads();
  umma_fence_after();
  um.smem = reinterpret_cast<uint8_t*>(((uintptr_t)dyn_smem + 1023) & ~(uintptr_t)1023);
  um.bar = s_bar;
  um.tmem = s_tmem;
  um.phase[0] = um.phase[1] = 0;
  um.pending[0] = um.pending[1] = 0;
  um.pfull = s_bar + 2;
  um.pempty = s_bar + 2 + kPkStages;
  for (int b = 0; b < kPkStages; ++b) um.fph[b] = um.eph[b] = um.fpend[b] = um.epend[b] = 0;
  bp.full = s_bsbar;
  bp.empty = s_bsbar + kBsMaxStages;
  for (int b = 0; b < kBsMaxStages; ++b) bp.fph[b] = bp.eph[b] = bp.fpend[b] = bp.epend[b] = 0;
  const bool oz = prec == GP_FP64_OZAKI;
  const int eA = oz ? cta_scale_exp(A, K, kUmmaM, K, &s_flag) : 0;
  const int eB = oz ? cta_scale_exp(B, K, kUmmaM, K, &s_flag) : 0;
  form_pack(prec, A, K, false, kUmmaM, K, work, eA);
  form_pack(prec, B, K, false, kUmmaM, K, work + half_bytes, eB);
  PkPairs pr;
  pr.n = 1;
  pr.A[0] = work;
  pr.B[0] = work + half_bytes;
  bool ok = true;
  for (int it = 0; it < reps && ok; ++it) {
    switch (prec) {
      case GP_BF16:
        ok = store ? bs_block_sub<1, false, true>(um, bp, C, kUmmaN, pr, K, 0, 0, false, 0, 0, 0, st, timeout_ns, -2)
                   : bs_block_sub<1, false, false>(um, bp, C, kUmmaN, pr, K, 0, 0, lower, 0, 0, 0, st, timeout_ns, -2);
        break;
      case GP_BF16X3:
        ok = store ? bs_block_sub<2, false, true>(um, bp, C, kUmmaN, pr, K, 0, 0, false, 0, 0, 0, st, timeout_ns, -2)
                   : bs_block_sub<2, false, false>(um, bp, C, kUmmaN, pr, K, 0, 0, lower, 0, 0, 0, st, timeout_ns, -2);
        break;
      case GP_BF16X6:
        ok = store ? bs_block_sub<3, false, true>(um, bp, C, kUmmaN, pr, K, 0, 0, false, 0, 0, 0, st, timeout_ns, -2)
                   : bs_block_sub<3, false, false>(um, bp, C, kUmmaN, pr, K, 0, 0, lower, 0, 0, 0, st, timeout_ns, -2);
        break;
      case GP_FP64_OZAKI:
        ok = store ? bs_block_sub<kOzSlices, true, true>(um, bp, C, kUmmaN, pr, K, 0, 0, false, eA, eB, kOzLsbTile, st, timeout_ns, -2)
                   : bs_block_sub<kOzSlices, true, false>(um, bp, C, kUmmaN, pr, K, 0, 0, lower, eA, eB, kOzLsbTile, st,
                                                          timeout_ns, -2);
        break;
      case GP_TF32:
        ok = store ? umma_pk_block_sub<true, 1>(um, C, kUmmaN, pr, K, 0, 0, false, st, timeout_ns, -2)
                   : umma_pk_block_sub<false, 1>(um, C, kUmmaN, pr, K, 0, 0, lower, st, timeout_ns, -2);
        break;
      default:
        ok = store ? umma_pk_block_sub<true, 3>(um, C, kUmmaN, pr, K, 0, 0, false, st, timeout_ns, -2)
                   : umma_pk_block_sub<false, 3>(um, C, kUmmaN, pr, K, 0, 0, lower, st, timeout_ns, -2);
        break;
    }
  }
  umma_fence_before();
  __syncthreads();
  if (threadIdx.x < 32) tmem_dealloc(um.tmem, kUmmaTmemCols);
}

// r = y - K alpha for the 32 rows (tile row I = blockIdx.x / nch, chunk ch) from the packed lower
// FP64 tiles of the symmetric K (diagonal tiles hold both triangles): row part from tiles (I, J<=I),
// transposed part from tiles (J>I, I). Per-block partials (6 doubles): sum r^2, sum y^2,
// max |r|, max row sum |K_i.|, max |alpha|, max |y| (for the normwise backward error). kNorm = false
// skips the row sums of |K| (they do not change between refinement steps; entry 3 is then 0), which
// halves the kernel's FP64 work.
template <bool kNorm>
__global__ void __launch_bounds__(kThreads) residual_kernel(const double* __restrict__ Kt, int T, int Mt,
                                                            long long n, const double* __restrict__ y,
                                                            const double* __restrict__ alpha, double* __restrict__ r,
                                                            double* __restrict__ partial) {
  __shared__ double red[kThreads / 32][32];
  __shared__ double redabs[kThreads / 32][32];
  __shared__ double rowsum[32], rowabs[32];
  __shared__ double stat[6][32];
  const int nch = T / 32;
  const int I = blockIdx.x / nch, ch = blockIdx.x % nch;
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  const size_t TT = (size_t)T * T;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // rows ch*32 + w*4 + k, lane-partial
  double abs4[4] = {0.0, 0.0, 0.0, 0.0};
  for (int J = 0; J <= I; ++J) {
    const double* tile = Kt + tri(I, J) * TT + (size_t)(ch * 32 + w * 4) * T;
    const double* aJ = alpha + (size_t)J * T;
    for (int c = lane; c < T; c += 32) {
      const double av = aJ[c];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const double kv = tile[(size_t)k * T + c];
        acc[k] = fma(kv, av, acc[k]);
        if (kNorm) abs4[k] += fabs(kv);
      }
    }
  }
  double accT = 0.0, absT = 0.0;  // column ch*32 + lane, warp-partial over rows
  for (int J = I + 1; J < Mt; ++J) {
    const double* tile = Kt + tri(J, I) * TT + ch * 32 + lane;
    const double* aJ = alpha + (size_t)J * T;
    for (int rr = w; rr < T; rr += kThreads / 32) {
      const double kv = tile[(size_t)rr * T];
      accT = fma(kv, aJ[rr], accT);
      if (kNorm) absT += fabs(kv);
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
      abs4[k] += __shfl_xor_sync(0xffffffffu, abs4[k], o);
    }
  }
  red[w][lane] = accT;
  redabs[w][lane] = absT;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0, u = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) {
      t += red[q][threadIdx.x];
      u += redabs[q][threadIdx.x];
    }
    rowsum[threadIdx.x] = t;
    rowabs[threadIdx.x] = u;
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int row = ch * 32 + w * 4 + k;
      const long long gi = (long long)I * T + row;
      const double tot = acc[k] + rowsum[w * 4 + k];
      const bool in = gi < n;
      const double yi = in ? y[gi] : 0.0;
      const double ri = in ? yi - tot : 0.0;
      r[gi] = ri;
      const int q = w * 4 + k;
      stat[0][q] = ri * ri;
      stat[1][q] = yi * yi;
      stat[2][q] = fabs(ri);
      stat[3][q] = in ? abs4[k] + rowabs[q] : 0.0;
      stat[4][q] = in ? fabs(alpha[gi]) : 0.0;
      stat[5][q] = fabs(yi);
    }
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int k = 0; k < 32; ++k) t = threadIdx.x < 2 ? t + stat[threadIdx.x][k] : fmax(t, stat[threadIdx.x][k]);
    partial[6 * blockIdx.x + threadIdx.x] = t;
  }
}

// out[0..2) = sums and out[2..6) = maxima of the per-block residual partials; one CTA.
__global__ void __launch_bounds__(kThreads) reduce_residual_kernel(const double* __restrict__ partial, int nb,
                                                                   double* __restrict__ out) {
  __shared__ double red[6][kThreads / 32];
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nb; b += kThreads)
    for (int k = 0; k < 6; ++k) v[k] = k < 2 ? v[k] + partial[6 * b + k] : fmax(v[k], partial[6 * b + k]);
  for (int k = 0; k < 6; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double x = __shfl_xor_sync(0xffffffffu, v[k], o);
      v[k] = k < 2 ? v[k] + x : fmax(v[k], x);
    }
    if (threadIdx.x % 32 == 0) red[k][threadIdx.x / 32] = v[k];
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t = threadIdx.x < 2 ? t + red[threadIdx.x][q] : fmax(t, red[threadIdx.x][q]);
    out[threadIdx.x] = t;
  }
}

// Input check: any NaN or infinity among a[0..cnt) raises GP_ERR_NONFINITE with info = base + (index of
// the first such entry) + 1 (1-based; the smallest index wins). The exponent field is tested with
// integer operations, one warp ballot per 32 entries, one lane of a warp with a hit raises.
__global__ void scan_nonfinite_kernel(const double* __restrict__ a, long long cnt, long long base,
                                      DevStatus* st) {
  for (long long i0 = (long long)blockIdx.x * kThreads; i0 < cnt; i0 += (long long)gridDim.x * kThreads) {
    const long long i = i0 + threadIdx.x;
    bool bad = false;
    if (i < cnt) bad = ((__double_as_longlong(a[i]) >> 52) & 0x7ff) == 0x7ff;
    const unsigned hit = __ballot_sync(0xffffffffu, bad);
    if (hit && (int)(threadIdx.x & 31) == __ffs(hit) - 1) raise_error(st, GP_ERR_NONFINITE, base + i + 1);
  }
}

// alpha[i] += d[i] for i < n.
__global__ void axpy_kernel(double* __restrict__ alpha, const double* __restrict__ d, long long n) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
    alpha[i] += d[i];
}

// out[r*n + j] = lower triangle of the tiled matrix, rows row0.. row0+nrows (0 above the diagonal).
__global__ void factor_rows_kernel(const double* __restrict__ Kt, int T, long long n, long long row0,
                                   double* __restrict__ out) {
  const long long row = row0 + blockIdx.y;
  const long long I = row / T, r = row % T;
  for (long long j = (long long)blockIdx.x * kThreads + threadIdx.x; j < n; j += (long long)gridDim.x * kThreads) {
    double v = 0.0;
    if (j <= row) v = Kt[tri(I, j / T) * (size_t)T * T + (size_t)r * T + (j % T)];
    out[(size_t)blockIdx.y * n + j] = v;
  }
}

// log det K = 2 sum_{i<n} log L_ii over the diagonal tiles (one CTA).
__global__ void __launch_bounds__(kThreads) logdet_kernel(const double* __restrict__ Kt, int T, long long n,
                                                          double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += kThreads) {
    const long long I = i / T, r = i % T;
    s += log(Kt[tri(I, I) * (size_t)T * T + (size_t)r * T + r]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    out[0] = 2.0 * t;
  }
}

// beta_I[c] = sum_{K>=I} sum_r L_KI[r][c] alpha_K[r]  (beta = L^T alpha); one CTA per (I, 32-column chunk).
__global__ void __launch_bounds__(kThreads) beta_kernel(const double* __restrict__ Lt, int T, int Mt,
                                                        const double* __restrict__ alpha, double* __restrict__ beta) {
  __shared__ double red[kThreads / 32][32];
  const int nch = T / 32;
  const int I = blockIdx.x / nch, ch = blockIdx.x % nch;
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  const size_t TT = (size_t)T * T;
  double acc = 0.0;
  for (int K = I; K < Mt; ++K) {
    const double* tile = Lt + tri(K, I) * TT + ch * 32 + lane;
    const double* aK = alpha + (size_t)K * T;
    for (int rr = w; rr < T; rr += kThreads / 32) acc = fma(tile[(size_t)rr * T], aK[rr], acc);
  }
  red[w][lane] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q][threadIdx.x];
    beta[(size_t)I * T + ch * 32 + threadIdx.x] = t;
  }
}

// Lbar = -tril(alpha beta^T) + diag(1/L_ii) on the first n rows/columns, 0 elsewhere (and above the
// diagonal of diagonal tiles). Tile blockIdx.x, rows [blockIdx.y*32, +32).
__global__ void __launch_bounds__(kThreads) init_lbar_kernel(const double* __restrict__ Lt, double* __restrict__ Bt,
                                                             int T, long long n, const double* __restrict__ alpha,
                                                             const double* __restrict__ beta) {
  const long long t = blockIdx.x;
  long long I = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > t) --I;
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  const long long J = t - I * (I + 1) / 2;
  const size_t base = (size_t)t * T * T;
  for (int e = threadIdx.x; e < 32 * T; e += kThreads) {
    const int r = blockIdx.y * 32 + e / T, c = e % T;
    const long long i = I * T + r, j = J * T + c;
    double v = 0.0;
    if (i < n && j < n && i >= j) {
      v = -alpha[i] * beta[j];
      if (i == j) v += 1.0 / Lt[base + (size_t)r * T + c];
    }
    Bt[base + (size_t)r * T + c] = v;
  }
}

// Per-(tile, 32-row chunk) partial sums of Abar_ij * dK_ij/dtheta over stored lower entries with
// i, j < n, theta = (l, v, s2), the kernel entries recomputed from X.
template <int D>
__global__ void __launch_bounds__(kThreads) grad_contract_kernel(const double* __restrict__ Bt, int T,
                                                                 const double* __restrict__ X, long long n, int Dr,
                                                                 double l, double v, double* __restrict__ partial,
                                                                 const long long* __restrict__ Q,
                                                                 const FxScale* __restrict__ fx) {
  __shared__ double red[3][kThreads / 32];
  const long long t = blockIdx.x;
  long long I = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > t) --I;
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  const long long J = t - I * (I + 1) / 2;
  const size_t base = (size_t)t * T * T;
  const double neg_half_inv_l2 = -0.5 / (l * l), inv_l3 = 1.0 / (l * l * l);
  double gl = 0.0, gv = 0.0, gs = 0.0;
  for (int e = threadIdx.x; e < 32 * T; e += kThreads) {
    const int r = blockIdx.y * 32 + e / T, c = e % T;
    const long long i = I * T + r, j = J * T + c;
    if (i >= n || j >= n || j > i) continue;
    double wgt = Bt[base + (size_t)r * T + c];
    if (i == j) wgt *= 0.5;  // diagonal tiles hold Abar + Abar^T
    const double r2 = (D > 0 && Q != nullptr && fx->usable) ? fx_sqdist_rt(Q + i * Dr, Q + j * Dr, Dr, 2 * fx->F)
                                                            : sqdist_t<D>(X + i * Dr, X + j * Dr, Dr);
    const double ex = exp_neg(r2 * neg_half_inv_l2);
    gl = fma(wgt, v * ex * r2 * inv_l3, gl);
    gv = fma(wgt, ex, gv);
    if (i == j) gs += wgt;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gl += __shfl_xor_sync(0xffffffffu, gl, o);
    gv += __shfl_xor_sync(0xffffffffu, gv, o);
    gs += __shfl_xor_sync(0xffffffffu, gs, o);
  }
  if (threadIdx.x % 32 == 0) {
    red[0][threadIdx.x / 32] = gl;
    red[1][threadIdx.x / 32] = gv;
    red[2][threadIdx.x / 32] = gs;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) s += red[threadIdx.x][q];
    partial[3 * ((size_t)blockIdx.x * gridDim.y + blockIdx.y) + threadIdx.x] = s;
  }
}

// out[k] = sum_b partial[3b + k], k < 3 (one CTA, fixed order).
__global__ void __launch_bounds__(kThreads) sum3_kernel(const double* __restrict__ partial, long long nb,
                                                        double* __restrict__ out) {
  __shared__ double red[3][kThreads / 32];
  double s[3] = {0.0, 0.0, 0.0};
  for (long long b = threadIdx.x; b < nb; b += kThreads)
    for (int k = 0; k < 3; ++k) s[k] += partial[3 * b + k];
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if (threadIdx.x % 32 == 0) red[k][threadIdx.x / 32] = s[k];
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[threadIdx.x][q];
    out[threadIdx.x] = t;
  }
}

__global__ void __launch_bounds__(kThreads) dot_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                       long long n, double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += kThreads) s = fma(a[i], b[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    out[0] = t;
  }
}

// Pieces of the Arnoldi process of GMRES-based refinement (FP64): out[i] = <V_i, w> for i < k, V_i the
// rows of V (leading dimension ldv), one CTA per i, fixed summation order.
__global__ void __launch_bounds__(kThreads) multi_dot_kernel(const double* __restrict__ V, long long ldv,
                                                             const double* __restrict__ w, long long n,
                                                             double* __restrict__ out) {
  __shared__ double red[kThreads / 32];
  const double* v = V + (size_t)blockIdx.x * ldv;
  double s = 0.0;
  for (long long i = threadIdx.x; i < n; i += kThreads) s = fma(v[i], w[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (threadIdx.x % 32 == 0) red[threadIdx.x / 32] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q];
    out[blockIdx.x] = t;
  }
}

// w[i] += sign * sum_{j<k} h[j] V_j[i] (h on the device).
__global__ void multi_axpy_kernel(double* __restrict__ w, const double* __restrict__ V, long long ldv,
                                  const double* __restrict__ h, int k, double sign, long long n) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(h[j], V[(size_t)j * ldv + i], acc);
    w[i] = fma(sign, acc, w[i]);
  }
}

// dst[i] = src[i] * a for i < n.
__global__ void scale_copy_kernel(double* __restrict__ dst, const double* __restrict__ src, double a, long long n) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads)
    dst[i] = src[i] * a;
}

// diag(K) += tau on the first n rows of the packed lower tiles (the shifted factorisation of the
// single-product forms; the stored FP64 copy of K keeps the unshifted matrix).
__global__ void add_diag_kernel(double* __restrict__ Kt, int T, long long n, double tau) {
  for (long long i = (long long)blockIdx.x * kThreads + threadIdx.x; i < n; i += (long long)gridDim.x * kThreads) {
    const long long I = i / T, r = i % T;
    Kt[tri(I, I) * (size_t)T * T + (size_t)r * T + r] += tau;
  }
}

// Per GP (one CTA each): the common scale over X and Xs (fx_decide), then both sets quantised.
__global__ void __launch_bounds__(1024) batch_fx_kernel(const GpDesc* __restrict__ descs) {
  __shared__ double red[32];
  __shared__ int bad[32];
  __shared__ FxScale sc;
  const GpDesc& d = descs[blockIdx.x];
  const long long nx = d.n * d.D, ns = d.m * d.D;
  double mx = 0.0;
  int nonfinite = 0;
  for (long long e = threadIdx.x; e < nx + ns; e += blockDim.x) {
    const double x = e < nx ? d.X[e] : d.Xs[e - nx];
    if (!(fabs(x) <= 1.7976931348623157e308)) nonfinite = 1;
    else mx = fmax(mx, fabs(x));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    nonfinite |= __shfl_xor_sync(0xffffffffu, nonfinite, o);
  }
  if (threadIdx.x % 32 == 0) {
    red[threadIdx.x / 32] = mx;
    bad[threadIdx.x / 32] = nonfinite;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0;
    int nf = 0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      S = fmax(S, red[w]);
      nf |= bad[w];
    }
    sc = fx_decide(S, nf, d.D, d.l);
    *d.fx = sc;
  }
  __syncthreads();
  if (!sc.usable) return;
  const double scale = ldexp(1.0, sc.F);
  for (long long e = threadIdx.x; e < nx + ns; e += blockDim.x) {
    if (e < nx)
      d.QX[e] = __double2ll_rn(d.X[e] * scale);
    else
      d.QXs[e - nx] = __double2ll_rn(d.Xs[e - nx] * scale);
  }
}

// Batched assembly and right-hand sides, one work item per CTA (see launch_batch_pre).
__global__ void __launch_bounds__(kThreads) batch_pre_kernel(const int4* __restrict__ items,
                                                             const GpDesc* __restrict__ descs, int noisy_prior) {
  const int4 it = items[blockIdx.x];
  const GpDesc& d = descs[it.y];
  const double c = -0.5 / (d.l * d.l);
  const int T = d.T;
  if (it.x == 0) {  // K tile it.z, rows [it.w*32, +32)
    const long long t = it.z;
    long long I = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while (I * (I + 1) / 2 > t) --I;
    while ((I + 1) * (I + 2) / 2 <= t) ++I;
    const long long J = t - I * (I + 1) / 2;
    double* tile = d.Kt + (size_t)t * T * T;
    const bool use_fx = d.fx && d.fx->usable;
    const int twoF = use_fx ? 2 * d.fx->F : 0;
    for (int e = threadIdx.x; e < 32 * T; e += kThreads) {
      const int r = it.w * 32 + e / T, cc = e % T;
      const long long i = I * T + r, j = J * T + cc;
      double val;
      if (i < d.n && j < d.n)
        val = d.v * exp_neg((use_fx ? fx_sqdist_rt(d.QX + i * d.D, d.QX + j * d.D, d.D, twoF)
                                    : sqdist_t<0>(d.X + i * d.D, d.X + j * d.D, d.D)) * c) +
              (i == j ? d.s2 : 0.0);
      else
        val = (i == j) ? 1.0 : 0.0;
      tile[(size_t)r * T + cc] = val;
    }
  } else if (it.x == 1 || it.x == 2) {  // dense rows [it.z, it.z + 8) of K_{X,Xs} (V) or K_{Xs,Xs} (S)
    const bool isV = it.x == 1;
    double* out = isV ? d.V : d.S;
    const long long ld = isV ? d.ldv : d.lds;
    const double* A = isV ? d.X : d.Xs;
    const long long na = isV ? d.n : d.m;
    const double diag = (!isV && noisy_prior) ? d.s2 : 0.0;
    const long long* QA = isV ? d.QX : d.QXs;
    const bool use_fx = d.fx && d.fx->usable;
    const int twoF = use_fx ? 2 * d.fx->F : 0;
    for (int q = 0; q < 8; ++q) {
      const long long i = (long long)it.z + q;
      for (long long j = threadIdx.x; j < ld; j += kThreads) {
        double val = 0.0;
        if (i < na && j < d.m)
          val = d.v * exp_neg((use_fx ? fx_sqdist_rt(QA + i * d.D, d.QXs + j * d.D, d.D, twoF)
                                      : sqdist_t<0>(A + i * d.D, d.Xs + j * d.D, d.D)) * c) +
                ((!isV && i == j) ? diag : 0.0);
        out[(size_t)i * ld + j] = val;
      }
    }
  } else {  // right-hand side of the mean solve
    const long long npad = (long long)d.Mt * T;
    for (long long i = threadIdx.x; i < npad; i += kThreads) d.bvec[i] = i < d.n ? d.y[i] : 0.0;
  }
}

// Batched outputs: fused mean GEMV (8 test points per item) and covariance copy (8 rows per item).
__global__ void __launch_bounds__(kThreads) batch_post_kernel(const int4* __restrict__ items,
                                                              const GpDesc* __restrict__ descs) {
  __shared__ double red[8][kThreads / 32];
  const int4 it = items[blockIdx.x];
  const GpDesc& d = descs[it.y];
  if (it.x == 0) {
    const double c = -0.5 / (d.l * d.l);
    const long long i0 = it.z;
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    const bool use_fx = d.fx && d.fx->usable;
    const int twoF = use_fx ? 2 * d.fx->F : 0;
    for (long long j = threadIdx.x; j < d.n; j += kThreads) {
      const double aj = d.bvec[j];
#pragma unroll
      for (int q = 0; q < 8; ++q)
        if (i0 + q < d.m) {
          const double r2 = use_fx ? fx_sqdist_rt(d.QXs + (i0 + q) * d.D, d.QX + j * d.D, d.D, twoF)
                                   : sqdist_t<0>(d.Xs + (i0 + q) * d.D, d.X + j * d.D, d.D);
          acc[q] = fma(d.v * exp_neg(r2 * c), aj, acc[q]);
        }
    }
    const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      double v = acc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) red[q][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 8 && i0 + threadIdx.x < d.m) {
      double t = 0.0;
      for (int q = 0; q < kThreads / 32; ++q) t += red[threadIdx.x][q];
      d.mean[i0 + threadIdx.x] = t;
    }
  } else if (d.cov) {
    for (int q = 0; q < 8; ++q) {
      const long long a = (long long)it.z + q;
      if (a >= d.m) break;
      for (long long b = threadIdx.x; b < d.m; b += kThreads)
        d.cov[a * d.m + b] = (a >= b) ? d.S[a * d.lds + b] : d.S[b * d.lds + a];
    }
  }
}

// var[j] = k(Xs_j, Xs_j) (+ s2 when noisy) - sum_i V[i][j]^2: the diagonal of Eq. (3) without forming
// V^T V. One thread per test column, rows in order (deterministic), coalesced across threads.
__global__ void __launch_bounds__(kThreads) var_from_v_kernel(const double* __restrict__ V, long long ldv,
                                                              long long nrows, double v, double diag_add,
                                                              double* __restrict__ var, long long m) {
  const long long j = (long long)blockIdx.x * kThreads + threadIdx.x;
  if (j >= m) return;
  double s = 0.0;
  for (long long i = 0; i < nrows; ++i) {
    const double x = V[i * ldv + j];
    s = fma(x, x, s);
  }
  var[j] = (v + diag_add) - s;
}

// ---------------------------------------------------------------- host launchers

__global__ void exp_neg_kernel(const double* __restrict__ x, long long n, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = exp_neg(x[i]);
}

double fx_sqdist_host(const long long* qa, const long long* qb, int D, int twoF) {
  U128 acc{0ull, 0ull};
  for (int d = 0; d < D; ++d) fx_add_sq(acc, qa[d], qb[d]);
  return fx_to_double(acc, twoF);
}

cudaError_t launch_exp_neg(const double* x, long long n, double* out, int sms, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long want = (n + kThreads - 1) / kThreads;
  exp_neg_kernel<<<(unsigned)(want < (long long)sms * 8 ? want : (long long)sms * 8), kThreads, 0, st>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t launch_fx_prepare(const double* A, long long na, const double* B, long long nb, int D, double l, FxScale* out,
                              int sms, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(FxScale), st);
  if (e != cudaSuccess) return e;
  const long long want = ((na + nb) * D + kThreads - 1) / kThreads;
  const long long grid = want < 1 ? 1 : (want < (long long)sms * 4 ? want : (long long)sms * 4);
  fx_reduce_kernel<<<(unsigned)grid, kThreads, 0, st>>>(A, na, B, nb, D, out);
  fx_decide_kernel<<<1, 1, 0, st>>>(D, l, out);
  return cudaGetLastError();
}

cudaError_t launch_fx_quantize(const double* X, long long cnt, const FxScale* fx, long long* Q, int sms, cudaStream_t st) {
  if (cnt <= 0) return cudaSuccess;
  const long long want = (cnt + kThreads - 1) / kThreads;
  const unsigned grid = (unsigned)(want < (long long)sms * 8 ? want : (long long)sms * 8);
  fx_quantize_kernel<<<grid, kThreads, 0, st>>>(X, cnt, fx, Q);
  return cudaGetLastError();
}

cudaError_t launch_assemble_tiles(const double* X, long long n, int D, double l, double v, double s2, double* Kt, int T,
                                  int Mt, cudaStream_t st, const long long* Q, const FxScale* fx) {
  const long long ntiles = (long long)Mt * (Mt + 1) / 2;
  if (ntiles == 0) return cudaSuccess;
  dim3 grid((unsigned)ntiles, (unsigned)(T / 32));
  const double c = -0.5 / (l * l);
  switch (D) {
    case 4: assemble_tiles_kernel<4><<<grid, kThreads, 0, st>>>(X, n, D, c, v, s2, Kt, T, Q, fx); break;
    case 8: assemble_tiles_kernel<8><<<grid, kThreads, 0, st>>>(X, n, D, c, v, s2, Kt, T, Q, fx); break;
    case 16: assemble_tiles_kernel<16><<<grid, kThreads, 0, st>>>(X, n, D, c, v, s2, Kt, T, Q, fx); break;
    default: assemble_tiles_kernel<0><<<grid, kThreads, 0, st>>>(X, n, D, c, v, s2, Kt, T, nullptr, nullptr); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_assemble_dense(const double* A, long long na, const double* B, long long nb, int D, double l,
                                  double v, double diag_add, double* out, long long ld, long long rows_pad,
                                  long long cols_pad, cudaStream_t st, const long long* QA, const long long* QB,
                                  const FxScale* fx) {
  if (rows_pad == 0 || cols_pad == 0) return cudaSuccess;
  dim3 grid((unsigned)((cols_pad + 127) / 128), (unsigned)((rows_pad + 7) / 8));
  const double c = -0.5 / (l * l);
  switch (D) {
    case 4: assemble_dense_kernel<4><<<grid, kThreads, 0, st>>>(A, na, B, nb, D, c, v, diag_add, out, ld, rows_pad, cols_pad, QA, QB, fx); break;
    case 8: assemble_dense_kernel<8><<<grid, kThreads, 0, st>>>(A, na, B, nb, D, c, v, diag_add, out, ld, rows_pad, cols_pad, QA, QB, fx); break;
    case 16: assemble_dense_kernel<16><<<grid, kThreads, 0, st>>>(A, na, B, nb, D, c, v, diag_add, out, ld, rows_pad, cols_pad, QA, QB, fx); break;
    default: assemble_dense_kernel<0><<<grid, kThreads, 0, st>>>(A, na, B, nb, D, c, v, diag_add, out, ld, rows_pad, cols_pad, nullptr, nullptr, nullptr); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_mean_gemv(const double* Xs, long long m, const double* X, long long n, int D, double l, double v,
                             const double* alpha, double* mean, cudaStream_t st, const long long* QXs,
                             const long long* QX, const FxScale* fx) {
  if (m == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((m + 7) / 8);
  const double c = -0.5 / (l * l);
  switch (D) {
    case 4: mean_gemv_kernel<4><<<grid, kThreads, 0, st>>>(Xs, m, X, n, D, c, v, alpha, mean, QXs, QX, fx); break;
    case 8: mean_gemv_kernel<8><<<grid, kThreads, 0, st>>>(Xs, m, X, n, D, c, v, alpha, mean, QXs, QX, fx); break;
    case 16: mean_gemv_kernel<16><<<grid, kThreads, 0, st>>>(Xs, m, X, n, D, c, v, alpha, mean, QXs, QX, fx); break;
    default: mean_gemv_kernel<0><<<grid, kThreads, 0, st>>>(Xs, m, X, n, D, c, v, alpha, mean, nullptr, nullptr, nullptr); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_var_from_v(const double* V, long long ldv, long long nrows, double v, double diag_add, double* var,
                              long long m, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  var_from_v_kernel<<<(unsigned)((m + kThreads - 1) / kThreads), kThreads, 0, st>>>(V, ldv, nrows, v, diag_add, var, m);
  return cudaGetLastError();
}

cudaError_t launch_cov_copy(const double* S, long long lds, double* cov, long long m, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  dim3 grid((unsigned)((m + kThreads - 1) / kThreads), (unsigned)(m < 65535 ? m : 65535));
  cov_copy_kernel<<<grid, kThreads, 0, st>>>(S, lds, cov, m);
  return cudaGetLastError();
}

cudaError_t launch_logdet(const double* Kt, int T, long long n, double* out, cudaStream_t st) {
  logdet_kernel<<<1, kThreads, 0, st>>>(Kt, T, n, out);
  return cudaGetLastError();
}

cudaError_t launch_factor_rows(const double* Kt, int T, long long n, long long row0, long long nrows, double* out,
                               cudaStream_t st) {
  if (nrows <= 0) return cudaSuccess;
  for (long long r = 0; r < nrows; r += 65535) {
    const long long cnt = (nrows - r) < 65535 ? (nrows - r) : 65535;
    const long long bx = (n + kThreads - 1) / kThreads;
    dim3 grid((unsigned)(bx < 64 ? bx : 64), (unsigned)cnt);
    factor_rows_kernel<<<grid, kThreads, 0, st>>>(Kt, T, n, row0 + r, out + (size_t)r * n);
  }
  return cudaGetLastError();
}

// Dynamic shared memory of the forward mixed kernel: the tensor-core stages, or (without the tensor
// cores) just the tile routines' scratch, which lives there in both cases.
static int mixed_dyn_smem(int use_umma) {
  return use_umma ? kUmmaSmemBytes : (int)(sizeof(TileSmem) > sizeof(TileSmemF32) ? sizeof(TileSmem) : sizeof(TileSmemF32)) + 1024;
}

cudaError_t launch_dag(const DagArgs& a, int grid, bool mixed, cudaStream_t st, bool reverse, bool batch) {
  if (a.ntasks == 0) return cudaSuccess;
  if (batch) {
    if (mixed)
      dag_kernel<true, false, true><<<grid, kThreads, mixed_dyn_smem(a.use_umma), st>>>(a);
    else
      dag_kernel<false, false, true><<<grid, kThreads, 0, st>>>(a);
  } else if (reverse) {
    if (mixed)
      dag_kernel<true, true, false><<<grid, kThreads, 0, st>>>(a);
    else
      dag_kernel<false, true, false><<<grid, kThreads, 0, st>>>(a);
  } else {
    if (mixed)
      dag_kernel<true, false, false><<<grid, kThreads, mixed_dyn_smem(a.use_umma), st>>>(a);
    else
      dag_kernel<false, false, false><<<grid, kThreads, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_debug_product(int prec, const double* A, const double* B, double* C, int K, int store, int lower,
                                 uint8_t* work, size_t half_bytes, int reps, DevStatus* st, long long timeout_ns,
                                 cudaStream_t stream) {
  cudaError_t e = cudaFuncSetAttribute(debug_product_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kUmmaSmemBytes);
  if (e != cudaSuccess) return e;
  debug_product_kernel<<<1, kThreads, kUmmaSmemBytes, stream>>>(prec, A, B, C, K, store, lower, work, half_bytes,
                                                                 reps, st, timeout_ns);
  return cudaGetLastError();
}

cudaError_t dag_enable_umma() {
  cudaError_t e = cudaFuncSetAttribute(dag_kernel<true, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kUmmaSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dag_kernel<true, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kUmmaSmemBytes);
  return e;
}

// Resident CTAs per SM of the forward kernels, with the dynamic shared memory launch_dag gives them.
int dag_max_ctas_per_sm_batch(bool mixed, int use_umma) {
  int nb = 0;
  if (mixed)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dag_kernel<true, false, true>, kThreads,
                                                  mixed_dyn_smem(use_umma));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dag_kernel<false, false, true>, kThreads, 0);
  return nb;
}

int dag_max_ctas_per_sm(bool mixed, int use_umma) {
  int nb = 0;
  if (mixed)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dag_kernel<true, false, false>, kThreads,
                                                  mixed_dyn_smem(use_umma));
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dag_kernel<false, false, false>, kThreads, 0);
  return nb;
}

cudaError_t launch_residual(const double* Kt, int T, int Mt, long long n, const double* y, const double* alpha,
                            double* r, double* partial, double* norms, cudaStream_t st, bool with_knorm) {
  const int nb = Mt * (T / 32);
  if (with_knorm)
    residual_kernel<true><<<nb, kThreads, 0, st>>>(Kt, T, Mt, n, y, alpha, r, partial);
  else
    residual_kernel<false><<<nb, kThreads, 0, st>>>(Kt, T, Mt, n, y, alpha, r, partial);
  reduce_residual_kernel<<<1, kThreads, 0, st>>>(partial, nb, norms);
  return cudaGetLastError();
}

cudaError_t launch_batch_fx(const GpDesc* descs, int B, cudaStream_t st) {
  if (B <= 0) return cudaSuccess;
  batch_fx_kernel<<<B, 1024, 0, st>>>(descs);
  return cudaGetLastError();
}

cudaError_t launch_batch_pre(const int4* items, int nitems, const GpDesc* descs, bool noisy_prior, cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  batch_pre_kernel<<<nitems, kThreads, 0, st>>>(items, descs, noisy_prior ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_batch_post(const int4* items, int nitems, const GpDesc* descs, cudaStream_t st) {
  if (nitems == 0) return cudaSuccess;
  batch_post_kernel<<<nitems, kThreads, 0, st>>>(items, descs);
  return cudaGetLastError();
}

cudaError_t launch_beta(const double* Lt, int T, int Mt, const double* alpha, double* beta, cudaStream_t st) {
  beta_kernel<<<Mt * (T / 32), kThreads, 0, st>>>(Lt, T, Mt, alpha, beta);
  return cudaGetLastError();
}

cudaError_t launch_init_lbar(const double* Lt, double* Bt, int T, int Mt, long long n, const double* alpha,
                             const double* beta, cudaStream_t st) {
  dim3 grid((unsigned)((long long)Mt * (Mt + 1) / 2), (unsigned)(T / 32));
  init_lbar_kernel<<<grid, kThreads, 0, st>>>(Lt, Bt, T, n, alpha, beta);
  return cudaGetLastError();
}

cudaError_t launch_grad_contract(const double* Bt, int T, int Mt, const double* X, long long n, int D, double l,
                                 double v, double* partial, double* out, cudaStream_t st, const long long* Q,
                                 const FxScale* fx) {
  const long long ntiles = (long long)Mt * (Mt + 1) / 2;
  dim3 grid((unsigned)ntiles, (unsigned)(T / 32));
  switch (D) {
    case 4: grad_contract_kernel<4><<<grid, kThreads, 0, st>>>(Bt, T, X, n, D, l, v, partial, Q, fx); break;
    case 8: grad_contract_kernel<8><<<grid, kThreads, 0, st>>>(Bt, T, X, n, D, l, v, partial, Q, fx); break;
    case 16: grad_contract_kernel<16><<<grid, kThreads, 0, st>>>(Bt, T, X, n, D, l, v, partial, Q, fx); break;
    default: grad_contract_kernel<0><<<grid, kThreads, 0, st>>>(Bt, T, X, n, D, l, v, partial, nullptr, nullptr); break;
  }
  sum3_kernel<<<1, kThreads, 0, st>>>(partial, ntiles * (T / 32), out);
  return cudaGetLastError();
}

cudaError_t launch_dot(const double* a, const double* b, long long n, double* out, cudaStream_t st) {
  dot_kernel<<<1, kThreads, 0, st>>>(a, b, n, out);
  return cudaGetLastError();
}

cudaError_t launch_scan_nonfinite(const double* a, long long cnt, long long base, DevStatus* status,
                                  cudaStream_t st) {
  if (cnt <= 0) return cudaSuccess;
  const long long b = (cnt + kThreads - 1) / kThreads;
  scan_nonfinite_kernel<<<(unsigned)(b < 1216 ? b : 1216), kThreads, 0, st>>>(a, cnt, base, status);
  return cudaGetLastError();
}

cudaError_t launch_multi_dot(const double* V, long long ldv, int k, const double* w, long long n, double* out,
                             cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  multi_dot_kernel<<<k, kThreads, 0, st>>>(V, ldv, w, n, out);
  return cudaGetLastError();
}

cudaError_t launch_multi_axpy(double* w, const double* V, long long ldv, const double* h, int k, double sign,
                              long long n, cudaStream_t st) {
  if (k <= 0 || n <= 0) return cudaSuccess;
  const long long b = (n + kThreads - 1) / kThreads;
  multi_axpy_kernel<<<(unsigned)(b < 1216 ? b : 1216), kThreads, 0, st>>>(w, V, ldv, h, k, sign, n);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(double* dst, const double* src, double a, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long b = (n + kThreads - 1) / kThreads;
  scale_copy_kernel<<<(unsigned)(b < 1216 ? b : 1216), kThreads, 0, st>>>(dst, src, a, n);
  return cudaGetLastError();
}

cudaError_t launch_add_diag(double* Kt, int T, long long n, double tau, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const long long b = (n + kThreads - 1) / kThreads;
  add_diag_kernel<<<(unsigned)(b < 1216 ? b : 1216), kThreads, 0, st>>>(Kt, T, n, tau);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* alpha, const double* d, long long n, cudaStream_t st) {
  const long long b = (n + kThreads - 1) / kThreads;
  axpy_kernel<<<(unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096), kThreads, 0, st>>>(alpha, d, n);
  return cudaGetLastError();
}

}  // namespace gpk
