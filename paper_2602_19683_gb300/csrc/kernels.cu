// Device kernels of the GP hot path: covariance assembly (Eq. 1), the persistent task-DAG kernel that
// runs the tiled Cholesky (Sec. 3.2, Fig. 1) and the tiled solves of Eqs. (2)-(3), and the fused
// cross-covariance GEMV of the predictive mean.
#include <climits>

#include "kernels.h"
#include "tiles_f32.cuh"

namespace gpk {

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

// Lower tiles of K: tile blockIdx.x (packed index), rows [blockIdx.y*32, +32) of it. Entries
// outside the n x n matrix form the identity padding.
template <int D>
__global__ void __launch_bounds__(kThreads) assemble_tiles_kernel(const double* __restrict__ X, long long n, int Dr,
                                                                  double neg_half_inv_l2, double v, double s2,
                                                                  double* __restrict__ Kt, int T) {
  const long long t = blockIdx.x;
  long long I = (long long)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while (I * (I + 1) / 2 > t) --I;
  while ((I + 1) * (I + 2) / 2 <= t) ++I;
  const long long J = t - I * (I + 1) / 2;
  double* tile = Kt + (size_t)t * T * T;
  const int r0 = blockIdx.y * 32;
  for (int e = threadIdx.x; e < 32 * T; e += kThreads) {
    const int r = r0 + e / T, c = e % T;
    const long long i = I * T + r, j = J * T + c;
    double val;
    if (i < n && j < n) {
      const double r2 = sqdist_t<D>(X + i * Dr, X + j * Dr, Dr);
      val = v * exp(r2 * neg_half_inv_l2) + (i == j ? s2 : 0.0);
    } else {
      val = (i == j) ? 1.0 : 0.0;
    }
    tile[(size_t)r * T + c] = val;
  }
}

// Dense block out[i*ld + j], i < rows_pad, j < cols_pad: k(A_i, B_j) for i < na, j < nb (no noise:
// different point sets), plus diag_add on i == j when same_set, and 0 in the padding.
template <int D>
__global__ void __launch_bounds__(kThreads) assemble_dense_kernel(const double* __restrict__ A, long long na,
                                                                  const double* __restrict__ B, long long nb, int Dr,
                                                                  double neg_half_inv_l2, double v, double diag_add,
                                                                  double* __restrict__ out, long long ld,
                                                                  long long rows_pad, long long cols_pad) {
  const long long i = (long long)blockIdx.y * 8 + threadIdx.x / 32;
  if (i >= rows_pad) return;
  for (long long j = (long long)blockIdx.x * 128 + (threadIdx.x % 32); j < cols_pad && j < (long long)(blockIdx.x + 1) * 128;
       j += 32) {
    double val = 0.0;
    if (i < na && j < nb) {
      const double r2 = sqdist_t<D>(A + i * Dr, B + j * Dr, Dr);
      val = v * exp(r2 * neg_half_inv_l2) + (i == j ? diag_add : 0.0);
    }
    out[(size_t)i * ld + j] = val;
  }
}

// mean[i] = sum_{j<n} k(Xs_i, X_j) alpha_j, the kernel row recomputed on the fly (Eq. 2's last
// step fused with the assembly of K_{Xs,X}). 8 test points per CTA.
template <int D>
__global__ void __launch_bounds__(kThreads) mean_gemv_kernel(const double* __restrict__ Xs, long long m,
                                                             const double* __restrict__ X, long long n, int Dr,
                                                             double neg_half_inv_l2, double v,
                                                             const double* __restrict__ alpha, double* __restrict__ mean) {
  __shared__ double red[8][kThreads / 32];
  const long long i0 = (long long)blockIdx.x * 8;
  double acc[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  for (long long j = threadIdx.x; j < n; j += kThreads) {
    const double aj = __ldg(alpha + j);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (i0 + q < m) {
        const double r2 = sqdist_t<D>(Xs + (i0 + q) * Dr, X + j * Dr, Dr);
        acc[q] = fma(v * exp(r2 * neg_half_inv_l2), aj, acc[q]);
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
    case TASK_UPD:  // (I=p, K=q, J=r)
      return wait_ge(a.cK + tri(p, r), r + 1, st, to, ti) && wait_ge(a.cK + tri(q, r), r + 1, st, to, ti) &&
             wait_ge(a.cK + tri(p, q), r, st, to, ti);
    case TASK_VTRSM:  // (J=p, c=q)
      return wait_ge(a.cV + (size_t)p * a.Mc + q, p, st, to, ti);
    case TASK_VGEMM:  // (I=p, J=q, c=r)
      return wait_ge(a.cV + (size_t)q * a.Mc + r, q + 1, st, to, ti) &&
             wait_ge(a.cV + (size_t)p * a.Mc + r, q, st, to, ti);
    case TASK_WSYRK:  // (a=p, b=q, J=r)
      return wait_ge(a.cV + (size_t)r * a.Mc + p, r + 1, st, to, ti) &&
             wait_ge(a.cV + (size_t)r * a.Mc + q, r + 1, st, to, ti) && wait_ge(a.cS + tri(p, q), r, st, to, ti);
    case TASK_FSOLVE: {  // (J=p)
      for (int ch = 0; ch < a.nch; ++ch)
        if (!wait_ge(a.cF + (size_t)p * a.nch + ch, p, st, to, ti)) return false;
      return true;
    }
    case TASK_FGEMV:  // (I=p, J=q, ch=r)
      return wait_ge(a.dF + q, 1, st, to, ti) && wait_ge(a.cF + (size_t)p * a.nch + r, q, st, to, ti);
    case TASK_BSOLVE: {  // (J=p)
      if (!wait_ge(a.dF + p, 1, st, to, ti)) return false;
      for (int ch = 0; ch < a.nch; ++ch)
        if (!wait_ge(a.cB + (size_t)p * a.nch + ch, a.Mt - 1 - p, st, to, ti)) return false;
      return true;
    }
    case TASK_BGEMV:  // (J=p, I=q, ch=r)
      return wait_ge(a.dB + q, 1, st, to, ti) && wait_ge(a.dF + p, 1, st, to, ti) &&
             wait_ge(a.cB + (size_t)p * a.nch + r, a.Mt - 1 - q, st, to, ti);
  }
  return false;
}

// The persistent kernel: each CTA repeatedly takes the next task in dispatch order, waits (bounded)
// until the counters of the tiles it reads say their producers are done, runs the tile operation,
// and publishes its own tile's counter. kMixed selects FP32 arithmetic for the trailing updates,
// the panel TRSMs after the first block column and the covariance solve; POTRF, the first block
// column's TRSM and the vector solves stay FP64.
template <bool kMixed>
__global__ void __launch_bounds__(kThreads, kMixed ? 1 : 2) dag_kernel(DagArgs a) {
  __shared__ union {
    TileSmem d;
    TileSmemF32 f;
  } u;
  __shared__ int s_task;
  __shared__ double s_red[kThreads / 32][32];
  TileSmem& s = u.d;
  const int T = a.T;
  const size_t TT = (size_t)T * T;
  while (true) {
    if (threadIdx.x == 0) s_task = ld_relaxed(&a.st->abort) ? INT_MAX : (int)atomicAdd(&a.st->next_task, 1ull);
    __syncthreads();
    const int ti = s_task;
    __syncthreads();
    if (ti >= a.ntasks) break;
    const int4 tk = a.tasks[ti];
    bool ok = true;
    if (threadIdx.x == 0) ok = wait_deps(a, tk, ti);
    if (__syncthreads_or(!ok)) break;
    const int p = tk.y, q = tk.z, r = tk.w;
    if (ti == a.withhold_task) continue;  // test hook: this task's completion is never published
    switch (tk.x) {
      case TASK_POTRF: {
        const int fail = cta_potrf(a.Kt + tri(p, p) * TT, T, T, s);
        if (fail) {
          if (threadIdx.x == 0) raise_error(a.st, GP_ERR_NOT_PD, (long long)p * T + fail);
          return;
        }
        cta_publish(a.cK + tri(p, p), p + 1);
        break;
      }
      case TASK_TRSM:
        if (kMixed && q > 0)
          cta_trsm_right_f32(a.Kt + tri(q, q) * TT, T, a.Kt + tri(p, q) * TT, T, T, T, u.f);
        else
          cta_trsm_right(a.Kt + tri(q, q) * TT, T, a.Kt + tri(p, q) * TT, T, T, T, s);
        cta_publish(a.cK + tri(p, q), q + 1);
        break;
      case TASK_UPD:
        if (kMixed)
          cta_gemm_sub_f32<0, 0>(a.Kt + tri(p, q) * TT, T, a.Kt + tri(p, r) * TT, T, a.Kt + tri(q, r) * TT, T, T, T,
                                 T, p == q, u.f.g);
        else
          cta_gemm_sub<A_MK, B_NK>(a.Kt + tri(p, q) * TT, T, a.Kt + tri(p, r) * TT, T, a.Kt + tri(q, r) * TT, T, T,
                                   T, T, p == q, 0, s.g);
        cta_publish(a.cK + tri(p, q), r + 1);
        break;
      case TASK_VTRSM: {
        double* B = a.V + (size_t)p * T * a.ldv + (size_t)q * T;
        if (kMixed)
          cta_trsm_left_f32(a.Kt + tri(p, p) * TT, T, B, (int)a.ldv, T, T, u.f);
        else
          cta_trsm_left(a.Kt + tri(p, p) * TT, T, B, (int)a.ldv, T, T, s);
        cta_publish(a.cV + (size_t)p * a.Mc + q, p + 1);
        break;
      }
      case TASK_VGEMM: {
        double* C = a.V + (size_t)p * T * a.ldv + (size_t)r * T;
        const double* B = a.V + (size_t)q * T * a.ldv + (size_t)r * T;
        if (kMixed)
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
        if (kMixed)
          cta_gemm_sub_f32<1, 1>(C, (int)a.lds, Va, (int)a.ldv, Vb, (int)a.ldv, T, T, T, p == q, u.f.g);
        else
          cta_gemm_sub<A_KM, B_KN>(C, (int)a.lds, Va, (int)a.ldv, Vb, (int)a.ldv, T, T, T, p == q, 0, s.g);
        cta_publish(a.cS + tri(p, q), r + 1);
        break;
      }
      case TASK_FSOLVE:
        cta_trsv_lower(a.Kt + tri(p, p) * TT, T, a.bvec + (size_t)p * T, T, &s_red[0][0], s.tri);
        cta_publish(a.dF + p, 1);
        break;
      case TASK_FGEMV:
        cta_gemv_sub(a.Kt + tri(p, q) * TT + (size_t)r * 32 * T, T, a.bvec + (size_t)q * T,
                     a.bvec + (size_t)p * T + r * 32, 32, T);
        cta_publish(a.cF + (size_t)p * a.nch + r, q + 1);
        break;
      case TASK_BSOLVE:
        cta_trsv_lower_T(a.Kt + tri(p, p) * TT, T, a.bvec + (size_t)p * T, T, &s_red[0][0], s.tri);
        cta_publish(a.dB + p, 1);
        break;
      case TASK_BGEMV:
        cta_gemv_T_sub(a.Kt + tri(q, p) * TT + (size_t)r * 32, T, a.bvec + (size_t)q * T,
                       a.bvec + (size_t)p * T + r * 32, T, 32, s_red);
        cta_publish(a.cB + (size_t)p * a.nch + r, a.Mt - q);
        break;
    }
  }
}

// r = y - K alpha for the 32 rows (tile row I = blockIdx.x / nch, chunk ch) from the packed lower
// FP64 tiles of the symmetric K (diagonal tiles hold both triangles): row part from tiles (I, J<=I),
// transposed part from tiles (J>I, I). Per-block partial sums of r^2 and y^2 go to partial[2b..2b+1].
__global__ void __launch_bounds__(kThreads) residual_kernel(const double* __restrict__ Kt, int T, int Mt,
                                                            long long n, const double* __restrict__ y,
                                                            const double* __restrict__ alpha, double* __restrict__ r,
                                                            double* __restrict__ partial) {
  __shared__ double red[kThreads / 32][32];
  const int nch = T / 32;
  const int I = blockIdx.x / nch, ch = blockIdx.x % nch;
  const int w = threadIdx.x / 32, lane = threadIdx.x % 32;
  const size_t TT = (size_t)T * T;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // rows ch*32 + w*4 + k, lane-partial
  for (int J = 0; J <= I; ++J) {
    const double* tile = Kt + tri(I, J) * TT + (size_t)(ch * 32 + w * 4) * T;
    const double* aJ = alpha + (size_t)J * T;
    for (int c = lane; c < T; c += 32) {
      const double av = aJ[c];
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k] = fma(tile[(size_t)k * T + c], av, acc[k]);
    }
  }
  double accT = 0.0;  // column ch*32 + lane, warp-partial over rows
  for (int J = I + 1; J < Mt; ++J) {
    const double* tile = Kt + tri(J, I) * TT + ch * 32 + lane;
    const double* aJ = alpha + (size_t)J * T;
    for (int rr = w; rr < T; rr += kThreads / 32) accT = fma(tile[(size_t)rr * T], aJ[rr], accT);
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
  }
  red[w][lane] = accT;
  __syncthreads();
  __shared__ double rowsum[32];
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[q][threadIdx.x];
    rowsum[threadIdx.x] = t;
  }
  __syncthreads();
  __shared__ double sq[2][32];
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int row = ch * 32 + w * 4 + k;
      const long long gi = (long long)I * T + row;
      const double tot = acc[k] + rowsum[w * 4 + k];
      const double yi = gi < n ? y[gi] : 0.0;
      const double ri = gi < n ? yi - tot : 0.0;
      r[gi] = ri;
      sq[0][w * 4 + k] = ri * ri;
      sq[1][w * 4 + k] = yi * yi;
    }
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int k = 0; k < 32; ++k) t += sq[threadIdx.x][k];
    partial[2 * blockIdx.x + threadIdx.x] = t;
  }
}

// out[0] = sum of even partials (||r||^2), out[1] = sum of odd partials (||y||^2); one CTA.
__global__ void __launch_bounds__(kThreads) sum_pairs_kernel(const double* __restrict__ partial, int nb,
                                                             double* __restrict__ out) {
  __shared__ double red[2][kThreads / 32];
  double s0 = 0.0, s1 = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) {
    s0 += partial[2 * b];
    s1 += partial[2 * b + 1];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
  }
  if (threadIdx.x % 32 == 0) {
    red[0][threadIdx.x / 32] = s0;
    red[1][threadIdx.x / 32] = s1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += red[threadIdx.x][q];
    out[threadIdx.x] = t;
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

// ---------------------------------------------------------------- host launchers

cudaError_t launch_assemble_tiles(const double* X, long long n, int D, double l, double v, double s2, double* Kt, int T,
                                  int Mt, cudaStream_t st) {
  const long long ntiles = (long long)Mt * (Mt + 1) / 2;
  if (ntiles == 0) return cudaSuccess;
  dim3 grid((unsigned)ntiles, (unsigned)(T / 32));
  const double c = -0.5 / (l * l);
  switch (D) {
    case 4: assemble_tiles_kernel<4><<<grid, kThreads, 0, st>>>(X, n, D, c, v, s2, Kt, T); break;
    case 8: assemble_tiles_kernel<8><<<grid, kThreads, 0, st>>>(X, n, D, c, v, s2, Kt, T); break;
    case 16: assemble_tiles_kernel<16><<<grid, kThreads, 0, st>>>(X, n, D, c, v, s2, Kt, T); break;
    default: assemble_tiles_kernel<0><<<grid, kThreads, 0, st>>>(X, n, D, c, v, s2, Kt, T); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_assemble_dense(const double* A, long long na, const double* B, long long nb, int D, double l,
                                  double v, double diag_add, double* out, long long ld, long long rows_pad,
                                  long long cols_pad, cudaStream_t st) {
  if (rows_pad == 0 || cols_pad == 0) return cudaSuccess;
  dim3 grid((unsigned)((cols_pad + 127) / 128), (unsigned)((rows_pad + 7) / 8));
  const double c = -0.5 / (l * l);
  switch (D) {
    case 4: assemble_dense_kernel<4><<<grid, kThreads, 0, st>>>(A, na, B, nb, D, c, v, diag_add, out, ld, rows_pad, cols_pad); break;
    case 8: assemble_dense_kernel<8><<<grid, kThreads, 0, st>>>(A, na, B, nb, D, c, v, diag_add, out, ld, rows_pad, cols_pad); break;
    case 16: assemble_dense_kernel<16><<<grid, kThreads, 0, st>>>(A, na, B, nb, D, c, v, diag_add, out, ld, rows_pad, cols_pad); break;
    default: assemble_dense_kernel<0><<<grid, kThreads, 0, st>>>(A, na, B, nb, D, c, v, diag_add, out, ld, rows_pad, cols_pad); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_mean_gemv(const double* Xs, long long m, const double* X, long long n, int D, double l, double v,
                             const double* alpha, double* mean, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((m + 7) / 8);
  const double c = -0.5 / (l * l);
  switch (D) {
    case 4: mean_gemv_kernel<4><<<grid, kThreads, 0, st>>>(Xs, m, X, n, D, c, v, alpha, mean); break;
    case 8: mean_gemv_kernel<8><<<grid, kThreads, 0, st>>>(Xs, m, X, n, D, c, v, alpha, mean); break;
    case 16: mean_gemv_kernel<16><<<grid, kThreads, 0, st>>>(Xs, m, X, n, D, c, v, alpha, mean); break;
    default: mean_gemv_kernel<0><<<grid, kThreads, 0, st>>>(Xs, m, X, n, D, c, v, alpha, mean); break;
  }
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

cudaError_t launch_dag(const DagArgs& a, int grid, bool mixed, cudaStream_t st) {
  if (a.ntasks == 0) return cudaSuccess;
  if (mixed)
    dag_kernel<true><<<grid, kThreads, 0, st>>>(a);
  else
    dag_kernel<false><<<grid, kThreads, 0, st>>>(a);
  return cudaGetLastError();
}

int dag_max_ctas_per_sm(bool mixed) {
  int nb = 0;
  if (mixed)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dag_kernel<true>, kThreads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dag_kernel<false>, kThreads, 0);
  return nb;
}

cudaError_t launch_residual(const double* Kt, int T, int Mt, long long n, const double* y, const double* alpha,
                            double* r, double* partial, double* norms, cudaStream_t st) {
  const int nb = Mt * (T / 32);
  residual_kernel<<<nb, kThreads, 0, st>>>(Kt, T, Mt, n, y, alpha, r, partial);
  sum_pairs_kernel<<<1, kThreads, 0, st>>>(partial, nb, norms);
  return cudaGetLastError();
}

cudaError_t launch_axpy(double* alpha, const double* d, long long n, cudaStream_t st) {
  const long long b = (n + kThreads - 1) / kThreads;
  axpy_kernel<<<(unsigned)(b < 4096 ? (b > 0 ? b : 1) : 4096), kThreads, 0, st>>>(alpha, d, n);
  return cudaGetLastError();
}

}  // namespace gpk
