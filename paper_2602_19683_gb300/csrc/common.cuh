// Device-side helpers shared by the GP kernels: status word, bounded waits, memory ordering.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gp.h"

namespace gpk {

constexpr int kThreads = 256;  // every CTA of the library's kernels

// Device status word, one per context. code: first error (0 = none); abort: set by the first
// failing CTA so that every other CTA of the persistent kernel drains; info: error detail
// (smallest failing 1-based column for GP_ERR_NOT_PD; task index for GP_ERR_TIMEOUT).
struct DevStatus {
  int32_t code;
  int32_t abort;
  long long info;
  unsigned long long next_task;  // dispatch counter of the running persistent kernel
  unsigned long long pad[5];
};

// Fixed-point coordinates of the covariance assembly (se_kernel.cuh): the quantisation shared by the
// point sets of one launch family (device resident, written by fx_prepare_kernel).
struct FxScale {
  int32_t F;                // q = round(x 2^F)
  int32_t usable;           // 1: every quantised coordinate |q| < 2^58 and max |x| <= 64 l (the error bound holds)
  unsigned long long smax;  // during the preparation: bit pattern of max |x| (orders like the value)
  int32_t nonfinite;        // during the preparation: 1 if some coordinate is NaN or infinite
  int32_t pad;
};

#ifdef __CUDACC__
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Records the first error and raises the abort flag.
__device__ __forceinline__ void raise_error(DevStatus* st, int code, long long info) {
  const int prev = atomicCAS(&st->code, 0, code);
  if (prev == 0 || prev == code) atomicMin(&st->info, info);  // info is reset to LLONG_MAX
  atomicExch(&st->abort, 1);
}

// Thread-0 spin until *p >= target. Bounded: returns false (and raises GP_ERR_TIMEOUT) when the
// wait exceeds timeout_ns, or false at once when another CTA has aborted.
__device__ __forceinline__ bool wait_ge(const int* p, int target, DevStatus* st, long long timeout_ns,
                                        long long where) {
  if (ld_acquire(p) >= target) return true;
  const uint64_t t0 = globaltimer();
  unsigned ns = 32;
  while (true) {
    if (ld_relaxed(&st->abort)) return false;
    if (ld_acquire(p) >= target) return true;
    if ((long long)(globaltimer() - t0) > timeout_ns) {
      raise_error(st, GP_ERR_TIMEOUT, where);
      return false;
    }
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
}

// Publishes a CTA's global-memory results: every thread's stores are complete and visible at GPU
// scope before thread 0 releases the counter.
__device__ __forceinline__ void cta_publish(int* counter, int value) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(counter, value);
  }
}

// Publishes a CTA's results by adding 1 to a counter that several CTAs complete together (the
// fence before the add makes every thread's stores visible first, as in cta_publish).
__device__ __forceinline__ void cta_publish_add(int* counter) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1);
  }
}

// FP64 <-> FP32 conversions on the integer pipe. On GB300 the cvt instructions between double and
// float issue on the FP64 pipe (about 2 per clock per SM, like an FP64 FMA), so staging FP64 operands
// as FP32 with cvt would cost as much FP64 issue as the FP32 FMAs they feed. These do the same
// IEEE conversion with 32-bit integer operations on the two halves of the double:
//   narrowing: round to nearest, ties to even; results below the FP32 normal range flush to a
//              signed zero, values beyond it become a signed infinity, NaN stays NaN;
//   widening:  exact (FP32 subnormals flush to a signed zero).
__device__ __forceinline__ float f64_to_f32_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);  // top 23 mantissa bits
  const unsigned rem = lo & 0x1FFFFFFFu;                   // the 29 bits rounded away
  if (e == 0x7FF) return __uint_as_float(sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u));
  const int e32 = e - 896;  // rebias 1023 -> 127
  if (e32 <= 0) return __uint_as_float(sign);
  if (e32 >= 255) return __uint_as_float(sign | 0x7F800000u);
  const unsigned inc = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
  return __uint_as_float((sign | ((unsigned)e32 << 23) | m) + inc);  // a mantissa carry bumps the exponent
}

__device__ __forceinline__ double f32_to_f64(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  if (e == 0) return __hiloint2double((int)sign, 0);
  const unsigned hi = (e == 0xFFu) ? (sign | 0x7FF00000u | (m >> 3)) : (sign | ((e + 896u) << 20) | (m >> 3));
  return __hiloint2double((int)hi, (int)(m << 29));
}

// L2-only load (bypasses L1, so data written by other SMs after an acquire is never stale).
template <class T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

#endif  // __CUDACC__

}  // namespace gpk
