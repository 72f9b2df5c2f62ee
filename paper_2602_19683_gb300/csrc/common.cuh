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

// L2-only load (bypasses L1, so data written by other SMs after an acquire is never stale).
template <class T>
__device__ __forceinline__ T ldcg(const T* p) {
  return __ldcg(p);
}

#endif  // __CUDACC__

}  // namespace gpk
