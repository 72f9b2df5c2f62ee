// Vendor baselines and pipe-throughput probes on the same GPU (never on libgp's product path):
//   cuSOLVER Dpotrf / Spotrf on an n x n SPD matrix (the single-call factorisation the paper's
//   tiled approach is compared with in Sec. 4.1), cuBLAS DGEMM, and register-only FP64 FFMA,
//   FP64 mma.sync (DMMA) and FP32 FFMA loops that bound what FMA-issue-bound kernels can reach, and
//   streaming probes (a read-only 4 GB buffer consumed by FP64 or by FP32 adds, through plain loads or
//   through a ring of bulk copies) that show whether a matrix-vector-type pass is bound by HBM or by
//   the FP64 pipe.
// Prints one JSON object per measurement.
// Usage: vendor_baselines [n] [--no-potrf] [--no-spotrf] [--no-probes] [--once]
//   --once: time the first Dpotrf call (no warm-up call; for sizes where one call takes a minute).
// Above n = 46340 (n^2 > 2^31 entries) Dpotrf goes through the 64-bit generic API (cusolverDnXpotrf).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>
#include <cublas_v2.h>
#include <cusolverDn.h>

#define CK(x)                                                                   \
  do {                                                                          \
    cudaError_t e = (x);                                                        \
    if (e != cudaSuccess) {                                                     \
      printf("{\"error\": \"%s\", \"line\": %d}\n", cudaGetErrorString(e), __LINE__); \
      exit(1);                                                                  \
    }                                                                           \
  } while (0)

__global__ void ffma64_loop(double* out, int iters, double a, double b) {
  double x[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = threadIdx.x + j;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = fma(x[j], a, b);
  double s = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void ffma32_loop(float* out, int iters, float a, float b) {
  float x[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) x[j] = threadIdx.x + j;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int j = 0; j < 16; ++j) x[j] = fmaf(x[j], a, b);
  float s = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) s += x[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dmma_loop(double* out, int iters) {
  double a = 1.0 + threadIdx.x * 1e-3, b = 1.0 - threadIdx.x * 1e-3;
  double c[8][2];
  for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = 0;
  for (int i = 0; i < iters; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j)
      asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                   : "+d"(c[j][0]), "+d"(c[j][1])
                   : "d"(a), "d"(b));
  double s = 0;
  for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// FP64 FFMA in the warps of one half of each CTA and FP64 mma.sync in the other, at the same time:
// whether the two issue to separate FP64 units (their rates would add) or share one.
__global__ void mixed_fp64_loop(double* out, int iters_ffma, int iters_dmma, double a, double b) {
  const int w = threadIdx.x >> 5;
  double s = 0;
  if (w & 1) {
    double x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = threadIdx.x + j;
    for (int i = 0; i < iters_ffma; ++i)
#pragma unroll
      for (int j = 0; j < 16; ++j) x[j] = fma(x[j], a, b);
#pragma unroll
    for (int j = 0; j < 16; ++j) s += x[j];
  } else {
    double c[8][2];
    for (int j = 0; j < 8; ++j) c[j][0] = c[j][1] = 0;
    for (int i = 0; i < iters_dmma; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
                     : "+d"(c[j][0]), "+d"(c[j][1])
                     : "d"(a), "d"(b));
    for (int j = 0; j < 8; ++j) s += c[j][0] + c[j][1];
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// A = exp(-((i-j)/64)^2) + 0.1 I: symmetric positive definite.
__global__ void fill_spd(double* A, long long n) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n * n; e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / n, j = e % n;
    const double d = (double)(i - j) / 64.0;
    A[e] = exp(-d * d) + (i == j ? 0.1 : 0.0);
  }
}
__global__ void to_float(const double* A, float* B, long long cnt) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt; e += (long long)gridDim.x * blockDim.x)
    B[e] = (float)A[e];
}

// Streaming probes. Each CTA reads its own contiguous slice (bytes_per_cta) once.
// FP64 consumer: one FP64 add per 8 bytes (the issue cost of a dense FP64 matrix-vector product).
__global__ void __launch_bounds__(512) stream_fp64(const double2* src, long long n2_per_cta, double* sink) {
  const double2* base = src + (long long)blockIdx.x * n2_per_cta;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n2_per_cta; i += 512 * 8) {
    double2 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (i + u * 512 < n2_per_cta) ? __ldg(base + i + u * 512) : make_double2(0, 0);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += v[u].x + v[u].y;
  }
  if (acc == 1234.5) sink[0] = acc;
}
// FP32 consumer: one FP32 add per 4 bytes.
__global__ void __launch_bounds__(512) stream_fp32(const float4* src, long long n4_per_cta, double* sink) {
  const float4* base = src + (long long)blockIdx.x * n4_per_cta;
  float acc = 0.f;
  for (long long i = threadIdx.x; i < n4_per_cta; i += 512 * 8) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = (i + u * 512 < n4_per_cta) ? __ldg(base + i + u * 512) : make_float4(0, 0, 0, 0);
#pragma unroll
    for (int u = 0; u < 8; ++u) acc += (v[u].x + v[u].y) + (v[u].z + v[u].w);
  }
  if (acc == 1234.5f) sink[0] = acc;
}
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool mbar_done(unsigned long long* b, unsigned par) {
  unsigned ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(smem_addr(b)), "r"(par) : "memory");
  return ok;
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bulk-copy ring: 64 KB chunks, 3 stages, thread 0 issues; FP32 consumer. Every wait is bounded (50 ms,
// then *err is set and the CTA drains its copies and leaves).
__global__ void __launch_bounds__(512, 1) stream_bulk_fp32(const unsigned char* src, long long bytes_per_cta,
                                                           double* sink, int* err) {
  constexpr int CB = 65536, S = 3;
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ unsigned long long full[S];
  __shared__ int fail;
  const unsigned char* base = src + (long long)blockIdx.x * bytes_per_cta;
  const long long nchunks = bytes_per_cta / CB;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&full[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fail = 0;
  }
  __syncthreads();
  long long issued = 0;
  auto issue = [&]() {
    if (issued >= nchunks) return;
    const int s = issued % S;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(&full[s])), "r"(CB) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(sm + (long long)s * CB)), "l"(base + issued * CB), "r"(CB), "r"(smem_addr(&full[s]))
                 : "memory");
    ++issued;
  };
  if (threadIdx.x == 0)
    for (int q = 0; q < S; ++q) issue();
  float acc = 0.f;
  long long i = 0;
  for (; i < nchunks; ++i) {
    const int s = i % S;
    const unsigned long long t0 = gtimer();
    while (!mbar_done(&full[s], (unsigned)(i / S) & 1u))
      if (gtimer() - t0 > 50000000ull) { fail = 1; atomicExch(err, 1); break; }
    const float4* d = reinterpret_cast<const float4*>(sm + (long long)s * CB);
    for (int e = threadIdx.x; e < CB / 16; e += 512) { const float4 v = d[e]; acc += (v.x + v.y) + (v.z + v.w); }
    __syncthreads();
    if (fail) break;
    if (threadIdx.x == 0) issue();
  }
  if (fail && threadIdx.x == 0)
    for (long long q = i; q < issued; ++q) {
      const unsigned long long t0 = gtimer();
      while (!mbar_done(&full[q % S], (unsigned)(q / S) & 1u) && gtimer() - t0 < 50000000ull) {}
    }
  if (acc == 1234.5f) sink[0] = acc;
}

template <class F>
float best_ms(F f, int reps) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  f();
  CK(cudaDeviceSynchronize());
  float best = 1e30f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0);
    f();
    cudaEventRecord(e1);
    CK(cudaEventSynchronize(e1));
    float ms;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  return best;
}

int main(int argc, char** argv) {
  long long n = 32768;
  bool potrf = true, spotrf = true, probes = true, once = false;
  for (int i = 1; i < argc; ++i) {
    if (!strcmp(argv[i], "--no-potrf")) potrf = false;
    else if (!strcmp(argv[i], "--no-spotrf")) spotrf = false;
    else if (!strcmp(argv[i], "--no-probes")) probes = false;
    else if (!strcmp(argv[i], "--once")) once = true;
    else n = atoll(argv[i]);
  }
  const bool big = n * n > 2147483647LL;
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, 0));
  const int sms = p.multiProcessorCount;
  double* out;
  CK(cudaMalloc(&out, sizeof(double) * sms * 2048));
  if (probes) {
    const int grid = sms * 8, iters = 4000;
    float ms = best_ms([&] { ffma64_loop<<<grid, 256>>>(out, iters, 0.999, 1e-3); }, 3);
    printf("{\"probe\": \"ffma64\", \"tflops\": %.4f}\n", 2.0 * 16 * iters * (double)grid * 256 / ms / 1e9);
  }
  if (probes) {
    const int grid = sms * 8, iters = 2000;
    float ms = best_ms([&] { ffma32_loop<<<grid, 256>>>((float*)out, iters, 0.999f, 1e-3f); }, 3);
    printf("{\"probe\": \"ffma32\", \"tflops\": %.4f}\n", 2.0 * 128 * iters * (double)grid * 256 / ms / 1e9);
  }
  if (probes) {
    const int grid = sms * 4, iters = 400;
    float ms = best_ms([&] { dmma_loop<<<grid, 256>>>(out, iters); }, 3);
    printf("{\"probe\": \"dmma_m8n8k4\", \"tflops\": %.4f}\n", 2.0 * 256 * 8 * iters * (double)grid * 8 / ms / 1e9);
  }
  if (probes) {  // FFMA and DMMA issued together (half the warps each); flops of both counted
    const int grid = sms * 4, it_f = 2000, it_d = 200;
    float ms = best_ms([&] { mixed_fp64_loop<<<grid, 256>>>(out, it_f, it_d, 0.999, 1e-3); }, 3);
    const double ffma = 2.0 * 16 * it_f * (double)grid * 128, dmma = 2.0 * 256 * 8 * it_d * (double)grid * 4;
    printf("{\"probe\": \"ffma64_and_dmma\", \"tflops\": %.4f, \"ffma_share\": %.3f}\n", (ffma + dmma) / ms / 1e9,
           ffma / (ffma + dmma));
  }
  if (probes) {  // streaming: whole GPU (one 512-thread CTA per SM, 4 GB) and one CTA (256 MB)
    const long long total = 4LL << 30;
    unsigned char* buf;
    int* err;
    CK(cudaMalloc(&buf, total));
    CK(cudaMemset(buf, 0, total));
    CK(cudaMalloc(&err, sizeof(int)));
    CK(cudaMemset(err, 0, sizeof(int)));
    CK(cudaFuncSetAttribute(stream_bulk_fp32, cudaFuncAttributeMaxDynamicSharedMemorySize, 3 * 65536));
    for (int grid : {sms, 1}) {
      const long long per = (grid == 1 ? (256LL << 20) : total / grid) / 65536 * 65536;
      const double gb = (double)per * grid / 1e9;
      const float m64 = best_ms([&] { stream_fp64<<<grid, 512>>>((const double2*)buf, per / 16, out); }, 3);
      const float m32 = best_ms([&] { stream_fp32<<<grid, 512>>>((const float4*)buf, per / 16, out); }, 3);
      const float mb = best_ms([&] { stream_bulk_fp32<<<grid, 512, 3 * 65536>>>(buf, per, out, err); }, 3);
      int herr = 0;
      CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
      printf("{\"probe\": \"stream_%s\", \"ctas\": %d, \"fp64_consumer_gbs\": %.1f, \"fp32_consumer_gbs\": %.1f, "
             "\"bulk64k_fp32_consumer_gbs\": %.1f, \"timeouts\": %d}\n",
             grid == 1 ? "one_cta" : "gpu", grid, gb / m64 * 1e3, gb / m32 * 1e3, gb / mb * 1e3, herr);
    }
    cudaFree(buf);
    cudaFree(err);
  }
  fflush(stdout);
  double* A;
  CK(cudaMalloc(&A, sizeof(double) * n * n));
  cublasHandle_t bh;
  cublasCreate(&bh);
  if (probes) {
    const int N = 8192;
    double *B, *C;
    CK(cudaMalloc(&B, sizeof(double) * N * N));
    CK(cudaMalloc(&C, sizeof(double) * N * N));
    fill_spd<<<4096, 256>>>(B, N);
    const double one = 1, zero = 0;
    float ms = best_ms([&] { cublasDgemm(bh, CUBLAS_OP_N, CUBLAS_OP_T, N, N, N, &one, B, N, B, N, &zero, C, N); }, 2);
    printf("{\"probe\": \"cublas_dgemm\", \"n\": %d, \"tflops\": %.4f}\n", N, 2.0 * N * N * (double)N / ms / 1e9);
    cudaFree(B);
    cudaFree(C);
    // the tensor-core kinds an FP64 emulation could build on: INT8 (int32 accumulation) and BF16 (FP32
    // accumulation) GEMMs of the same size, operands zero-filled (the rate, not the values, is measured)
    void *A8, *C32;
    CK(cudaMalloc(&A8, (size_t)N * N * 2));
    CK(cudaMalloc(&C32, (size_t)N * N * 4));
    CK(cudaMemset(A8, 0, (size_t)N * N * 2));
    const int32_t ione = 1, izero = 0;
    const float fone = 1.f, fzero = 0.f;
    cublasStatus_t s8 = CUBLAS_STATUS_SUCCESS;
    float ms8 = best_ms([&] {
      s8 = cublasGemmEx(bh, CUBLAS_OP_T, CUBLAS_OP_N, N, N, N, &ione, A8, CUDA_R_8I, N, A8, CUDA_R_8I, N, &izero, C32,
                        CUDA_R_32I, N, CUBLAS_COMPUTE_32I, CUBLAS_GEMM_DEFAULT);
    }, 2);
    if (s8 == CUBLAS_STATUS_SUCCESS)
      printf("{\"probe\": \"cublas_igemm_int8\", \"n\": %d, \"tops\": %.1f}\n", N, 2.0 * N * N * (double)N / ms8 / 1e9);
    else
      printf("{\"probe\": \"cublas_igemm_int8\", \"n\": %d, \"status\": %d}\n", N, (int)s8);
    cublasStatus_t sb = CUBLAS_STATUS_SUCCESS;
    float msb = best_ms([&] {
      sb = cublasGemmEx(bh, CUBLAS_OP_T, CUBLAS_OP_N, N, N, N, &fone, A8, CUDA_R_16BF, N, A8, CUDA_R_16BF, N, &fzero,
                        C32, CUDA_R_32F, N, CUBLAS_COMPUTE_32F, CUBLAS_GEMM_DEFAULT);
    }, 2);
    if (sb == CUBLAS_STATUS_SUCCESS)
      printf("{\"probe\": \"cublas_bf16gemm\", \"n\": %d, \"tflops\": %.1f}\n", N, 2.0 * N * N * (double)N / msb / 1e9);
    cudaFree(A8);
    cudaFree(C32);
  }
  fflush(stdout);
  if (potrf) {
    cusolverDnHandle_t sh;
    cusolverDnCreate(&sh);
    int* info;
    CK(cudaMalloc(&info, sizeof(int)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    if (!big) {
      int lw = 0;
      cusolverDnDpotrf_bufferSize(sh, CUBLAS_FILL_MODE_LOWER, (int)n, A, (int)n, &lw);
      double* W;
      CK(cudaMalloc(&W, sizeof(double) * (lw + 1)));
      for (int r = once ? 1 : 0; r < 2; ++r) {  // r = 0 warms up
        fill_spd<<<4096, 256>>>(A, n);
        CK(cudaDeviceSynchronize());
        cudaEventRecord(e0);
        cusolverDnDpotrf(sh, CUBLAS_FILL_MODE_LOWER, (int)n, A, (int)n, W, lw, info);
        cudaEventRecord(e1);
        CK(cudaEventSynchronize(e1));
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = ms;
      }
      cudaFree(W);
    } else {
      cusolverDnParams_t prm;
      cusolverDnCreateParams(&prm);
      size_t wd = 0, wh = 0;
      cusolverDnXpotrf_bufferSize(sh, prm, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A, n, CUDA_R_64F, &wd, &wh);
      void* Wd = nullptr;
      CK(cudaMalloc(&Wd, wd + 16));
      void* Wh = malloc(wh + 16);
      for (int r = once ? 1 : 0; r < 2; ++r) {
        fill_spd<<<4096, 256>>>(A, n);
        CK(cudaDeviceSynchronize());
        cudaEventRecord(e0);
        cusolverDnXpotrf(sh, prm, CUBLAS_FILL_MODE_LOWER, n, CUDA_R_64F, A, n, CUDA_R_64F, Wd, wd, Wh, wh, info);
        cudaEventRecord(e1);
        CK(cudaEventSynchronize(e1));
        float ms;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0) best = ms;
      }
      cudaFree(Wd);
      free(Wh);
      cusolverDnDestroyParams(prm);
    }
    int hinfo = -1;
    cudaMemcpy(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost);
    printf("{\"probe\": \"cusolver_dpotrf\", \"n\": %lld, \"ms\": %.3f, \"tflops\": %.4f, \"info\": %d, \"api\": \"%s\"}\n",
           n, best, (double)n * n * (double)n / 3.0 / best / 1e9, hinfo, big ? "Xpotrf" : "Dpotrf");
    fflush(stdout);
  }
  if (potrf && spotrf && !big) {
    cusolverDnHandle_t sh;
    cusolverDnCreate(&sh);
    int* info;
    CK(cudaMalloc(&info, sizeof(int)));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    float* Af;
    CK(cudaMalloc(&Af, sizeof(float) * n * n));
    int lwf = 0;
    cusolverDnSpotrf_bufferSize(sh, CUBLAS_FILL_MODE_LOWER, (int)n, Af, (int)n, &lwf);
    float* Wf;
    CK(cudaMalloc(&Wf, sizeof(float) * (lwf + 1)));
    for (int r = 0; r < 2; ++r) {
      fill_spd<<<4096, 256>>>(A, n);
      to_float<<<4096, 256>>>(A, Af, n * n);
      CK(cudaDeviceSynchronize());
      cudaEventRecord(e0);
      cusolverDnSpotrf(sh, CUBLAS_FILL_MODE_LOWER, (int)n, Af, (int)n, Wf, lwf, info);
      cudaEventRecord(e1);
      CK(cudaEventSynchronize(e1));
      float ms;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) best = ms;
    }
    printf("{\"probe\": \"cusolver_spotrf\", \"n\": %lld, \"ms\": %.3f, \"tflops\": %.4f}\n", n, best,
           (double)n * n * (double)n / 3.0 / best / 1e9);
  }
  return 0;
}
