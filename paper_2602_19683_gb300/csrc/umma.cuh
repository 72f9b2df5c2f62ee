// Tensor-core (tcgen05) primitives of the mixed-precision mode and its FP32-in-TMEM epilogue:
// TMEM allocation, shared-memory matrix and instruction descriptors (mbarriers and bulk copies: bulk.cuh),
// the kind::tf32 MMA and its commit, and tcgen05.ld of the accumulator.
//
// The mixed trailing updates form C (FP64) -= A B^T from three TF32 split products (3xTF32:
// a_hi b_hi + a_hi b_lo + a_lo b_hi, a = a_hi + a_lo with a_hi the TF32 rounding of the FP32 value and
// a_lo the TF32-rounded remainder), accumulated in FP32 in tensor memory. Their main path is the
// packed-operand pipeline of umma_packed.cuh: every panel tile is split once into the exact
// shared-memory image the MMA reads, and the products are fed by bulk copies through three 64 KB
// stages, one thread issuing the MMAs of each landed 32-wide k chunk. The epilogue (umma_epilogue
// below) reads TMEM with tcgen05.ld (warp w: lanes 32(w%4).., a 64-column half), stages the
// accumulator in shared memory and read-modify-writes the FP64 C tile with coalesced double2 accesses.
//
// umma_block_sub / umma_gemm_sub below are the register-staged form of the same product (operands
// loaded from FP64 and split by all threads, two stages): the path of tiles whose packed operands
// do not exist (tile edges that are multiples of 128 but run without the packed buffers).
//
// Every mbarrier wait is bounded by the task's time limit; a wait that gives up reports
// GP_ERR_TIMEOUT and the caller returns after freeing its TMEM.
#pragma once
#include "bulk.cuh"
#include "tiles_f32.cuh"

namespace gpk {

constexpr int kUmmaM = 128, kUmmaN = 128, kUmmaKChunk = 32;
constexpr int kUmmaTileBytes = kUmmaM * 128;           // 128 rows x 32 tf32
constexpr int kUmmaStageBytes = 4 * kUmmaTileBytes;    // A_hi, A_lo, B_hi, B_lo
constexpr int kPkStages = 3;                           // stages of the packed-operand pipeline
// Dynamic shared memory of the mixed kernel: the operand stages, also the home of a 128 x 129 FP64
// diagonal tile during a shared-memory POTRF (and of two 128 x 129 FP32 tiles while its inverse is
// formed), and of the FP64/FP32 tile routines' scratch; plus alignment slack.
constexpr int kMixedTileSmemBytes = 128 * 129 * 8;
// The BF16-slice products (bslice.cuh) take 210 KB of stages; 1 KB of alignment slack on top.
constexpr int kUmmaSmemBytes = 210 * 1024 + 1024;
static_assert(kUmmaSmemBytes >= kPkStages * kUmmaStageBytes + 1024 && kUmmaSmemBytes >= kMixedTileSmemBytes + 4096,
              "the dynamic smem holds the TF32 stages and the shared-memory POTRF tile");
// four 128 x 128 FP32 accumulators: two per output tile, for the paired-row updates (umma_packed.cuh);
// the whole tensor memory of the SM, which holds one CTA of the mixed kernel (shared memory bound)
constexpr int kUmmaTmemCols = 512;

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols));
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void umma_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void umma_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t umma_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor: kind::tf32, FP32 accumulator, A and B TF32, both K-major, M = N = 128.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kUmmaN >> 3) << 17) |
                                ((uint32_t)(kUmmaM >> 4) << 24);

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdescTf32), "r"(accumulate));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Per-CTA state of the tensor-core path (lives in the persistent kernel for its whole run).
struct UmmaState {
  uint8_t* smem;       // 1024-aligned dynamic shared memory: 2 register-staged or kPkStages packed stages
  uint64_t* bar;       // 2 mbarriers (smem)
  uint32_t tmem;       // TMEM base address (kUmmaTmemCols columns: four 128-column accumulators)
  uint32_t phase[2];   // next parity to wait for, per stage
  uint32_t pending[2]; // stage has an uncompleted commit
  // packed-operand pipeline (umma_packed.cuh): per stage, a "full" barrier completed by the bulk
  // copies' transaction bytes and an "empty" barrier completed by the MMA commit
  uint64_t* pfull;
  uint64_t* pempty;
  uint32_t fph[kPkStages], eph[kPkStages];      // next parity to wait for
  uint32_t fpend[kPkStages], epend[kPkStages];  // a copy / a commit is outstanding on the stage
};

// Waits (thread 0, bounded) until the MMAs committed to stage s have completed; the outcome is made
// uniform across the CTA. On a time-out thread 0 waits once more (same bound) for the MMAs still in
// flight, so that the caller can free TMEM, and the CTA returns false.
__device__ __forceinline__ bool umma_stage_wait(UmmaState& u, int s, DevStatus* st, long long timeout_ns,
                                                long long where) {
  bool ok = true;
  if (threadIdx.x == 0) {
    ok = mbar_wait(&u.bar[s], u.phase[s], st, timeout_ns, where);
    if (!ok) {
      const uint64_t t0 = globaltimer();
      while (!mbar_try_wait(&u.bar[s], u.phase[s]) && (long long)(globaltimer() - t0) < timeout_ns) {
      }
    }
  }
  if (__syncthreads_or(!ok)) return false;
  u.phase[s] ^= 1u;
  u.pending[s] = 0;
  return true;
}

// Byte offset of element (r, k) (k < 32) in a 128-row K-major tile with 128-byte swizzle.
__device__ __forceinline__ uint32_t sw128_offset(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7))) << 4) + (k & 3) * 4);
}

// TF32 rounding (to nearest) of an FP32 value, on the integer pipe.
__device__ __forceinline__ float tf32_rn(float f) { return __uint_as_float((__float_as_uint(f) + 0x1000u) & 0xFFFFE000u); }

// Staging of rows [r0, r0+128) x k [k0, k0+32) of an FP64 row-major operand: coalesced loads (16 lanes
// cover a row's 32 values, 256 B, with one double2 each; a warp reads two whole row segments per pass)
// into registers, then a split of each value into a TF32 high part and a TF32-rounded remainder,
// stored 128-byte-swizzled. The two halves are separate so that the next chunk's loads can be in
// flight while the current chunk is converted and multiplied.
struct UmmaChunkRegs {
  double2 a[8], b[8];
};

__device__ __forceinline__ void umma_load_operand(double2 (&d)[8], const double* P, int ld, int r0, int k0) {
  const int t = threadIdx.x;
  const int kp = t & 15, rr = t >> 4;
#pragma unroll
  for (int pass = 0; pass < 8; ++pass)
    d[pass] = __ldcg(reinterpret_cast<const double2*>(P + (size_t)(r0 + rr + 16 * pass) * ld + k0) + kp);
}

__device__ __forceinline__ void umma_store_operand(uint8_t* hi_tile, uint8_t* lo_tile, const double2 (&d)[8]) {
  const int t = threadIdx.x;
  const int kp = t & 15, rr = t >> 4;
#pragma unroll
  for (int pass = 0; pass < 8; ++pass) {
    const float f0 = f64_to_f32_rn(d[pass].x), f1 = f64_to_f32_rn(d[pass].y);
    const float h0 = tf32_rn(f0), h1 = tf32_rn(f1);
    const uint32_t off = sw128_offset(rr + 16 * pass, 2 * kp);
    *reinterpret_cast<float2*>(hi_tile + off) = make_float2(h0, h1);
    *reinterpret_cast<float2*>(lo_tile + off) = make_float2(tf32_rn(f0 - h0), tf32_rn(f1 - h1));
  }
}

// C[128 x 128 block at (m0, n0)] (FP64, ldc) -= A[m0.., 0..K) B[n0.., 0..K)^T, A and B FP64 row-major
// K-contiguous (K a multiple of 32). lower: write only entries with n <= m (diagonal blocks).
// Returns false on a time-out (error already raised).
// Up to kUmmaMaxPairs (A, B) operand pairs whose products are summed: C -= sum_p A_p B_p^T (K each).
constexpr int kUmmaMaxPairs = 8;
struct UmmaPairs {
  const double* A[kUmmaMaxPairs];
  const double* B[kUmmaMaxPairs];
  int n;
};

__device__ void umma_epilogue_sub(UmmaState& u, double* C, int ldc, int m0, int n0, bool lower);

__device__ bool umma_block_sub(UmmaState& u, double* C, int ldc, const UmmaPairs& pr, int lda, int ldb, int m0,
                               int n0, int K, bool lower, DevStatus* st, long long timeout_ns, long long where) {
  const int nkp = K / kUmmaKChunk, nk = nkp * pr.n;
  UmmaChunkRegs rg;
  umma_load_operand(rg.a, pr.A[0], lda, m0, 0);
  umma_load_operand(rg.b, pr.B[0], ldb, n0, 0);
  for (int kc = 0; kc < nk; ++kc) {
    const int s = kc & 1;
    uint8_t* base = u.smem + s * kUmmaStageBytes;
    if (u.pending[s]) {  // the MMAs that read this stage two chunks ago must be done
      if (!umma_stage_wait(u, s, st, timeout_ns, where)) return false;
    }
    umma_store_operand(base, base + kUmmaTileBytes, rg.a);
    umma_store_operand(base + 2 * kUmmaTileBytes, base + 3 * kUmmaTileBytes, rg.b);
    if (kc + 1 < nk) {  // next chunk's loads fly during the barrier, the MMA issue and the next wait
      const int pi = (kc + 1) / nkp, kk = ((kc + 1) % nkp) * kUmmaKChunk;
      umma_load_operand(rg.a, pr.A[pi], lda, m0, kk);
      umma_load_operand(rg.b, pr.B[pi], ldb, n0, kk);
    }
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      umma_fence_after();
      const uint32_t a_hi = smem_u32(base), a_lo = a_hi + kUmmaTileBytes;
      const uint32_t b_hi = a_hi + 2 * kUmmaTileBytes, b_lo = a_hi + 3 * kUmmaTileBytes;
#pragma unroll
      for (int ks = 0; ks < kUmmaKChunk / 8; ++ks) {
        const uint32_t o = ks * 32;  // 8 tf32 = 32 bytes along K inside the swizzled row
        const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
        umma_tf32(u.tmem, umma_desc_sw128(a_hi + o), umma_desc_sw128(b_hi + o), acc0);
        umma_tf32(u.tmem, umma_desc_sw128(a_hi + o), umma_desc_sw128(b_lo + o), 1u);
        umma_tf32(u.tmem, umma_desc_sw128(a_lo + o), umma_desc_sw128(b_hi + o), 1u);
      }
      umma_commit(&u.bar[s]);
    }
    u.pending[s] = 1;
  }
  // wait for every outstanding stage (the last commit covers all earlier MMAs)
  for (int s = 0; s < 2; ++s)
    if (u.pending[s]) {
      if (!umma_stage_wait(u, s, st, timeout_ns, where)) return false;
    }
  umma_epilogue_sub(u, C, ldc, m0, n0, lower);
  return true;
}

// Epilogue of a 128 x 128 block whose MMAs are all complete: TMEM -> registers (warp w: lanes
// 32(w%4).., a 64-column half) -> smem (row-major, the operand stages are free now) -> coalesced
// FP64 read-modify-write of C (a warp per row, 4 columns per lane): C -= acc, only n <= m when lower.
// The accumulator starts at TMEM column acc_col (a second one, nacc = 2, at acc_col + 128).
// Ends with __syncthreads().
template <bool kStore>
__device__ void umma_epilogue(UmmaState& u, double* C, int ldc, int m0, int n0, bool lower, int nacc = 1,
                              uint32_t acc_col = 0) {
  umma_fence_after();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* acc_s = reinterpret_cast<float*>(u.smem);  // 128 x (128 + 4) floats
  constexpr int ldacc = kUmmaN + 4;
  constexpr int kRows = kUmmaM / (kThreads / 32);    // rows per warp: w, w + 8, ...
  constexpr int kBatch = 8;                          // rows whose C loads are in flight together
  const int n = n0 + 4 * lane;
  double2 c[kBatch][2];
  auto load_batch = [&](int b) {
    if (kStore) return;
#pragma unroll
    for (int i = 0; i < kBatch; ++i) {
      const double2* c2 = reinterpret_cast<const double2*>(C + (size_t)(m0 + w + 8 * (b * kBatch + i)) * ldc + n);
      c[i][0] = __ldcg(c2);
      c[i][1] = __ldcg(c2 + 1);
    }
  };
  load_batch(0);  // the first rows of C fly while the accumulator is staged
  {
    const int row = (w & 3) * 32 + lane, colh = (w >> 2) * 64;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      float v[32];
      tmem_ld32(u.tmem + ((uint32_t)((w & 3) * 32) << 16) + acc_col + (uint32_t)(colh + 32 * half), v);
      if (nacc > 1) {  // second accumulator (the next 128 columns): one FP32 round-to-nearest add
        float v2[32];
        tmem_ld32(u.tmem + ((uint32_t)((w & 3) * 32) << 16) + acc_col + (uint32_t)(kUmmaN + colh + 32 * half), v2);
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] += v2[j];
      }
      float* dst = acc_s + row * ldacc + colh + 32 * half;
#pragma unroll
      for (int j = 0; j < 32; j += 4) *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    }
  }
  umma_fence_before();
  __syncthreads();
  for (int b = 0; b < kRows / kBatch; ++b) {
    if (b > 0) load_batch(b);
#pragma unroll
    for (int i = 0; i < kBatch; ++i) {
      const int r = w + 8 * (b * kBatch + i), m = m0 + r;
      const float4 a = *reinterpret_cast<const float4*>(acc_s + r * ldacc + 4 * lane);
      double2* c2 = reinterpret_cast<double2*>(C + (size_t)m * ldc + n);
      double2 c01, c23;
      if (kStore) {  // C = acc (every entry)
        c01 = make_double2(f32_to_f64(a.x), f32_to_f64(a.y));
        c23 = make_double2(f32_to_f64(a.z), f32_to_f64(a.w));
      } else {
        c01 = c[i][0];
        c23 = c[i][1];
        if (!lower || n + 3 <= m) {
          c01.x -= f32_to_f64(a.x);
          c01.y -= f32_to_f64(a.y);
          c23.x -= f32_to_f64(a.z);
          c23.y -= f32_to_f64(a.w);
        } else {
          if (n <= m) c01.x -= f32_to_f64(a.x);
          if (n + 1 <= m) c01.y -= f32_to_f64(a.y);
          if (n + 2 <= m) c23.x -= f32_to_f64(a.z);
          if (n + 3 <= m) c23.y -= f32_to_f64(a.w);
        }
      }
      c2[0] = c01;
      c2[1] = c23;
    }
  }
  __syncthreads();  // smem and TMEM are reused by the next block
}

__device__ void umma_epilogue_sub(UmmaState& u, double* C, int ldc, int m0, int n0, bool lower) {
  umma_epilogue<false>(u, C, ldc, m0, n0, lower);
}

// C[M x N] -= sum_p A_p B_p^T on the tensor cores for M, N multiples of 128 and K a multiple of 32;
// lower skips blocks above the diagonal and masks the diagonal blocks. Returns false on a time-out.
__device__ bool umma_gemm_sub(UmmaState& u, double* C, int ldc, const UmmaPairs& pr, int lda, int ldb, int M, int N,
                              int K, bool lower, DevStatus* st, long long timeout_ns, long long where) {
  for (int m0 = 0; m0 < M; m0 += kUmmaM)
    for (int n0 = 0; n0 < N; n0 += kUmmaN) {
      if (lower && n0 > m0) continue;
      if (!umma_block_sub(u, C, ldc, pr, lda, ldb, m0, n0, K, lower && n0 == m0, st, timeout_ns, where)) return false;
    }
  return true;
}

}  // namespace gpk
