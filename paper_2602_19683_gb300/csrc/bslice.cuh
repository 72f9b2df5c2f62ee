// BF16-slice products on the 5th-generation tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32
// accumulation in tensor memory) for the reduced-precision and the FP64-emulating forms of the
// trailing updates, the panel TRSMs and the covariance products (Sec. 3.2's SYRK/GEMM/TRSM tile
// operations, Eq. 3's V and W products). A value x is represented by kS BF16 "slices":
//
//  * floating split (GP_BF16 kS = 1, GP_BF16X3 kS = 2, GP_BF16X6 kS = 3): x is rounded to FP32 f,
//    s1 = bf16(f), s2 = bf16(f - s1), s3 = bf16(f - s1 - s2) (each remainder exact in FP32). A product
//    a b^T is formed from the slice products s_p t_q with p + q <= kS + 1 (1, 3 or 6 of them), all
//    accumulated into one FP32 accumulator.
//  * fixed-point digits (GP_FP64_OZAKI, kS = 7; the error-free splitting of Ozaki et al. 2012 with
//    BF16 digits, as in the tensor-core DGEMM emulations of Mukunoki et al. 2020 and Ootomo, Ozaki and
//    Yokota 2024): with a power-of-two scale S = 2^e (|x| <= S), F = round(x 2^(56-e)) is cut into
//    balanced base-256 digits, x ~ S sum_{p=1..7} d_p 2^(-8p), |d_1| <= 256, d_2..d_7 in [-128, 128).
//    Every digit is an integer of at most 8 significant bits, so BF16 holds it exactly and every
//    digit product is exact in FP32. The digit products of equal weight (level L = p + q, L = 2..8:
//    28 products) are accumulated in their own TMEM region. Their FP32 sums stay exact integers
//    (below 2^24): for one 128-wide tile product at any scale up to level 7, and for the grouped
//    updates (at most 512 k, rows of norm <= S: L's rows, V's columns) up to level 4 by the
//    Cauchy-Schwarz bound on the leading digits, the deeper levels being sums of rounding digits
//    whose size is ~2^17; a rounded deep level costs at most 2^(2-8L) S_A S_B. The epilogue turns
//    the seven level sums into one 64-bit fixed-point sum sum_L A_L 2^(lsb - 8L) on the integer pipe
//    (lsb = 56 for norm-bounded operands, 52 for max-scaled single tiles, so the sum fits 63 bits)
//    and that into an FP64 value scaled by S_A S_B 2^-lsb. Truncating at level 8 drops terms of
//    weight 2^-72 S_A S_B per digit product: the product is as accurate as an FP64 product, at 28
//    BF16 tensor-core products instead of one FP64 product.
//
// Packed operand layout (global memory, written once by cta_pack_bs, copied verbatim into shared
// memory by bulk copies): an R x Kd operand (R a multiple of 128) is a sequence of chunks, one per
// (128-row block rb, kKC-wide k block kc) in the order rb (Kd / kKC) + kc; a chunk holds the kS slices
// one after the other, each 128 rows x kKC BF16 in the K-major swizzled layout the MMA reads: kKC = 32
// (floating split: 8 KB slices, 64-byte swizzle, 8-row groups 512 B apart) or kKC = 16 (fixed point: 4 KB
// slices, 32-byte swizzle, groups 256 B apart). Rows 64h..64h+63 of a slice are its contiguous second
// half, themselves a valid 64-row operand.
//
// Every wait is bounded (DevStatus time-out); after a time-out the issuing thread waits, bounded, for
// its own copies and MMAs in flight before the CTA leaves, so shared memory and TMEM are quiet.
#pragma once
#include "umma_packed.cuh"

namespace gpk {

// Chunk widths: 32-wide k chunks (64 bytes of BF16 per row, 64-byte swizzle) for every form; the
// layout also takes 16-wide chunks (32 bytes per row, 32-byte swizzle), which let the fixed-point
// form's stages come five deep instead of two but measured slower (Cholesky at n = 32768: 0.64 s
// against 0.52 s): the per-chunk issue and barrier work, not the bytes in flight, set its rate.
constexpr int kBsKcFloat = 32, kBsKcFixed = 32;
template <int kKC>
__host__ __device__ constexpr int bs_slice_bytes() { return kUmmaM * kKC * 2; }  // one slice of a 128-row chunk
constexpr int kBsMaxStages = 6;
constexpr int kBsStageMem = 210 * 1024;                // stage memory (inside kUmmaSmemBytes)
constexpr int kOzSlices = 7, kOzLevels = 7;            // digits 1..7, levels 2..8
constexpr int kOzLsbBounded = 56;   // fixed-point sum unit 2^-56 S_A S_B: operands with rows of norm <= S
constexpr int kOzLsbTile = 52;      // 2^-52 S_A S_B: max-scaled operands of one 128-wide tile product
static_assert(kBsStageMem + 1024 <= kUmmaSmemBytes, "slice stages must fit the dynamic smem");
static_assert(kOzLevels * 64 <= kUmmaTmemCols, "seven 64-column level accumulators must fit TMEM");
static_assert(128 * 129 * 8 + 10 * 1024 * 8 + 1024 <= kUmmaSmemBytes,
              "the factored 128 tile and the blocks of its FP64 inverse must fit the dynamic smem");

// Byte offset of BF16 element (r, k) (k < kKC) in a K-major swizzled slice: rows of 2 kKC bytes in
// 8-row groups; the 16-byte unit u of row r is stored at u ^ ((r >> 1) & 3) (64-byte swizzle, kKC = 32)
// or u ^ ((r >> 2) & 1) (32-byte swizzle, kKC = 16).
template <int kKC>
__device__ __forceinline__ uint32_t bs_offset(int r, int k) {
  if constexpr (kKC == 32)
    return (uint32_t)((r >> 3) * 512 + (r & 7) * 64 + ((((k >> 3) ^ ((r >> 1) & 3))) << 4) + (k & 7) * 2);
  else
    return (uint32_t)((r >> 3) * 256 + (r & 7) * 32 + ((((k >> 3) ^ ((r >> 2) & 1))) << 4) + (k & 7) * 2);
}

// Shared-memory matrix descriptor of a K-major swizzled BF16 operand: 64-byte swizzle with 8-row
// groups 512 B apart (kKC = 32), or 32-byte swizzle with groups 256 B apart (kKC = 16).
template <int kKC>
__device__ __forceinline__ uint64_t bs_desc(uint32_t saddr) {
  constexpr uint64_t sbo = (uint64_t)(8 * kKC * 2) >> 4, mode = kKC == 32 ? 4 : 6;
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | (sbo << 32) | ((uint64_t)1 << 46) |
         (mode << 61);
}

// Instruction descriptor: kind::f16, FP32 accumulator, A and B BF16, both K-major, M = 128, N given.
__device__ __forceinline__ uint32_t idesc_bf16(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kUmmaM >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// BF16 bits (round to nearest, ties to even) of an FP32 value; finite inputs of ordinary size.
__device__ __forceinline__ uint32_t bf16_rn_bits(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b + 0x7FFFu + ((b >> 16) & 1u)) >> 16;
}
__device__ __forceinline__ float bf16_to_f32(uint32_t h) { return __uint_as_float(h << 16); }

// Floating split of an FP32 value into kS BF16 slices (kS <= 3); each remainder is exact in FP32.
template <int kS>
__device__ __forceinline__ void split_float(float f, uint32_t (&h)[kS]) {
#pragma unroll
  for (int s = 0; s < kS; ++s) {
    h[s] = bf16_rn_bits(f);
    f -= bf16_to_f32(h[s]);
  }
}

// Exact FP32 value of a small integer d (|d| < 2^22) with an FP32 add (magic-number conversion).
__device__ __forceinline__ float small_int_to_f32(int d) {
  return __uint_as_float(0x4B400000u + (uint32_t)d) - 12582912.0f;
}

// Fixed-point digits of x at scale 2^e (|x| <= 2^e): F = round(x 2^(56-e)) (ties away from zero),
// cut into balanced base-256 digits d_1..d_7 (most significant first), returned as BF16 bits. Integer
// operations on the bits of x only.
__device__ __forceinline__ void split_fixed(double x, int e, uint32_t (&h)[kOzSlices]) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  long long F = 0;
  if (ex != 0) {
    const long long m = (bits & 0xFFFFFFFFFFFFFLL) | 0x10000000000000LL;  // 53-bit integer
    const int sh = (ex - 1023) + 4 - e;  // x = m 2^(ex-1023-52); F = m 2^(ex-1023-52+56-e)
    if (sh >= 0)
      F = m << (sh < 10 ? sh : 10);  // |x| <= 2^e keeps sh <= 4; the clamp only guards the shift
    else if (sh > -54)
      F = (m + (1LL << (-sh - 1))) >> (-sh);
    if (bits < 0) F = -F;
  }
#pragma unroll
  for (int p = kOzSlices - 1; p >= 1; --p) {
    const int d = (int)((F + 128) & 255) - 128;
    F = (F - d) >> 8;
    h[p] = __float_as_uint(small_int_to_f32(d)) >> 16;
  }
  h[0] = __float_as_uint(small_int_to_f32((int)F)) >> 16;
}

template <int kKC>
__device__ __forceinline__ size_t bs_chunk_off(int rb, int kc, int Kd, int kS) {
  return ((size_t)rb * (Kd / kKC) + kc) * (size_t)kS * bs_slice_bytes<kKC>();
}

// Writes the packed kS-slice operand of an R x Kd FP64 block: Op[r][k] = src[r * ld + k] (trans = false)
// or src[k * ld + r] (trans = true). kOz: fixed-point digits at scale 2^e; otherwise floating split.
// kKC: the chunk width of the layout. R a multiple of 128, Kd of kKC. Loads coalesced in both forms.
template <int kS, bool kOz, int kKC>
__device__ void cta_pack_bs(const double* src, int ld, bool trans, int R, int Kd, uint8_t* dst, int e) {
  constexpr int kSlice = bs_slice_bytes<kKC>();
  const int t = threadIdx.x;
  for (int rb = 0; rb < R / kUmmaM; ++rb)
    for (int kc = 0; kc < Kd / kKC; ++kc) {
      uint8_t* ch = dst + bs_chunk_off<kKC>(rb, kc, Kd, kS);
      if (!trans) {  // thread: k pair 2 kp of its row; kKC / 2 threads per row
        constexpr int kPairs = kKC / 2, kRowsPerPass = kThreads / kPairs, kPasses = kUmmaM / kRowsPerPass;
        const int kp = t % kPairs, rr = t / kPairs;
        double2 d[kPasses];
#pragma unroll
        for (int pass = 0; pass < kPasses; ++pass)
          d[pass] = __ldcg(reinterpret_cast<const double2*>(
                               src + (size_t)(rb * kUmmaM + rr + kRowsPerPass * pass) * ld + kc * kKC) + kp);
#pragma unroll
        for (int pass = 0; pass < kPasses; ++pass) {
          const uint32_t off = bs_offset<kKC>(rr + kRowsPerPass * pass, 2 * kp);
          uint32_t h0[kS], h1[kS];
          if constexpr (kOz) {
            split_fixed(d[pass].x, e, h0);
            split_fixed(d[pass].y, e, h1);
          } else {
            split_float<kS>(f64_to_f32_rn(d[pass].x), h0);
            split_float<kS>(f64_to_f32_rn(d[pass].y), h1);
          }
#pragma unroll
          for (int s = 0; s < kS; ++s)
            *reinterpret_cast<uint32_t*>(ch + s * kSlice + off) = h0[s] | (h1[s] << 16);
        }
      } else {  // thread: k = t % kKC, a run of kRows consecutive r (two per double2 load)
        constexpr int kGroups = kThreads / kKC, kRows = kUmmaM / kGroups;
        const int k = t % kKC, g = t / kKC;
        double2 d[kRows / 2];
#pragma unroll
        for (int q = 0; q < kRows / 2; ++q)
          d[q] = __ldcg(reinterpret_cast<const double2*>(src + (size_t)(kc * kKC + k) * ld + rb * kUmmaM +
                                                         g * kRows) + q);
#pragma unroll
        for (int q = 0; q < kRows / 2; ++q) {
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            uint32_t hv[kS];
            if constexpr (kOz)
              split_fixed(c ? d[q].y : d[q].x, e, hv);
            else
              split_float<kS>(f64_to_f32_rn(c ? d[q].y : d[q].x), hv);
            const uint32_t off = bs_offset<kKC>(g * kRows + 2 * q + c, k);
#pragma unroll
            for (int s = 0; s < kS; ++s)
              *reinterpret_cast<uint16_t*>(ch + s * kSlice + off) = (uint16_t)hv[s];
          }
        }
      }
    }
  fence_proxy_async_global();  // read later by bulk copies (async proxy)
  __syncthreads();
}

// Packed kS-slice operand of an FP32 nb x nb matrix in shared memory (leading dimension ld; rows and
// columns beyond nb are zero), floating split (the mixed forms' FP32 inverse of a diagonal tile).
template <int kS>
__device__ void cta_pack_bs_f32(const float* Xs, int ld, int nb, uint8_t* dst) {
  constexpr int kKC = kBsKcFloat, kSlice = bs_slice_bytes<kKC>();
  for (int kc = 0; kc < nb / kKC; ++kc) {
    uint8_t* ch = dst + bs_chunk_off<kKC>(0, kc, nb, kS);
    for (int e2 = threadIdx.x; e2 < kUmmaM * 16; e2 += kThreads) {
      const int r = e2 >> 4, kp = e2 & 15;
      float f0 = 0.f, f1 = 0.f;
      if (r < nb) {
        f0 = Xs[r * ld + kc * kKC + 2 * kp];
        f1 = Xs[r * ld + kc * kKC + 2 * kp + 1];
      }
      uint32_t h0[kS], h1[kS];
      split_float<kS>(f0, h0);
      split_float<kS>(f1, h1);
      const uint32_t off = bs_offset<kKC>(r, 2 * kp);
#pragma unroll
      for (int s = 0; s < kS; ++s) *reinterpret_cast<uint32_t*>(ch + s * kSlice + off) = h0[s] | (h1[s] << 16);
    }
  }
  fence_proxy_async_global();
  __syncthreads();
}

// An e with max |src| < 2^e (the smallest such power of two, or the next) over an R x C FP64 block
// (row-major, ld): the per-tile scale of a fixed-point operand used in a single-tile product. Returns
// -1022 for an all-zero block.
__device__ int cta_scale_exp(const double* src, int ld, int R, int C, int* s_flag) {
  int mx = 0;  // largest biased exponent field; a value with field ex is < 2^(ex - 1022)
  for (int e2 = threadIdx.x; e2 < R * C; e2 += kThreads) {
    const long long b = __double_as_longlong(__ldcg(src + (size_t)(e2 / C) * ld + e2 % C));
    const int ex = (int)((b >> 52) & 0x7FF);
    mx = ex > mx ? ex : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (threadIdx.x == 0) *s_flag = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) atomicMax(s_flag, mx);
  __syncthreads();
  const int ex = *s_flag;
  __syncthreads();
  return ex == 0 ? -1022 : ex - 1022;  // |x| < 2^(ex-1022)
}

// x 2^e as an FP64 value, rounded to nearest (ties to even), on the integer pipe (|x| < 2^63, the
// result in the normal range or flushed to a signed zero below it).
__device__ __forceinline__ double i64_to_f64_scaled(long long x, int e) {
  if (x == 0) return 0.0;
  const unsigned long long sign = x < 0 ? 0x8000000000000000ULL : 0ULL;
  unsigned long long u = x < 0 ? (unsigned long long)(-x) : (unsigned long long)x;
  const int lz = __clzll((long long)u);
  u <<= lz;  // leading one at bit 63
  unsigned long long mant = u >> 11;
  const unsigned long long rem = u & 0x7FFULL;
  if (rem > 0x400ULL || (rem == 0x400ULL && (mant & 1ULL))) ++mant;
  int E = 63 - lz + e;
  if (mant >> 53) {
    mant >>= 1;
    ++E;
  }
  if (E + 1023 <= 0) return __longlong_as_double((long long)sign);
  return __longlong_as_double((long long)(sign | ((unsigned long long)(E + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFULL)));
}

// Epilogue of one 128 x 64 half of a fixed-point product whose MMAs are all complete: the seven
// level sums (TMEM columns 64 (L - 2) + c, L = 2..8; integers in FP32) of every entry are combined
// into sum_L A_L 2^(lsb - 8L) in 64-bit integers (the levels below the unit rounded to nearest),
// converted to FP64 with the factor 2^e2 (e2 = eA + eB - lsb), staged in shared memory and applied to
// C with coalesced accesses:
// C -= result (kStore: C = result); lower: entries with column > row are left as they are.
// Warp w reads TMEM lanes 32 (w % 4).. and the 32-column quarter (w / 4) of the half.
template <bool kStore>
__device__ void oz_epilogue(UmmaState& u, double* C, int ldc, int m0, int n0, bool lower, int e2, int lsb) {
  umma_fence_after();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int ldS = 65;
  double* sC = reinterpret_cast<double*>(u.smem);  // 128 x 65 doubles (the stages are free now)
  const int row = (w & 3) * 32 + lane, cb = (w >> 2) * 32;
  const uint32_t tl = u.tmem + ((uint32_t)((w & 3) * 32) << 16);
#pragma unroll 1
  for (int g = 0; g < 4; ++g) {
    long long acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0;
#pragma unroll
    for (int L = 2; L <= 8; ++L) {
      uint32_t v[8];
      tmem_ld8(tl + (uint32_t)((L - 2) * 64 + cb + 8 * g), v);
      tmem_wait_ld();
      const int sh = lsb - 8 * L;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const long long a = (long long)__float2int_rn(__uint_as_float(v[j]));
        acc[j] += sh >= 0 ? (a << sh) : ((a + (1LL << (-sh - 1))) >> (-sh));
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) sC[row * ldS + cb + 8 * g + j] = i64_to_f64_scaled(acc[j], e2);
  }
  umma_fence_before();
  __syncthreads();
  for (int r = w; r < kUmmaM; r += kThreads / 32) {
    const int m = m0 + r, n = n0 + 2 * lane;
    double2* c2 = reinterpret_cast<double2*>(C + (size_t)m * ldc + n);
    const double x0 = sC[r * ldS + 2 * lane], x1 = sC[r * ldS + 2 * lane + 1];
    double2 c;
    if (kStore) {
      c = make_double2(x0, x1);
    } else {
      c = __ldcg(c2);
      if (!lower || n <= m) c.x -= x0;
      if (!lower || n + 1 <= m) c.y -= x1;
    }
    *c2 = c;
  }
  __syncthreads();  // smem and TMEM are reused next
}

// X = L^{-1} in FP64 for a factored nb x nb diagonal tile still held in shared memory by the POTRF
// (sL: nb x (nb + 1) doubles at the start of `smem`, lower triangle; nb a multiple of 32, at most 128),
// written to Xg (nb x nb row-major, upper triangle zero). Blocked by 32: warp d inverts diagonal block d
// (lane j solves column j, the pivots' reciprocals taken once and shared by shuffles), then block rows
// bi = 1.. follow X_{bi,bj} = -X_{bi,bi} sum_{bj <= k < bi} L_{bi,k} X_{k,bj}. The lower blocks of X live
// in shared memory behind the factor (10 blocks of 32 x 32 doubles for nb = 128).
__device__ __noinline__ void cta_inverse_f64_smem(uint8_t* smem, int nb, double* Xg) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31, ldl = nb + 1, nblk = nb / 32;
  const double* sL = reinterpret_cast<const double*>(smem);
  double* sX = reinterpret_cast<double*>(smem + (size_t)nb * ldl * 8);
  auto xblk = [&](int bi, int bj) { return sX + (size_t)(bi * (bi + 1) / 2 + bj) * 1024; };
  if (w < nblk) {  // diagonal blocks
    const int d0 = 32 * w;
    const double rd = 1.0 / sL[(d0 + lane) * ldl + d0 + lane];
    double x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      double acc = (i == lane) ? 1.0 : 0.0;
#pragma unroll
      for (int k = 0; k < i; ++k) acc = fma(-sL[(d0 + i) * ldl + d0 + k], x[k], acc);
      x[i] = acc * __shfl_sync(0xffffffffu, rd, i);
    }
    double* X = xblk(w, w);
#pragma unroll
    for (int i = 0; i < 32; ++i) X[i * 32 + lane] = x[i];
  }
  __syncthreads();
  for (int bi = 1; bi < nblk; ++bi) {
    // W_bj = sum_{bj <= k < bi} L_{bi,k} X_{k,bj}, parked in the (unused) slots of X_{bi,bj}
    for (int e = t; e < bi * 1024; e += kThreads) {
      const int bj = e >> 10, r = (e >> 5) & 31, c = e & 31;
      const double* lrow = sL + (32 * bi + r) * ldl;
      double acc = 0.0;
      for (int kb = bj; kb < bi; ++kb) {
        const double* Xk = xblk(kb, bj);
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) acc = fma(lrow[32 * kb + kk], Xk[kk * 32 + c], acc);
      }
      xblk(bi, bj)[r * 32 + c] = acc;
    }
    __syncthreads();
    // X_{bi,bj} = -X_{bi,bi} W_bj (through registers: W is read in place); bi * 1024 <= 3 * 1024 entries,
    // twelve per thread
    constexpr int kPer = 3 * 1024 / kThreads;
    static_assert(kPer * kThreads == 3 * 1024, "the entries of block row 3 split evenly over the CTA");
    double res[kPer];
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = t + q * kThreads;
      res[q] = 0.0;
      if (e < bi * 1024) {
        const int bj = e >> 10, r = (e >> 5) & 31, c = e & 31;
        const double* xrow = xblk(bi, bi) + r * 32;
        const double* Wb = xblk(bi, bj);
        double acc = 0.0;
        for (int k = 0; k <= r; ++k) acc = fma(xrow[k], Wb[k * 32 + c], acc);
        res[q] = -acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      const int e = t + q * kThreads;
      if (e < bi * 1024) {
        const int bj = e >> 10, r = (e >> 5) & 31, c = e & 31;
        xblk(bi, bj)[r * 32 + c] = res[q];
      }
    }
    __syncthreads();
  }
  for (int e = t; e < nb * nb; e += kThreads) {  // coalesced write-out, zero above the diagonal
    const int i = e / nb, j = e % nb, bi = i >> 5, bj = j >> 5;
    Xg[e] = bj <= bi ? xblk(bi, bj)[(i & 31) * 32 + (j & 31)] : 0.0;
  }
  __syncthreads();
}

// Pipeline state of the slice products (barriers in smem; thread 0 drives it).
struct BsPipe {
  uint64_t* full;   // kBsMaxStages: completed by the bulk copies' transaction bytes
  uint64_t* empty;  // kBsMaxStages: completed by the MMA commit
  uint32_t fph[kBsMaxStages], eph[kBsMaxStages];
  uint32_t fpend[kBsMaxStages], epend[kBsMaxStages];
};

// Product C[128 x 128 tile at (m0, n0)] (FP64, ldc) -= (or, kStore, =) sum_j A_j[m0..] B_j[n0..]^T over
// Kd from packed kS-slice operands (pairs j < pr.n, each A_j / B_j a packed operand whose 128-row blocks
// rb = m0 / 128, n0 / 128 are used). kOz: fixed-point digits, scale exponents eA, eB, fixed-point
// unit 2^-lsb S_A S_B (kOzLsbBounded or kOzLsbTile); else floating split. lower: only entries with
// column <= row of the tile are written (diagonal tiles).
// Thread 0 runs copies and MMAs; all threads run the epilogue. False (error raised, copies and MMAs
// drained) on a time-out.
template <int kS, bool kOz, bool kStore = false>
__device__ bool bs_block_sub(UmmaState& u, BsPipe& bp, double* C, int ldc, const PkPairs& pr, int Kd, int m0,
                             int n0, bool lower, int eA, int eB, int lsb, DevStatus* st, long long timeout_ns,
                             long long where) {
  constexpr int kKC = kOz ? kBsKcFixed : kBsKcFloat;  // k per chunk
  constexpr int kSlice = bs_slice_bytes<kKC>();
  constexpr int kRowsB = kOz ? 64 : 128;  // B rows per pass (the fixed-point form runs two 64-column halves)
  constexpr int kBSlice = kRowsB * kKC * 2;  // bytes of one B slice in a stage
  constexpr int kABytes = kS * kSlice, kBBytes = kS * kBSlice;
  constexpr int kStage = kABytes + kBBytes;
  constexpr int kStages = (kBsStageMem / kStage) < kBsMaxStages ? (kBsStageMem / kStage) : kBsMaxStages;
  static_assert(kStages >= 2, "at least two stages");
  static_assert(kStage % 1024 == 0, "stages stay 1024-byte aligned");
  const int nkp = Kd / kKC, nk = nkp * pr.n;
  const int rbA = m0 / kUmmaM, rbB = n0 / kUmmaM;
  constexpr int kHalves = kOz ? 2 : 1;
  for (int half = 0; half < kHalves; ++half) {
    bool ok = true;
    fence_async_smem();  // earlier generic use of the stage memory before the copies
    __syncthreads();
    if (threadIdx.x == 0) {
      fence_proxy_async_global();  // packed tiles acquired through the dependency counters
      auto load = [&](int i) {
        const int s = i % kStages, p = i / nkp, kc = i % nkp;
        uint8_t* base = u.smem + s * kStage;
        mbar_expect_tx(&bp.full[s], kStage);
        tma_bulk_g2s(base, pr.A[p] + bs_chunk_off<kKC>(rbA, kc, Kd, kS), kABytes, &bp.full[s]);
        const uint8_t* bsrc = pr.B[p] + bs_chunk_off<kKC>(rbB, kc, Kd, kS);
        if (kOz) {  // rows 64 half .. of every slice: a contiguous kBSlice bytes at half * kBSlice
#pragma unroll
          for (int q = 0; q < kS; ++q)
            tma_bulk_g2s(base + kABytes + q * kBSlice, bsrc + q * kSlice + half * kBSlice, kBSlice, &bp.full[s]);
        } else {
          tma_bulk_g2s(base + kABytes, bsrc, kBBytes, &bp.full[s]);
        }
        bp.fpend[s] = 1;
      };
      // Chunk loads are requested in order as soon as their stage is free (the MMAs of the chunk it held
      // kStages earlier have completed). The fixed-point form probes that without blocking after each
      // chunk's MMAs are issued, so several chunks' MMAs stay queued on the tensor pipe while copies
      // fly; the floating-split forms wait for the previous chunk's MMAs and refill its stage. Either
      // way a bounded blocking wait when the chunk about to be consumed has not been requested yet.
      int next_load = 0, issued = 0;
      auto refill = [&](bool block) -> bool {
        while (next_load < nk) {
          const int j = next_load, sj = j % kStages;
          if (j >= kStages) {
            if (j - kStages >= issued) break;  // the stage still holds an unconsumed chunk
            if (bp.epend[sj]) {
              if (block) {
                if (!mbar_wait(&bp.empty[sj], bp.eph[sj], st, timeout_ns, where)) return false;
              } else if (!mbar_test_wait(&bp.empty[sj], bp.eph[sj])) {
                break;
              }
              bp.eph[sj] ^= 1u;
              bp.epend[sj] = 0;
            }
          }
          load(j);
          ++next_load;
          block = false;
        }
        return true;
      };
      for (int i = 0; i < nk && ok; ++i) {
        if (next_load <= i && !refill(true)) {
          ok = false;
          break;
        }
        const int s = i % kStages;
        if (!mbar_wait(&bp.full[s], bp.fph[s], st, timeout_ns, where)) {
          ok = false;
          break;
        }
        bp.fph[s] ^= 1u;
        bp.fpend[s] = 0;
        umma_fence_after();
        const uint32_t a0 = smem_u32(u.smem + s * kStage), b0 = a0 + kABytes;
#pragma unroll
        for (int ks = 0; ks < kKC / 16; ++ks) {
          const uint32_t o = ks * 32;  // 16 BF16 = 32 bytes along K inside the swizzled row
          if constexpr (kOz) {
            // slice p of A against slices q = 1 .. 8 - p of B, stacked along N (64 columns each), into
            // the level regions L = p + q (TMEM columns 64 (L - 2)); at most 4 levels per instruction
#pragma unroll
            for (int p = 1; p <= kOzSlices; ++p) {
              const int nq = kOzSlices + 1 - p;
#pragma unroll
              for (int q0 = 1; q0 <= nq; q0 += 4) {
                const int q1 = (q0 + 3 < nq) ? q0 + 3 : nq;
                const int N = (q1 - q0 + 1) * 64;
                const uint32_t acc = (i > 0 || ks > 0 || p > 1) ? 1u : 0u;  // p = 1 opens every level
                umma_bf16(u.tmem + (uint32_t)((p + q0 - 2) * 64), bs_desc<kKC>(a0 + (p - 1) * kSlice + o),
                          bs_desc<kKC>(b0 + (q0 - 1) * kBSlice + o), idesc_bf16(N), acc);
              }
            }
          } else {
            // products s_p t_q with p + q <= kS + 1, accumulated in one 128-column accumulator; pairs
            // j >= 4 go to a second one (TMEM columns 128..255), so no FP32 chain spans more than four
            const int acc_i = (i / nkp) >= kPairsPerAcc ? 1 : 0;
            const bool first = (i % (kPairsPerAcc * nkp)) == 0 && ks == 0;
            const uint32_t d = u.tmem + (uint32_t)(acc_i * kUmmaN);
            bool opened = false;
#pragma unroll
            for (int p = 1; p <= kS; ++p)
#pragma unroll
              for (int q = 1; q + p <= kS + 1; ++q) {
                umma_bf16(d, bs_desc<kKC>(a0 + (p - 1) * kSlice + o), bs_desc<kKC>(b0 + (q - 1) * kBSlice + o),
                          idesc_bf16(kUmmaN),
                          (first && !opened) ? 0u : 1u);
                opened = true;
              }
          }
        }
        umma_commit(&bp.empty[s]);
        bp.epend[s] = 1;
        issued = i + 1;
        if constexpr (kOz) {
          refill(false);
        } else if (i >= 1 && next_load < nk && next_load == i - 1 + kStages) {
          // floating-split forms (4-6 stages): refill the stage of chunk i-1 as soon as its MMAs are
          // done, waiting for them (measured faster for these deep pipelines than the probes)
          if (!refill(true)) {
            ok = false;
            break;
          }
        }
      }
      // every MMA complete before TMEM is read and the stages are reused
      for (int i = 0; i < kStages; ++i) {
        const int s = (nk + i) % kStages;  // oldest outstanding commit first
        if (bp.epend[s]) {
          if (ok)
            ok = mbar_wait(&bp.empty[s], bp.eph[s], st, timeout_ns, where);
          else
            mbar_drain(&bp.empty[s], bp.eph[s], timeout_ns);
          bp.eph[s] ^= 1u;
          bp.epend[s] = 0;
        }
      }
      if (!ok) {
        for (int s = 0; s < kStages; ++s)
          if (bp.fpend[s]) {
            mbar_drain(&bp.full[s], bp.fph[s], timeout_ns);
            bp.fph[s] ^= 1u;
            bp.fpend[s] = 0;
          }
        for (int s = 0; s < kStages; ++s)
          if (bp.epend[s]) {
            mbar_drain(&bp.empty[s], bp.eph[s], timeout_ns);
            bp.eph[s] ^= 1u;
            bp.epend[s] = 0;
          }
      }
    }
    if (__syncthreads_or(!ok)) return false;
    if constexpr (kOz) {
      oz_epilogue<kStore>(u, C, ldc, m0, n0 + 64 * half, lower, eA + eB - lsb, lsb);
    } else {
      umma_epilogue<kStore>(u, C, ldc, m0, n0, lower, pr.n > kPairsPerAcc ? 2 : 1);
    }
    fence_async_smem();  // generic smem traffic of the epilogue before the next bulk copies
    __syncthreads();
  }
  return true;
}

}  // namespace gpk
