// Packed tensor-core operands of the mixed-precision mode, and the products fed from them by bulk
// tensor-memory-access (TMA) copies.
//
// A tile that many trailing updates read (a panel tile L_IJ after its TRSM, a block V_Jc of the
// covariance solve after its triangular solve) is converted ONCE into the operand format of the
// tcgen05 3xTF32 product: each FP64 value is split into a TF32 high part and a TF32-rounded remainder,
// and the halves are stored exactly as the MMA reads them from shared memory (K-major, 128-byte
// swizzle, 8-row groups 1024 bytes apart). A packed R x Kd operand is a sequence of chunks, one per
// (128-row block rb, 32-wide k block kc) in the order rb * (Kd / 32) + kc; a chunk is the 16 KB high
// tile followed by the 16 KB low tile (32 KB, the same bytes per value as the FP64 source).
//
// A consumer then moves each 32 KB chunk into shared memory with one cp.async.bulk (no registers, no
// conversion), completion counted on an mbarrier by bytes, and one thread issues the 12 MMAs of the
// chunk as soon as its A and B halves have landed. Stages alternate so that the copies of the next
// chunk fly while the tensor cores work on the current one. The accumulator (FP32 in TMEM) leaves
// through the same epilogue as the register-staged path: subtracted from the FP64 C tile.
//
// Every wait is bounded; after a time-out the thread waits (bounded) for its own copies and MMAs in
// flight so that shared memory and TMEM are quiet when the CTA leaves.
#pragma once
#include "umma.cuh"

namespace gpk {

constexpr int kPkChunkBytes = 2 * kUmmaTileBytes;  // high + low tile of one 128-row x 32-k chunk
constexpr int kPairsPerAcc = 4;                     // operand pairs per TMEM accumulator (two of them)
static_assert(2 * kPairsPerAcc >= kUmmaMaxPairs, "every pair needs an accumulator");
static_assert(2 * kUmmaN <= kUmmaTmemCols, "two accumulators must fit the allocated TMEM columns");
static_assert(2 * kPkChunkBytes == kUmmaStageBytes, "a stage holds one A and one B chunk");
static_assert(kPkStages * kUmmaStageBytes + 1024 <= kUmmaSmemBytes, "stages must fit the dynamic smem");
static_assert(kMixedTileSmemBytes + 128 * 128 * 4 + 1024 <= kUmmaSmemBytes,
              "a 128 x 129 FP64 tile and a 128 x 128 FP32 copy must fit the dynamic smem");

__device__ __forceinline__ size_t pk_chunk_off(int rb, int kc, int Kd) {
  return ((size_t)rb * (Kd / kUmmaKChunk) + kc) * kPkChunkBytes;
}

// Writes the packed operand of an R x Kd FP64 block: Op[r][k] = src[r * ld + k] (trans = false) or
// src[k * ld + r] (trans = true). R a multiple of 128, Kd of 32. Loads are coalesced in both forms;
// stores of the transposed form are one 128-byte packed row per warp instruction.
__device__ void cta_pack_operand(const double* src, int ld, bool trans, int R, int Kd, uint8_t* dst) {
  const int t = threadIdx.x;
  for (int rb = 0; rb < R / kUmmaM; ++rb)
    for (int kc = 0; kc < Kd / kUmmaKChunk; ++kc) {
      uint8_t* hi = dst + pk_chunk_off(rb, kc, Kd);
      uint8_t* lo = hi + kUmmaTileBytes;
      if (!trans) {
        const int kp = t & 15, rr = t >> 4;
        double2 d[8];
#pragma unroll
        for (int pass = 0; pass < 8; ++pass)
          d[pass] = __ldcg(reinterpret_cast<const double2*>(src + (size_t)(rb * kUmmaM + rr + 16 * pass) * ld +
                                                            kc * kUmmaKChunk) + kp);
#pragma unroll
        for (int pass = 0; pass < 8; ++pass) {
          const float f0 = f64_to_f32_rn(d[pass].x), f1 = f64_to_f32_rn(d[pass].y);
          const float h0 = tf32_rn(f0), h1 = tf32_rn(f1);
          const uint32_t off = sw128_offset(rr + 16 * pass, 2 * kp);
          *reinterpret_cast<float2*>(hi + off) = make_float2(h0, h1);
          *reinterpret_cast<float2*>(lo + off) = make_float2(tf32_rn(f0 - h0), tf32_rn(f1 - h1));
        }
      } else {
        const int k = t & 31, w = t >> 5;  // lane: k row of the source; warp: 16 consecutive r
        double2 d[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
          d[q] = __ldcg(reinterpret_cast<const double2*>(src + (size_t)(kc * kUmmaKChunk + k) * ld + rb * kUmmaM +
                                                         w * 16) + q);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const float f = f64_to_f32_rn(e ? d[q].y : d[q].x), h = tf32_rn(f);
            const uint32_t off = sw128_offset(w * 16 + 2 * q + e, k);
            *reinterpret_cast<float*>(hi + off) = h;
            *reinterpret_cast<float*>(lo + off) = tf32_rn(f - h);
          }
        }
      }
    }
  fence_proxy_async_global();  // the bytes are read later by bulk copies (async proxy)
  __syncthreads();
}

// Operand pairs of a packed product: C -= sum_p A_p B_p^T, each A_p / B_p a packed T-row operand.
struct PkPairs {
  const uint8_t* A[kUmmaMaxPairs];
  const uint8_t* B[kUmmaMaxPairs];
  int n;
};

// Thread 0: bounded wait without raising an error (used while draining after a time-out).
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity, long long timeout_ns) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity) && (long long)(globaltimer() - t0) < timeout_ns) {
  }
}

// C[128 x 128 block at (m0, n0)] (FP64, ldc) -= sum_p A_p[m0..] B_p[n0..]^T over Kd, from packed
// operands. Thread 0 runs the copy/MMA pipeline; all threads run the epilogue. Returns false (error
// raised, copies and MMAs drained) on a time-out.
// kProd: 3 = the three split products (3xTF32); 1 = the high parts only (plain TF32, GP_TF32).
template <bool kStore = false, int kProd = 3>
__device__ bool umma_pk_block_sub(UmmaState& u, double* C, int ldc, const PkPairs& pr, int Kd, int m0, int n0,
                                  bool lower, DevStatus* st, long long timeout_ns, long long where) {
  const int nkp = Kd / kUmmaKChunk, nk = nkp * pr.n;
  const int rbA = m0 / kUmmaM, rbB = n0 / kUmmaN;
  bool ok = true;
  fence_async_smem();  // earlier generic use of the stage memory (other tile routines) before the copies
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_proxy_async_global();  // tiles acquired through the dependency counters feed bulk copies
    auto load = [&](int i) {
      const int s = i % kPkStages, p = i / nkp, kc = i % nkp;
      uint8_t* base = u.smem + s * 2 * kPkChunkBytes;
      mbar_expect_tx(&u.pfull[s], 2 * kPkChunkBytes);
      tma_bulk_g2s(base, pr.A[p] + pk_chunk_off(rbA, kc, Kd), kPkChunkBytes, &u.pfull[s]);
      tma_bulk_g2s(base + kPkChunkBytes, pr.B[p] + pk_chunk_off(rbB, kc, Kd), kPkChunkBytes, &u.pfull[s]);
      u.fpend[s] = 1;
    };
    // loads requested as soon as their stage is free, probed without blocking after each chunk's MMAs
    // (several chunks' MMAs stay queued); a bounded blocking wait only for the chunk about to be consumed
    int next_load = 0, issued = 0;
    auto refill = [&](bool block) -> bool {
      while (next_load < nk) {
        const int j = next_load, sj = j % kPkStages;
        if (j >= kPkStages) {
          if (j - kPkStages >= issued) break;  // the stage still holds an unconsumed chunk
          if (u.epend[sj]) {
            if (block) {
              if (!mbar_wait(&u.pempty[sj], u.eph[sj], st, timeout_ns, where)) return false;
            } else if (!mbar_test_wait(&u.pempty[sj], u.eph[sj])) {
              break;
            }
            u.eph[sj] ^= 1u;
            u.epend[sj] = 0;
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
      const int s = i % kPkStages;
      if (!mbar_wait(&u.pfull[s], u.fph[s], st, timeout_ns, where)) {
        ok = false;
        break;
      }
      u.fph[s] ^= 1u;
      u.fpend[s] = 0;
      umma_fence_after();
      const uint32_t a_hi = smem_u32(u.smem + s * 2 * kPkChunkBytes), a_lo = a_hi + kUmmaTileBytes;
      const uint32_t b_hi = a_hi + kPkChunkBytes, b_lo = b_hi + kUmmaTileBytes;
      // pairs 0..3 accumulate in TMEM columns 0..127, pairs 4..7 in columns 128..255, so no FP32
      // accumulation chain (whose additions truncate) runs over more than four column pairs
      const int pair = i / nkp, acc_i = pair >= kPairsPerAcc ? 1 : 0;
      const uint32_t d_tmem = u.tmem + (uint32_t)(acc_i * kUmmaN);
      const bool first = (i % (kPairsPerAcc * nkp)) == 0;  // first chunk of this accumulator
#pragma unroll
      for (int ks = 0; ks < kUmmaKChunk / 8; ++ks) {
        const uint32_t o = ks * 32;
        umma_tf32(d_tmem, umma_desc_sw128(a_hi + o), umma_desc_sw128(b_hi + o), (!first || ks > 0) ? 1u : 0u);
        if (kProd == 3) {
          umma_tf32(d_tmem, umma_desc_sw128(a_hi + o), umma_desc_sw128(b_lo + o), 1u);
          umma_tf32(d_tmem, umma_desc_sw128(a_lo + o), umma_desc_sw128(b_hi + o), 1u);
        }
      }
      umma_commit(&u.pempty[s]);
      u.epend[s] = 1;
      issued = i + 1;
      refill(false);
    }
    // every MMA of the block must be complete before TMEM is read (and before the stages are reused)
    for (int i = 0; i < kPkStages; ++i) {
      const int s = (nk + i) % kPkStages;  // oldest outstanding commit first
      if (u.epend[s]) {
        if (ok) {
          ok = mbar_wait(&u.pempty[s], u.eph[s], st, timeout_ns, where);
        } else {
          mbar_drain(&u.pempty[s], u.eph[s], timeout_ns);
        }
        u.eph[s] ^= 1u;
        u.epend[s] = 0;
      }
    }
    if (!ok) {
      for (int s = 0; s < kPkStages; ++s)
        if (u.fpend[s]) {
          mbar_drain(&u.pfull[s], u.fph[s], timeout_ns);
          u.fph[s] ^= 1u;
          u.fpend[s] = 0;
        }
      for (int s = 0; s < kPkStages; ++s)
        if (u.epend[s]) {
          mbar_drain(&u.pempty[s], u.eph[s], timeout_ns);
          u.eph[s] ^= 1u;
          u.epend[s] = 0;
        }
    }
  }
  if (__syncthreads_or(!ok)) return false;
  umma_epilogue<kStore>(u, C, ldc, m0, n0, lower, pr.n > kPairsPerAcc ? 2 : 1);
  fence_async_smem();  // generic smem traffic of the epilogue before the next bulk copies
  __syncthreads();
  return true;
}

// Two output tiles that share their right operands: C0 -= sum_p A0_p B_p^T and C1 -= sum_p A1_p B_p^T.
struct PkPairs2 {
  const uint8_t* A0[kUmmaMaxPairs];
  const uint8_t* A1[kUmmaMaxPairs];
  const uint8_t* B[kUmmaMaxPairs];
  int n;
};

// Both 128 x 128 FP64 tiles C0, C1 (ldc) of a PkPairs2 product from packed 128-row operands (Kd a
// multiple of 32), in one pass over the shared B_p: a stage holds the k chunk of A0_p, A1_p and B_p
// (three bulk copies, 96 KB; two stages in the stage memory), and one thread issues the MMAs of both
// outputs on it. Accumulators: output o, column pairs 0..3 / 4..7 -> TMEM columns 256 o + 128 h, so
// no FP32 accumulation chain runs over more than four column pairs. lower0: C0 is a diagonal tile
// (only its lower triangle is updated). Same bounded waits and drain as umma_pk_block_sub; false on a
// time-out.
__device__ bool umma_pk_block2_sub(UmmaState& u, double* C0, double* C1, int ldc, const PkPairs2& pr, int Kd,
                                   bool lower0, DevStatus* st, long long timeout_ns, long long where) {
  constexpr int kStages2 = 2, kStage2Bytes = 3 * kPkChunkBytes;
  static_assert(kStages2 * kStage2Bytes <= kPkStages * kUmmaStageBytes, "two three-operand stages fit the stages");
  static_assert(kStages2 <= kPkStages, "the stages use the first kStages2 barrier pairs");
  static_assert(kUmmaTmemCols >= 4 * kUmmaN, "four accumulators");
  static_assert(kStage2Bytes % 1024 == 0 && kPkChunkBytes % 1024 == 0, "swizzled operands stay 1024-byte aligned");
  const int nkp = Kd / kUmmaKChunk, nk = nkp * pr.n;
  bool ok = true;
  fence_async_smem();  // earlier generic use of the stage memory (other tile routines) before the copies
  __syncthreads();
  if (threadIdx.x == 0) {
    fence_proxy_async_global();  // tiles acquired through the dependency counters feed bulk copies
    auto load = [&](int i) {
      const int s = i % kStages2, p = i / nkp, kc = i % nkp;
      uint8_t* base = u.smem + s * kStage2Bytes;
      mbar_expect_tx(&u.pfull[s], 3 * kPkChunkBytes);
      tma_bulk_g2s(base, pr.A0[p] + pk_chunk_off(0, kc, Kd), kPkChunkBytes, &u.pfull[s]);
      tma_bulk_g2s(base + kPkChunkBytes, pr.A1[p] + pk_chunk_off(0, kc, Kd), kPkChunkBytes, &u.pfull[s]);
      tma_bulk_g2s(base + 2 * kPkChunkBytes, pr.B[p] + pk_chunk_off(0, kc, Kd), kPkChunkBytes, &u.pfull[s]);
      u.fpend[s] = 1;
    };
    int next_load = 0, issued = 0;  // the same lazy refill as umma_pk_block_sub
    auto refill = [&](bool block) -> bool {
      while (next_load < nk) {
        const int j = next_load, sj = j % kStages2;
        if (j >= kStages2) {
          if (j - kStages2 >= issued) break;
          if (u.epend[sj]) {
            if (block) {
              if (!mbar_wait(&u.pempty[sj], u.eph[sj], st, timeout_ns, where)) return false;
            } else if (!mbar_test_wait(&u.pempty[sj], u.eph[sj])) {
              break;
            }
            u.eph[sj] ^= 1u;
            u.epend[sj] = 0;
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
      const int s = i % kStages2;
      if (!mbar_wait(&u.pfull[s], u.fph[s], st, timeout_ns, where)) {
        ok = false;
        break;
      }
      u.fph[s] ^= 1u;
      u.fpend[s] = 0;
      umma_fence_after();
      const uint32_t a0_hi = smem_u32(u.smem + s * kStage2Bytes), a0_lo = a0_hi + kUmmaTileBytes;
      const uint32_t a1_hi = a0_hi + kPkChunkBytes, a1_lo = a1_hi + kUmmaTileBytes;
      const uint32_t b_hi = a0_hi + 2 * kPkChunkBytes, b_lo = b_hi + kUmmaTileBytes;
      const int pair = i / nkp, h = pair >= kPairsPerAcc ? 1 : 0;
      const uint32_t d0 = u.tmem + (uint32_t)(h * kUmmaN), d1 = d0 + (uint32_t)(2 * kUmmaN);
      const bool first = (i % (kPairsPerAcc * nkp)) == 0;  // first chunk of these accumulators
#pragma unroll
      for (int ks = 0; ks < kUmmaKChunk / 8; ++ks) {
        const uint32_t o = ks * 32, acc = (!first || ks > 0) ? 1u : 0u;
        const uint64_t bh = umma_desc_sw128(b_hi + o), bl = umma_desc_sw128(b_lo + o);
        umma_tf32(d0, umma_desc_sw128(a0_hi + o), bh, acc);
        umma_tf32(d0, umma_desc_sw128(a0_hi + o), bl, 1u);
        umma_tf32(d0, umma_desc_sw128(a0_lo + o), bh, 1u);
        umma_tf32(d1, umma_desc_sw128(a1_hi + o), bh, acc);
        umma_tf32(d1, umma_desc_sw128(a1_hi + o), bl, 1u);
        umma_tf32(d1, umma_desc_sw128(a1_lo + o), bh, 1u);
      }
      umma_commit(&u.pempty[s]);
      u.epend[s] = 1;
      issued = i + 1;
      refill(false);
    }
    // every MMA must be complete before TMEM is read (and before the stages are reused)
    for (int i = 0; i < kStages2; ++i) {
      const int s = (nk + i) % kStages2;  // oldest outstanding commit first
      if (u.epend[s]) {
        if (ok) {
          ok = mbar_wait(&u.pempty[s], u.eph[s], st, timeout_ns, where);
        } else {
          mbar_drain(&u.pempty[s], u.eph[s], timeout_ns);
        }
        u.eph[s] ^= 1u;
        u.epend[s] = 0;
      }
    }
    if (!ok) {
      for (int s = 0; s < kStages2; ++s)
        if (u.fpend[s]) {
          mbar_drain(&u.pfull[s], u.fph[s], timeout_ns);
          u.fph[s] ^= 1u;
          u.fpend[s] = 0;
        }
      for (int s = 0; s < kStages2; ++s)
        if (u.epend[s]) {
          mbar_drain(&u.pempty[s], u.eph[s], timeout_ns);
          u.eph[s] ^= 1u;
          u.epend[s] = 0;
        }
    }
  }
  if (__syncthreads_or(!ok)) return false;
  const int nacc = pr.n > kPairsPerAcc ? 2 : 1;
  umma_epilogue<false>(u, C0, ldc, 0, 0, lower0, nacc, 0);
  umma_epilogue<false>(u, C1, ldc, 0, 0, false, nacc, (uint32_t)(2 * kUmmaN));
  fence_async_smem();  // generic smem traffic of the epilogues before the next bulk copies
  __syncthreads();
  return true;
}

// C[M x N] -= sum_p A_p B_p^T from packed operands (M, N multiples of 128; Kd of 32); lower skips the
// blocks above the diagonal and masks the diagonal blocks. kStore: C = sum_p A_p B_p^T instead (every
// entry written; lower must be false). False on a time-out.
template <bool kStore = false, int kProd = 3>
__device__ bool umma_pk_gemm_sub(UmmaState& u, double* C, int ldc, const PkPairs& pr, int Kd, int M, int N, bool lower,
                                 DevStatus* st, long long timeout_ns, long long where) {
  for (int m0 = 0; m0 < M; m0 += kUmmaM)
    for (int n0 = 0; n0 < N; n0 += kUmmaN) {
      if (lower && n0 > m0) continue;
      if (!umma_pk_block_sub<kStore, kProd>(u, C, ldc, pr, Kd, m0, n0, lower && n0 == m0, st, timeout_ns, where))
        return false;
    }
  return true;
}

// ---------------------------------------------------------------- the inverse of a diagonal tile

// X = L^{-1} in FP32 for a factored nb x nb diagonal tile (nb a multiple of 32, at most 128), written as
// the packed operand Op[r][k] = X[r][k] (upper triangle zero). It turns the TRSMs of the tile's block
// column (L_IJ = K_IJ X^T) and the diagonal-block solves of the covariance (V_Jc <- X V_Jc) into
// tensor-core products. Blocked by 32: warp d inverts diagonal block d (lane j solves column j), then
// block rows i = 1.. follow X_ij = -X_ii sum_{j <= k < i} L_ik X_kj.
// Ls: the factor's lower triangle in FP32 (leading dimension lds, upper triangle zero); Xs: zeroed
// FP32 workspace (leading dimension ldx).
__device__ void cta_inverse_compute(const float* Ls, int lds, float* Xs, int ldx, int nb);

// Packs an FP32 nb x nb matrix held in shared memory (leading dimension ldx) as the TF32 hi/lo operand
// (rows and columns beyond nb zero).
__device__ void cta_pack_tf32_f32(const float* Xs, int ldx, int nb, uint8_t* dst) {
  const int t = threadIdx.x;
  for (int kc = 0; kc < nb / kUmmaKChunk; ++kc) {
    uint8_t* hi = dst + pk_chunk_off(0, kc, nb);
    uint8_t* lo = hi + kUmmaTileBytes;
    for (int e = t; e < kUmmaM * 16; e += kThreads) {  // pairs (r, 2 kp), rows beyond nb are zero
      const int r = e >> 4, kp = e & 15;
      float f0 = 0.f, f1 = 0.f;
      if (r < nb) {
        f0 = Xs[r * ldx + kc * kUmmaKChunk + 2 * kp];
        f1 = Xs[r * ldx + kc * kUmmaKChunk + 2 * kp + 1];
      }
      const float h0 = tf32_rn(f0), h1 = tf32_rn(f1);
      const uint32_t off = sw128_offset(r, 2 * kp);
      *reinterpret_cast<float2*>(hi + off) = make_float2(h0, h1);
      *reinterpret_cast<float2*>(lo + off) = make_float2(tf32_rn(f0 - h0), tf32_rn(f1 - h1));
    }
  }
  fence_proxy_async_global();
  __syncthreads();
}

__device__ void cta_inverse_core(const float* Ls, int lds, float* Xs, int ldx, int nb, uint8_t* dst) {
  cta_inverse_compute(Ls, lds, Xs, ldx, nb);
  cta_pack_tf32_f32(Xs, ldx, nb, dst);
}

__device__ void cta_inverse_compute(const float* Ls, int lds, float* Xs, int ldx, int nb) {
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const int nblk = nb / 32;
  if (w < nblk) {  // diagonal blocks
    const int d0 = 32 * w;
    float x[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      float acc = (i == lane) ? 1.f : 0.f;
#pragma unroll
      for (int k = 0; k < i; ++k) acc = fmaf(-Ls[(d0 + i) * lds + d0 + k], x[k], acc);
      x[i] = acc / Ls[(d0 + i) * lds + d0 + i];
    }
#pragma unroll
    for (int i = 0; i < 32; ++i) Xs[(d0 + i) * ldx + d0 + lane] = x[i];
  }
  __syncthreads();
  for (int bi = 1; bi < nblk; ++bi) {
    // W_bj = sum_{bj <= k < bi} L_{bi,k} X_{k,bj}, parked in the (still zero) slots X_{bi,bj}
    for (int e = t; e < bi * 1024; e += kThreads) {
      const int bj = e >> 10, r = (e >> 5) & 31, c = e & 31;
      const float* lrow = Ls + (32 * bi + r) * lds;
      float acc = 0.f;
      for (int kk = 32 * bj; kk < 32 * bi; ++kk) acc = fmaf(lrow[kk], Xs[kk * ldx + 32 * bj + c], acc);
      Xs[(32 * bi + r) * ldx + 32 * bj + c] = acc;
    }
    __syncthreads();
    // X_{bi,bj} = -X_{bi,bi} W_bj (through registers: W is read in place)
    float res[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const int e = t + q * kThreads;
      res[q] = 0.f;
      if (e < bi * 1024) {
        const int bj = e >> 10, r = (e >> 5) & 31, c = e & 31;
        const float* xrow = Xs + (32 * bi + r) * ldx + 32 * bi;
        float acc = 0.f;
        for (int k = 0; k <= r; ++k) acc = fmaf(xrow[k], Xs[(32 * bi + k) * ldx + 32 * bj + c], acc);
        res[q] = -acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const int e = t + q * kThreads;
      if (e < bi * 1024) {
        const int bj = e >> 10, r = (e >> 5) & 31, c = e & 31;
        Xs[(32 * bi + r) * ldx + 32 * bj + c] = res[q];
      }
    }
    __syncthreads();
  }
}

// The inverse of a factored diagonal tile still held in shared memory as FP64 (sL, leading dimension
// nb + 1, the layout cta_potrf_smem leaves behind at the start of `smem`): converted to FP32 beside it
// (smem + nb (nb + 1) 8 bytes, leading dimension nb), then the FP32 workspace takes the FP64 tile's
// place. Needs nb (nb + 1) 8 + nb nb 4 bytes of shared memory; no global reads.
// The same FP32 inverse without the packing: returns the shared-memory FP32 result (leading dimension
// nb + 1, at the start of `smem`) for the caller to pack in the operand format it needs.
__device__ float* cta_inverse_f32_smem(uint8_t* smem, int nb) {
  const int t = threadIdx.x, ldl = nb + 1;
  const double* sL = reinterpret_cast<const double*>(smem);
  float* Ls = reinterpret_cast<float*>(smem + (size_t)nb * ldl * 8);
  float* Xs = reinterpret_cast<float*>(smem);
  for (int e = t; e < nb * nb; e += kThreads) {
    const int i = e / nb, j = e % nb;
    Ls[i * nb + j] = (j <= i) ? f64_to_f32_rn(sL[i * ldl + j]) : 0.f;
  }
  __syncthreads();  // the FP64 tile is dead from here: Xs reuses its bytes
  for (int e = t; e < nb * ldl; e += kThreads) Xs[e] = 0.f;
  __syncthreads();
  cta_inverse_compute(Ls, nb, Xs, ldl, nb);
  return Xs;
}

__device__ void cta_inverse_pack_smem(uint8_t* smem, int nb, uint8_t* dst) {
  const float* Xs = cta_inverse_f32_smem(smem, nb);
  cta_pack_tf32_f32(Xs, nb + 1, nb, dst);
}

}  // namespace gpk
