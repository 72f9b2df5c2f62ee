// Blocked triangular solves with the factor in FP32 (Eq. 2's two substitutions, L beta = b then
// L^T alpha = beta): the correction solves of the iteratively refined precision forms, whose factor is
// FP32-accurate. The diagonal-block solves are products with the stored inverses of the diagonal tiles.
// Right-hand side and solution are FP64 in memory; the tiles, the products and the sums are FP32.
//
// The solve is bound by its dependency chain (and by HBM: 4 bytes per value of L per sweep against one
// FMA). One persistent CTA per SM owns the tile rows I = c, c + G, c + 2G, ... (G CTAs). For the forward
// sweep it walks the tile columns J = 0, 1, ... in order and, for each owned row I, subtracts L_IJ beta_J
// from that row's running right-hand side (kept in shared memory) as soon as beta_J is published. After
// tile (I, I-2) it forms y_I = L_II^-1 (that right-hand side); the chain's step of row I is then the
// single product beta_I = y_I - M_I beta_{I-1}, M_I = L_II^-1 L_{I,I-1} precomputed once per factor
// (chain_mats_kernel), so the wait for beta_{I-1} is followed by one tile product only. The backward
// sweep mirrors this: alpha_J = y_J - P_J^T alpha_{J+1}, P_J = L_{J+1,J} L_JJ^-1, y_J = L_JJ^-T (beta_J -
// sum_{I > J+1} L_IJ^T alpha_I). Blocks are published strictly in order (each one waits for its
// predecessor), so one counter per sweep carries every dependency.
//
// A CTA's tiles and inverses stream through shared memory as 64 KB row chunks moved by cp.async.bulk,
// several stages ahead of the arithmetic and independent of the dependency waits (the factor does not
// change), so that a CTA waiting for its next vector block already holds the tiles it will multiply.
// Every wait is bounded: a CTA that gives up raises GP_ERR_TIMEOUT, waits (bounded) for its own copies
// in flight and returns.
#include "kernels.h"
#include "bulk.cuh"

namespace gpk {

namespace {

constexpr int kTsThreads = 512;
constexpr int kTsChunkBytes = 64 * 1024;
constexpr int kTsMaxStages = 4;
constexpr int kTsSmemLimit = 226 * 1024;  // dynamic shared memory cap (227 KB less the static part)

// Item kinds. Forward (kind < 4): a tile product L_IJ beta_J (kFTile); the chain's step beta_I = y_I -
// M_I beta_{I-1} with M_I = L_II^-1 L_{I,I-1} (kFFinal); y_I = L_II^-1 (the right-hand side less every
// tile product but the last) (kFPrep); beta_0 = L_00^-1 b_0 (kFDiag). Backward mirrors them with
// transposed products: L_IJ^T alpha_I, alpha_J = y_J - P_J^T alpha_{J+1} with P_J = L_{J+1,J} L_JJ^-1,
// y_J = L_JJ^-T (...), alpha_{Mt-1} = L^-T beta_{Mt-1}.
enum : int { kFTile = 0, kFFinal = 1, kFPrep = 2, kFDiag = 3, kBTile = 4, kBFinal = 5, kBPrep = 6, kBDiag = 7 };

struct TsItem {
  int kind, I, J;  // the final steps carry (I, I - 1); the diagonal items (blk, blk)
};

// The sequence of work items of CTA c (rows c, c + G, ... owned), identical for its producer thread and
// its consumers. Forward: beta_0 (owner of row 0), y_1 (owner of row 1); then per column J the chain's
// step of row J + 1 (its owner) first, then the owned rows I >= J + 2 in ascending order, y_I right after
// tile (I, I - 2), its last tile before the chain reaches it. Backward: alpha_{Mt-1}, y_{Mt-2}; then per row
// I = Mt-1, ..., 1 the chain's step of block I - 1 first, then the owned blocks J <= I - 2 in descending
// order, y_J right after tile (J + 2, J). The chain's steps wait only for the previous block; every
// other product of a block is done a step ahead.
struct TsIter {
  int phase = 0;  // 0 forward start, 1 forward columns, 2 backward start, 3 backward rows, 4 done
  int col = 0;    // forward: tile column J; backward: tile row I
  int k = 0;      // next owned-row index within the column / row
  int stage = 0;  // position within a start list, or 0/1 before/after a column's chain step
  int pend = -1;  // y block to emit next (-1: none)
};

__host__ __device__ __forceinline__ bool ts_own(int r, int c, int G, int Mt) { return r >= c && r < Mt && (r - c) % G == 0; }
// first owned row index k with c + k G >= J + 2; last owned block index with c + k G <= I - 2 (-1: none)
__host__ __device__ __forceinline__ int ts_kfirst(int J, int c, int G) { return J + 2 <= c ? 0 : (J + 2 - c + G - 1) / G; }
__host__ __device__ __forceinline__ int ts_klast(int I, int c, int G) { return I - 2 < c ? -1 : (I - 2 - c) / G; }

__host__ __device__ bool ts_next(TsIter& s, int c, int G, int Mt, TsItem& it) {
  const int last = c + ((Mt - 1 - c) / G) * G;  // the CTA's last row
  for (;;) {
    if (s.pend >= 0) {
      it = TsItem{s.phase < 2 ? kFPrep : kBPrep, s.pend, s.pend};
      s.pend = -1;
      return true;
    }
    switch (s.phase) {
      case 0:
        if (s.stage == 0) {
          s.stage = 1;
          if (c == 0) {
            it = TsItem{kFDiag, 0, 0};
            return true;
          }
        }
        if (s.stage == 1) {
          s.stage = 2;
          if (Mt > 1 && ts_own(1, c, G, Mt)) {
            it = TsItem{kFPrep, 1, 1};
            return true;
          }
        }
        s.phase = 1;
        s.col = 0;
        s.stage = 0;
        continue;
      case 1: {
        if (s.col > Mt - 2 || s.col >= last) {  // no owned row below this column's diagonal
          s.phase = 2;
          s.stage = 0;
          continue;
        }
        if (s.stage == 0) {
          s.stage = 1;
          s.k = ts_kfirst(s.col, c, G);
          if (ts_own(s.col + 1, c, G, Mt)) {
            it = TsItem{kFFinal, s.col + 1, s.col};
            return true;
          }
        }
        const int I = c + s.k * G;
        if (I < Mt) {
          ++s.k;
          if (I == s.col + 2) s.pend = I;
          it = TsItem{kFTile, I, s.col};
          return true;
        }
        ++s.col;
        s.stage = 0;
        continue;
      }
      case 2:
        if (s.stage == 0) {
          s.stage = 1;
          if (ts_own(Mt - 1, c, G, Mt)) {
            it = TsItem{kBDiag, Mt - 1, Mt - 1};
            return true;
          }
        }
        if (s.stage == 1) {
          s.stage = 2;
          if (Mt > 1 && ts_own(Mt - 2, c, G, Mt)) {
            it = TsItem{kBPrep, Mt - 2, Mt - 2};
            return true;
          }
        }
        s.phase = 3;
        s.col = Mt - 1;
        s.stage = 0;
        continue;
      case 3: {
        if (s.col <= c) {  // rows at or above the CTA's first block hold none of its items
          s.phase = 4;
          return false;
        }
        if (s.stage == 0) {
          s.stage = 1;
          s.k = ts_klast(s.col, c, G);
          if (ts_own(s.col - 1, c, G, Mt)) {
            it = TsItem{kBFinal, s.col, s.col - 1};
            return true;
          }
        }
        if (s.k >= 0) {
          const int J = c + s.k * G;
          --s.k;
          if (J == s.col - 2) s.pend = J;
          it = TsItem{kBTile, s.col, J};
          return true;
        }
        --s.col;
        s.stage = 0;
        continue;
      }
      default:
        return false;
    }
  }
}

struct TsArgs {
  const float* Lt;     // packed lower tiles of L (FP32), tile (I, J) at (I(I+1)/2 + J) T^2, row-major
  const float* Linv;   // Mt inverses of the diagonal tiles (FP32), T x T row-major (upper triangle not read)
  const float* M;      // M_I = L_II^-1 L_{I,I-1} at I T^2 (I >= 1), T x T row-major
  const float* P;      // P_J = L_{J+1,J} L_JJ^-1 at J T^2 (J <= Mt - 2), T x T row-major
  double* b;           // Mt*T: right-hand side on entry, alpha on exit
  double* xb;          // Mt*T: beta (forward result)
  int* front;          // [0]: forward blocks published, [1]: backward blocks published (zero on entry)
  int T, Mt, CR, S;    // tile edge, tile rows, rows per chunk, pipeline stages
  DevStatus* st;
  long long timeout_ns;
  int withhold;        // test hook: forward block whose completion is never published (-1: off)
  long long* trace;    // optional: per item {CTA, t_start, t_ready, t_done} (%globaltimer ns)
  int4* trace_items;   // with trace: per item {kind (TASK_FGEMV/FSOLVE/BGEMV/BSOLVE), I, J, 0}
  unsigned long long* trace_next;  // with trace: slot counter (zero on entry)
};

__device__ __forceinline__ size_t ts_tri(long long I, long long J) { return (size_t)(I * (I + 1) / 2 + J); }

__device__ __forceinline__ const float* ts_chunk_src(const TsArgs& a, const TsItem& it, int ch) {
  const size_t TT = (size_t)a.T * a.T, off = (size_t)ch * a.CR * a.T;
  switch (it.kind) {
    case kFFinal: return a.M + (size_t)it.I * TT + off;
    case kBFinal: return a.P + (size_t)it.J * TT + off;
    case kFTile:
    case kBTile: return a.Lt + ts_tri(it.I, it.J) * TT + off;
    default: return a.Linv + (size_t)it.I * TT + off;  // the diagonal items: (blk, blk)
  }
}

// Thread 0: bounded wait until *p >= target. Returns the value seen (>= target), or -1 after a time-out
// (GP_ERR_TIMEOUT raised, info = where) or when another CTA has aborted. Every waiting CTA polls the same
// counter: only the wait on the dependency chain (urgent) polls at a short fixed interval; the others
// back off to about a microsecond, which keeps the counter's L2 slice free for the tile copies.
__device__ int ts_wait(const int* p, int target, bool urgent, DevStatus* st, long long timeout_ns,
                       long long where) {
  int v = ld_acquire(p);
  if (v >= target) return v;
  const uint64_t t0 = globaltimer();
  unsigned ns = 64;
  while (true) {
    if (ld_relaxed(&st->abort)) return -1;
    v = ld_acquire(p);
    if (v >= target) return v;
    if ((long long)(globaltimer() - t0) > timeout_ns) {
      raise_error(st, GP_ERR_TIMEOUT, where);
      return -1;
    }
    __nanosleep(ns);
    if (!urgent && ns < 1024) ns <<= 1;
  }
}

// Sums over the 32 lanes of a warp of R per-lane values at once (R = 4 or 8): halving exchanges, after
// which lane l holds the total of value row_of(l) = the high log2(R) bits of l's top five bits, and
// lanes with (l & (32 / R - 1)) == 0 are its holders.
template <int R>
__device__ __forceinline__ float warp_sum_rows(float (&v)[R], int lane) {
#pragma unroll
  for (int h = R / 2, o = 16; h >= 1; h /= 2, o /= 2) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float send = up ? v[i] : v[i + h];
      const float keep = up ? v[i + h] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  float x = v[0];
#pragma unroll
  for (int o = 16 / R; o >= 1; o /= 2) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
// The value index whose total a lane holds after warp_sum_rows<R> (lane bits 4, 3[, 2], high first).
template <int R>
__device__ __forceinline__ int warp_sum_row_of(int lane) {
  return R == 8 ? ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)
                : ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);
}

// Dynamic shared memory: S chunk stages, the owned blocks' running sums (nown x T floats), the vector
// block being multiplied (T floats), the column-form reduction buffer (2048 floats), S mbarriers.
// T = 128 (one 128-row chunk per tile) or 256 (four 64-row chunks per tile); kR = rows per warp per
// chunk in the row form (CR / 16).
template <int T>
__global__ void __launch_bounds__(kTsThreads, 1) trsv32_kernel(TsArgs a) {
  constexpr int CR = kTsChunkBytes / (4 * T);   // rows per chunk: 128 or 64
  constexpr int nch = T / CR;                   // chunks per tile: 1 or 4
  constexpr int kR = CR / 16;                   // rows per warp per chunk (row form): 8 or 4
  constexpr int K4 = T / 128;                   // float4 per lane per row (row form): 1 or 2
  constexpr int NC4 = T / 4, NG = kTsThreads / NC4, RG = CR / NG;  // column form: groups, rows per group
  extern __shared__ __align__(128) uint8_t ts_smem[];
  __shared__ int s_fail;
  const int S = a.S, Mt = a.Mt;
  const int c = blockIdx.x, G = gridDim.x, t = threadIdx.x, w = t / 32, lane = t % 32;
  const uint32_t chunk_bytes = kTsChunkBytes;
  const int nown = (Mt - 1 - c) / G + 1;
  float* acc = reinterpret_cast<float*>(ts_smem + (size_t)S * chunk_bytes);
  float* xs = acc + (size_t)nown * T;
  float* red = xs + T;
  uint64_t* full = reinterpret_cast<uint64_t*>(red + 2048);
  // running right-hand sides of the owned blocks: b_I, minus the tile products as they arrive
  for (int e = t; e < nown * T; e += kTsThreads) acc[e] = (float)a.b[(size_t)(c + (e / T) * G) * T + e % T];
  if (t == 0) {
    for (int s = 0; s < S; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  __syncthreads();

  // producer (thread 0): the next chunk of the item sequence into stage issued % S
  TsIter pit;
  TsItem pitem{0, 0, 0};
  int pch = nch, issued = 0;
  auto issue = [&]() {
    if (pch >= nch) {
      if (!ts_next(pit, c, G, Mt, pitem)) return;
      pch = 0;
    }
    const int s = issued % S;
    fence_async_smem();
    mbar_expect_tx(&full[s], chunk_bytes);
    tma_bulk_g2s(ts_smem + (size_t)s * chunk_bytes, ts_chunk_src(a, pitem, pch), chunk_bytes, &full[s]);
    ++pch;
    ++issued;
  };
  if (t == 0)
    for (int q = 0; q < S; ++q) issue();

  const int c4 = t % NC4, g = t / NC4;  // column form: float4 column block and row group of this thread
  TsIter it_s;
  TsItem it{0, 0, 0};
  int i = 0;            // chunks consumed
  long long xkey = -1;  // vector block held in xs (forward J, or Mt + backward I); -1: none
  int known_f = 0, known_b = 0;  // thread 0: published counts already seen
  bool fail = false;
  long long t_start = 0, t_ready = 0;
  while (ts_next(it_s, c, G, Mt, it)) {
    if (a.trace && t == 0) t_start = (long long)globaltimer();
    const bool fwd = it.kind < kBTile;
    // diagonal items: the product with L_blk^-1 (or its transpose) of the running right-hand side
    const bool diag = it.kind == kFDiag || it.kind == kFPrep || it.kind == kBDiag || it.kind == kBPrep;
    const bool final = it.kind == kFFinal || it.kind == kBFinal;  // the chain's steps
    const bool publish = final || it.kind == kFDiag || it.kind == kBDiag;
    const int blk = fwd ? it.I : it.J;  // the owned block this item contributes to
    float* accb = acc + (size_t)((blk - c) / G) * T;
    if (!diag) {
      const long long key = fwd ? it.J : Mt + it.I;
      if (key != xkey) {
        if (t == 0) {
          const int need = fwd ? it.J + 1 : Mt - it.I;
          int& known = fwd ? known_f : known_b;
          if (known < need) {
            const int v = ts_wait(a.front + (fwd ? 0 : 1), need, final, a.st, a.timeout_ns, fwd ? it.J : it.I);
            if (v < 0)
              s_fail = 1;
            else
              known = v;
          }
        }
        __syncthreads();
        if (s_fail) {
          fail = true;
          break;
        }
        const double* src = fwd ? a.xb + (size_t)it.J * T : a.b + (size_t)it.I * T;
        for (int e = t; e < T; e += kTsThreads) xs[e] = (float)ldcg(src + e);
        xkey = key;
        __syncthreads();
      }
    } else {
      // right-hand side of the diagonal block: the running one (b_I or beta_J minus the tile products)
      for (int e = t; e < T; e += kTsThreads) xs[e] = accb[e];
      xkey = -1;
      __syncthreads();
    }
    if (a.trace && t == 0) t_ready = (long long)globaltimer();
    float4 xr[K4];  // row form: this lane's x columns
    if (fwd) {
#pragma unroll
      for (int k = 0; k < K4; ++k) xr[k] = reinterpret_cast<const float4*>(xs)[lane + 32 * k];
    }
    float4 pc = make_float4(0.f, 0.f, 0.f, 0.f);  // column form: partial sums of 4 columns over the item
    for (int ch = 0; ch < nch; ++ch) {
      const int s = i % S;
      if (!mbar_wait(&full[s], (uint32_t)(i / S) & 1u, a.st, a.timeout_ns, blk)) s_fail = 1;
      const float* L = reinterpret_cast<const float*>(ts_smem + (size_t)s * chunk_bytes);
      const int r0 = ch * CR;
      if (fwd) {
        float v[kR];
#pragma unroll
        for (int q = 0; q < kR; ++q) {
          const int rl = w + 16 * q, r = r0 + rl;
          float sum = 0.f;
#pragma unroll
          for (int k = 0; k < K4; ++k) {
            const int col = 4 * (lane + 32 * k);
            const float4 l = reinterpret_cast<const float4*>(L + (size_t)rl * T)[lane + 32 * k];
            if (!diag || col + 3 <= r) {
              sum = fmaf(l.x, xr[k].x, sum);
              sum = fmaf(l.y, xr[k].y, sum);
              sum = fmaf(l.z, xr[k].z, sum);
              sum = fmaf(l.w, xr[k].w, sum);
            } else {
              if (col <= r) sum = fmaf(l.x, xr[k].x, sum);
              if (col + 1 <= r) sum = fmaf(l.y, xr[k].y, sum);
              if (col + 2 <= r) sum = fmaf(l.z, xr[k].z, sum);
            }
          }
          v[q] = sum;
        }
        const float tot = warp_sum_rows<kR>(v, lane);
        if ((lane & (32 / kR - 1)) == 0) {
          const int r = r0 + w + 16 * warp_sum_row_of<kR>(lane);
          if (it.kind == kFTile) {
            accb[r] -= tot;
          } else if (it.kind == kFPrep) {
            accb[r] = tot;  // y_I, the chain step's starting value
          } else {  // beta (kFDiag: the product itself; kFFinal: y_I - M_I beta_{I-1})
            const float beta = it.kind == kFDiag ? tot : accb[r] - tot;
            a.xb[(size_t)blk * T + r] = (double)beta;
            accb[r] = beta;  // the backward sweep's right-hand side of this block starts at beta
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < RG; ++q) {
          const int rl = g + NG * q, r = r0 + rl;
          const float4 l = reinterpret_cast<const float4*>(L + (size_t)rl * T)[c4];
          const float x = xs[r];
          const int col = 4 * c4;
          if (!diag || r >= col + 3) {
            pc.x = fmaf(l.x, x, pc.x);
            pc.y = fmaf(l.y, x, pc.y);
            pc.z = fmaf(l.z, x, pc.z);
            pc.w = fmaf(l.w, x, pc.w);
          } else {
            if (r >= col) pc.x = fmaf(l.x, x, pc.x);
            if (r >= col + 1) pc.y = fmaf(l.y, x, pc.y);
            if (r >= col + 2) pc.z = fmaf(l.z, x, pc.z);
          }
        }
      }
      __syncthreads();  // stage s read by every thread
      if (s_fail) {
        fail = true;
        break;
      }
      ++i;
      if (t == 0) issue();
    }
    if (fail) break;
    if (!fwd) {
      reinterpret_cast<float4*>(red + (size_t)g * T)[c4] = pc;
      __syncthreads();
      if (t < T) {
        float sum = 0.f;
#pragma unroll
        for (int q = 0; q < NG; ++q) sum += red[(size_t)q * T + t];
        if (it.kind == kBTile) {
          accb[t] -= sum;
        } else if (it.kind == kBPrep) {
          accb[t] = sum;  // y_J
        } else {  // alpha (kBDiag: the product itself; kBFinal: y_J - P_J^T alpha_{J+1})
          const float alpha = it.kind == kBDiag ? sum : accb[t] - sum;
          accb[t] = alpha;
          a.b[(size_t)blk * T + t] = (double)alpha;
        }
      }
      __syncthreads();
    }
    if (publish) {
      const bool withheld = fwd && blk == a.withhold;
      __syncthreads();
      if (t == 0 && !withheld) {
        __threadfence();
        st_release(a.front + (fwd ? 0 : 1), fwd ? blk + 1 : Mt - blk);
      }
    }
    if (a.trace && t == 0) {
      const unsigned long long slot = atomicAdd(a.trace_next, 1ull);
      // chain steps and the first block as FSOLVE/BSOLVE, the y products as FSOLVE_C/BSOLVE_C
      const int kinds[8] = {TASK_FGEMV, TASK_FSOLVE, TASK_FSOLVE_C, TASK_FSOLVE,
                            TASK_BGEMV, TASK_BSOLVE, TASK_BSOLVE_C, TASK_BSOLVE};
      a.trace_items[slot] = make_int4(kinds[it.kind], it.I, it.J, 0);
      long long* rec = a.trace + 4 * slot;
      rec[0] = c;
      rec[1] = t_start;
      rec[2] = t_ready;
      rec[3] = (long long)globaltimer();
    }
  }
  // after a failure: wait (bounded) for this CTA's copies still in flight before leaving
  if (fail && t == 0)
    for (int q = i; q < issued; ++q) mbar_wait(&full[q % S], (uint32_t)(q / S) & 1u, a.st, a.timeout_ns, -1);
}

// The chain's matrices, once per factor (FP32 products with FP32 sums): blockIdx.y = 0 writes
// M_I = L_II^-1 L_{I,I-1} for I = blockIdx.x >= 1, blockIdx.y = 1 writes P_J = L_{J+1,J} L_JJ^-1 for
// J = blockIdx.x <= Mt - 2. The inverses' upper triangles are masked (not read as data). T = 128 or 256:
// four (or sixteen) 128 x 128 output quadrants, each thread an 8 x 8 block of one quadrant, k in chunks
// of 16 staged in shared memory.
template <int T>
__global__ void __launch_bounds__(256) chain_mats_kernel(const float* __restrict__ Lt, const float* __restrict__ Linv,
                                                         float* __restrict__ M, float* __restrict__ P, int Mt) {
  __shared__ float As[128][17];
  __shared__ float Bs[16][128];
  const int b = blockIdx.x, t = threadIdx.x, tx = t % 16, ty = t / 16;
  const bool isM = blockIdx.y == 0;
  if (isM ? b < 1 : b > Mt - 2) return;
  const size_t TT = (size_t)T * T;
  // A (row-major T x T) and B (row-major T x T); amask: A lower triangular, bmask: B lower triangular
  const float* A = isM ? Linv + (size_t)b * TT : Lt + ts_tri(b + 1, b) * TT;
  const float* B = isM ? Lt + ts_tri(b, b - 1) * TT : Linv + (size_t)b * TT;
  float* C = (isM ? M : P) + (size_t)b * TT;
  for (int q0 = 0; q0 < T; q0 += 128)
    for (int q1 = 0; q1 < T; q1 += 128) {
      float acc[8][8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = 0.f;
      for (int k0 = 0; k0 < T; k0 += 16) {
        for (int e = t; e < 128 * 16; e += 256) {
          const int r = e / 16, k = e % 16, gr = q0 + r, gk = k0 + k;
          As[r][k] = (!isM || gk <= gr) ? A[(size_t)gr * T + gk] : 0.f;
          const int kb = e / 128, cb = e % 128, gkb = k0 + kb, gc = q1 + cb;
          Bs[kb][cb] = (isM || gc <= gkb) ? B[(size_t)gkb * T + gc] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          float av[8], bv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) av[u] = As[ty * 8 + u][k];
#pragma unroll
          for (int v = 0; v < 8; ++v) bv[v] = Bs[k][tx * 8 + v];
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) C[(size_t)(q0 + ty * 8 + u) * T + q1 + tx * 8 + v] = acc[u][v];
    }
}

}  // namespace

long long trsv32_items(int Mt, int G, int c, int* out, long long cap) {
  if (Mt < 1 || G < 1 || c < 0 || c >= (G < Mt ? G : Mt)) return -1;
  G = G < Mt ? G : Mt;
  TsIter s;
  TsItem it{0, 0, 0};
  long long n = 0;
  while (ts_next(s, c, G, Mt, it)) {
    if (out && n < cap) {
      out[3 * n] = it.kind;
      out[3 * n + 1] = it.I;
      out[3 * n + 2] = it.J;
    }
    ++n;
  }
  return n;
}

int trsv32_smem_bytes(int T, int Mt, int grid, int* stages) {
  if ((T != 128 && T != 256) || grid < 1 || Mt < 1) return -1;
  const int G = grid < Mt ? grid : Mt;
  const int nown = (Mt + G - 1) / G;
  const size_t fixed = ((size_t)nown * T + T + 2048) * sizeof(float) + kTsMaxStages * sizeof(uint64_t);
  if (fixed + 2 * (size_t)kTsChunkBytes > (size_t)kTsSmemLimit) return -1;
  int s = (int)(((size_t)kTsSmemLimit - fixed) / kTsChunkBytes);
  s = s > kTsMaxStages ? kTsMaxStages : s;
  *stages = s;
  return (int)((size_t)s * kTsChunkBytes + fixed);
}

cudaError_t launch_chain_mats(const float* Lt, const float* Linv, float* M, float* P, int T, int Mt, cudaStream_t stream) {
  if (Mt < 2) return cudaSuccess;
  const dim3 grid((unsigned)Mt, 2);
  if (T == 128)
    chain_mats_kernel<128><<<grid, 256, 0, stream>>>(Lt, Linv, M, P, Mt);
  else if (T == 256)
    chain_mats_kernel<256><<<grid, 256, 0, stream>>>(Lt, Linv, M, P, Mt);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_trsv32(const float* Lt, const float* Linv, const float* M, const float* P, double* b, double* xb,
                          int* front, int T, int Mt, int grid, DevStatus* st, long long timeout_ns, int withhold,
                          long long* trace, int4* trace_items, cudaStream_t stream) {
  int S = 0;
  const int smem = trsv32_smem_bytes(T, Mt, grid, &S);
  if (smem < 0) return cudaErrorInvalidValue;
  TsArgs a;
  a.Lt = Lt;
  a.Linv = Linv;
  a.M = M;
  a.P = P;
  a.b = b;
  a.xb = xb;
  a.front = front;
  a.T = T;
  a.Mt = Mt;
  a.CR = kTsChunkBytes / (4 * T);
  a.S = S;
  a.st = st;
  a.timeout_ns = timeout_ns;
  a.withhold = withhold;
  a.trace = trace;
  a.trace_items = trace_items;
  a.trace_next = &st->next_task;
  const int G = grid < Mt ? grid : Mt;
  if (T == 128) {
    const cudaError_t e = cudaFuncSetAttribute(trsv32_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    trsv32_kernel<128><<<G, kTsThreads, smem, stream>>>(a);
  } else {
    const cudaError_t e = cudaFuncSetAttribute(trsv32_kernel<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    trsv32_kernel<256><<<G, kTsThreads, smem, stream>>>(a);
  }
  return cudaGetLastError();
}

// FP32 copies of the factor for the correction solves: dst[i] = src[i] rounded to nearest FP32, n values
// (src 16-byte aligned). The conversion runs on the integer pipe (f64_to_f32_rn), so the pass is bound by
// HBM, not by FP64 issue.
__global__ void to_f32_kernel(const double* __restrict__ src, float* __restrict__ dst, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x * 2;
  for (long long i = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x); i < n; i += stride) {
    if (i + 1 < n) {
      const double2 v = __ldcs(reinterpret_cast<const double2*>(src + i));
      *reinterpret_cast<float2*>(dst + i) = make_float2(f64_to_f32_rn(v.x), f64_to_f32_rn(v.y));
    } else {
      dst[i] = f64_to_f32_rn(src[i]);
    }
  }
}

cudaError_t launch_to_f32(const double* src, float* dst, long long n, int sms, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  to_f32_kernel<<<sms * 8, 256, 0, stream>>>(src, dst, n);
  return cudaGetLastError();
}

}  // namespace gpk
