// Host-side task graphs of the tiled algorithms and their dispatch order.
#pragma once
#include <cstdint>
#include <vector>

namespace gpk {

struct Task4 {
  int32_t kind, p, q, r;
};

// Relative speed model used to order tasks (seconds per flop of one CTA, plus a fixed overhead).
struct CostModel {
  double sec_per_flop = 1.0 / 3.9e9;     // FP64 work: one CTA on a shared SM, FP64 FFMA
  double sec_per_flop32 = 1.0 / 3.0e11;  // FP32 work (mixed mode): one CTA per SM
  bool mixed = false;                    // trailing updates / later panel TRSMs / V solve in FP32
  int update_group = 1;                  // trailing updates per task for tiles off the critical path
  // Mixed mode on the tensor cores (packed operands, T a multiple of 128): task costs measured on
  // GB300 at T = 128 (per-task trace at n = 32768) replace the flop-rate model, scaled by (T/128)^3
  // for the FP64 work and (T/128)^2 for the memory-bound products.
  bool tensor_cores = false;
  // Grouped updates of tiles (I, K) and (I + 1, K) as one task (TASK_UPD2; tile edge 128 on the tensor
  // cores): the shared L_KJ is copied once for both, a quarter fewer operand bytes requested per product.
  bool pair_rows = false;
  // > 0: the grouped updates are ordered with operand locality (LocalityKeys, this eps).
  double locality_eps = 0.0;
  // Task costs of the tensor-core path at T = 128 (seconds; measured for the 3xTF32 form, per-task trace
  // at n = 32768): POTRF with the diagonal-tile inverse, first-column FP64 TRSM, tensor-core TRSM, one
  // column of a grouped update (off the diagonal / on it), V solve, one column of a grouped V/W product.
  // Other precision forms set their own (api.cu).
  double tc_potrf = 403e-6, tc_trsm0 = 440e-6, tc_trsm = 30e-6, tc_gemm = 6.6e-6, tc_syrk = 5.0e-6;
  double tc_vtrsm = 35e-6, tc_vgemm = 5.5e-6;
  double potrf_eff = 0.5, trsm_eff = 0.8, gemm_eff = 0.97, vec_eff = 0.3;
  double task_overhead = 3e-6;
  // Tile-algorithm variant of the Cholesky graph (Sec. 3.2 names all three): 0 = right-looking (each
  // column's updates applied as soon as the column is factored, dispatched by longest remaining path);
  // 1 = left-looking and 2 = top-looking (every tile's updates from all earlier columns fused into one
  // task run just before the tile is factored, dispatched column by column / row by row).
  int variant = 0;
};

// Operand locality for list_schedule: per task the keys of the packed left (a) and right (b) operand
// groups it reads (-1: none). After starting a task, the scheduler starts next a ready task that
// shares the last started task's a or b key -- the best-ranked such task -- as long as its bottom
// level is within a factor (1 - eps) of the best ready task's; otherwise the best ready task. Tasks
// started back to back run side by side on the persistent kernel's CTAs, so the shared operand is
// read from HBM once and from L2 by the others.
struct LocalityKeys {
  std::vector<long long> a, b;
  double eps = 0.0;
};

// Tasks of the tiled right-looking Cholesky (Fig. 1) on Mt x Mt tiles of edge T, in the order a
// simulated list scheduler with `workers` CTAs would start them (priority: longest remaining
// path). The order is a topological order of the dependency DAG.
std::vector<Task4> cholesky_tasks(int Mt, int T, int workers, const CostModel& cm);
// Tasks of L V = B (B: Mt x Mc tiles) followed by S -= V^T V on the Mc x Mc lower tiles.
std::vector<Task4> cov_tasks(int Mt, int Mc, int T, int workers, const CostModel& cm, bool with_w = true);
// Tasks of the reverse sweep of the tiled Cholesky (adjoint of Fig. 1), columns J = Mt-1 .. 0.
std::vector<Task4> cholesky_adjoint_tasks(int Mt, int T, int workers, const CostModel& cm);
// Tasks of L beta = y then L^T alpha = beta on Mt tiles, vector chunks of 32 rows.
std::vector<Task4> mean_tasks(int Mt, int T, int workers, const CostModel& cm);

// One dispatch order for a batch of independent GPs, each running its tiled Cholesky, the two
// substitutions of the mean solve and the covariance solve (each solve task depending on the factor
// tiles it reads). Task kinds carry the GP index in their high bits (kind | g << 5).
struct BatchGp {
  int Mt, Mc, T;
};
// order 0: every ready task ranked by its bottom level (longest remaining cost path) across all GPs;
// order 1: GPs ranked by their total work (largest first), bottom level within a GP.
std::vector<Task4> batch_tasks(const std::vector<BatchGp>& gps, bool want_cov, int workers, const CostModel& cm,
                               int order = 0);

// Generic list scheduling: returns the start order of tasks with the given costs and
// predecessor lists, simulated on `workers` identical workers. Ready tasks are ranked by
// (group_key, bottom level) when group_key is given, else by bottom level alone; with loc, a ready
// task sharing an operand with the last started one may go first (LocalityKeys).
std::vector<int> list_schedule(const std::vector<double>& cost, const std::vector<std::vector<int>>& preds,
                               int workers, const std::vector<double>* group_key = nullptr,
                               const LocalityKeys* loc = nullptr);

}  // namespace gpk
