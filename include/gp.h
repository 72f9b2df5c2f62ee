/* gp.h -- C ABI of the GB300 exact-GP prediction library (libgp.so).
 *
 * What it computes (arxiv 2602.19683, Sec. 3.1-3.2):
 *   K      = K_{X,X}   with K_ij = v*exp(-|x_i-x_j|^2/(2 l^2)) + [i==j]*s2        (Eq. 1)
 *   K      = L L^T     by the tiled right-looking Cholesky of Sec. 3.2 (Fig. 1): POTRF on the
 *                      diagonal tile, TRSM on the tiles below it, SYRK/GEMM on the trailing tiles
 *   mean   = K_{Xs,X} K^{-1} y, via L beta = y, L^T alpha = beta, mean = K_{Xs,X} alpha  (Eq. 2)
 *   cov    = K_{Xs,Xs} - K_{Xs,X} K^{-1} K_{X,Xs}, via L V = K_{X,Xs}, cov = K_{Xs,Xs} - V^T V (Eq. 3)
 *   nlml   = 1/2 y^T alpha + sum_i log L_ii + n/2 log(2 pi) and its gradient w.r.t. (l, v, s2)
 *            (Rasmussen & Williams 2006, Eqs. 2.30 and 5.9; the paper cites them for the kernel and
 *            says hyperparameters are normally optimised, Sec. 3.1)
 *
 * Lengthscale convention: the paper prints the exponent as -(1/(2 l)) sum_d (x_id - x_jd)^2. This
 * library uses the textbook -|x_i - x_j|^2 / (2 l^2); pass l = sqrt(paper's l). At the paper's l = 1
 * both are the same kernel.
 *
 * Conventions for every entry point:
 *   - Returns gp_status (0 = GP_OK). Argument errors are detected synchronously on the host.
 *   - Work is enqueued on the context's CUDA stream and is ASYNCHRONOUS unless the entry point says
 *     otherwise. Device-side failures (not positive definite, time-out of a bounded device wait)
 *     are written to a device status word; gp_sync() waits for the stream and returns them.
 *   - All numeric arrays are caller-owned DEVICE pointers to contiguous row-major FP64 data:
 *     X is n x D, Xs is m x D, y is n, mean is m, cov is m x m. The library never frees them.
 *   - Host pointers appear only for scalar outputs (documented as "host").
 *   - The library owns its workspace (tile storage, packed panels, task lists, counters) inside the
 *     context and the factor objects, allocated with cudaMalloc when they are created or grown.
 *   - Nothing traps: every device-side wait is bounded by cfg.timeout_ns and ends with
 *     GP_ERR_TIMEOUT instead of hanging.
 *   - Input values are checked on the device: a NaN or infinity in X (gp_assemble), y or Xs
 *     (gp_predict_mean), or Xs (gp_predict_full_cov, gp_predict_var) raises GP_ERR_NONFINITE in the
 *     status word with info = 1-based flat index of the first such entry (for gp_predict_mean: y's
 *     n entries first, then Xs's m*D). The first device error of a context stops every later
 *     persistent-kernel launch on it (their tasks are skipped) until gp_sync returns and clears it.
 *     The batched entry points and gp_predict_mean_noalloc do not check input values.
 */
#ifndef GP_H_
#define GP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t gp_status;
enum {
  GP_OK = 0,
  GP_ERR_INVALID_ARG = 1,     /* bad size, null pointer, unsupported option                     */
  GP_ERR_NOT_PD = 2,          /* a Cholesky pivot was not positive; info = 1-based column       */
  GP_ERR_NONFINITE = 3,       /* NaN/Inf in an input (a NaN pivot reports GP_ERR_NOT_PD)        */
  GP_ERR_OOM = 4,             /* cudaMalloc failed                                               */
  GP_ERR_CUDA = 5,            /* another CUDA runtime error (launch, copy)                      */
  GP_ERR_TIMEOUT = 6,         /* a bounded device wait expired (scheduler dependency not met)   */
  GP_ERR_NO_CONVERGENCE = 7,  /* iterative refinement stopped above its tolerance; result kept  */
  GP_ERR_NO_DEVICE = 8        /* no usable sm_103 GPU                                            */
};

/* Precision of the trailing SYRK/GEMM updates, of the panel TRSMs after the first block column and of
 * the covariance products (the diagonal POTRFs and every residual stay FP64). The reduced forms keep
 * an FP64 copy of K and refine K^{-1} y in FP64 (classic iterative refinement; GMRES for GP_TF32 and
 * GP_BF16); their covariance and log-determinant are not refined, and the shifted factors of GP_TF32 and
 * GP_BF16 give the mean only. The tensor-core forms other than GP_FP32 need tile edge 128 (the
 * automatic choice; cfg.tile 0 or 128) and cfg.tensor_cores = 0. */
enum {
  GP_FP64 = 0,       /* everything FP64 on the FP64 pipe                                            */
  GP_FP32 = 1,       /* FP32-class: tensor cores with three TF32 split products (3xTF32), or FP32
                        FMAs (cfg.tensor_cores = -1); FP64 first-column TRSM                        */
  GP_TF32X3 = 1,     /* the same form under its operand name                                       */
  GP_BF16X3 = 2,     /* tensor cores, BF16 split of the FP32 value into two slices, three products,
                        FP32 accumulation (about 16 significant bits per product)                   */
  GP_BF16X6 = 3,     /* tensor cores, three BF16 slices, six products (FP32-class, 24 bits)          */
  GP_TF32 = 4,       /* tensor cores, one TF32 product (about 11 bits) on K + shift I (cfg.shift);
                        K^{-1} y refined by GMRES in FP64 preconditioned with that factor          */
  GP_BF16 = 5,       /* tensor cores, one BF16 product (about 8 bits): as GP_TF32, coarser            */
  GP_FP64_OZAKI = 6  /* FP64-accurate products on the BF16 tensor cores: each FP64 value cut into
                        seven 8-bit fixed-point digits (Ozaki-style error-free splitting), the 28
                        digit products of weight >= 2^-64 accumulated exactly per weight and summed
                        in 64-bit integers; FP64 POTRF and diagonal-tile inverses; no refinement    */
};

typedef struct {
  double l;   /* lengthscale (textbook form, see above) */
  double v;   /* vertical scale                          */
  double s2;  /* noise variance                          */
} gp_hyper;

typedef struct {
  int32_t tile;           /* tile edge T (multiple of 32, 32..1024); 0 = choose automatically        */
  int32_t precision;      /* GP_FP64, GP_FP32 (= GP_TF32X3), GP_BF16X3, GP_BF16X6, GP_TF32, GP_BF16,
                             GP_FP64_OZAKI (above)                                                    */
  double ir_tol;          /* refinement stops when the normwise backward error ||y - K alpha||_inf /
                             (||K||_inf ||alpha||_inf + ||y||_inf) <= ir_tol (0 = 1e-15), or when it
                             stagnates at <= 100 ir_tol; otherwise GP_ERR_NO_CONVERGENCE            */
  int32_t ir_maxit;       /* refinement iteration limit (0 = 10)                                      */
  int32_t noisy_prior;    /* 1: K_{Xs,Xs} includes s2 on its diagonal (noisy-target covariance)       */
  int64_t timeout_ns;     /* bound on any single device-side wait (0 = 60 s)                          */
  int32_t grid;           /* persistent-kernel CTAs (0 = as many as fit, up to two per SM; the mean's
                             triangular-solve kernel takes one per SM at most)                        */
  int32_t withhold_task;  /* TEST HOOK, read only when withhold_enable != 0. withhold_enable = 1: the
                             persistent-kernel task with this index (in dispatch order) is skipped and
                             never publishes its completion; = 2: the mean solve's forward block with
                             this index is computed but never published. Either way the bounded waits
                             that depend on it expire and the call ends with GP_ERR_TIMEOUT. Leave both
                             fields 0.                                                                */
  int32_t withhold_enable;
  int32_t tensor_cores;   /* GP_FP32 trailing updates: 0 = tensor cores (tcgen05, 3xTF32 split products)
                             when the tile edge is a multiple of 128, -1 = FP32 FMA pipes only       */
  int32_t trace;          /* 1: the persistent kernel records, per task, the CTA and the %globaltimer
                             times at which the task was taken, became ready and finished (read with
                             gp_trace); 0 = off                                                       */
  int32_t batch_order;    /* dispatch order of gp_batch_create: 0 = every ready task ranked by its longest
                             remaining cost path across all GPs; 1 = GPs ranked by total work (largest
                             first), longest path within a GP. gp_batch_autotune stores its choice here. */
  int32_t batch_ctas_per_sm; /* persistent-kernel CTAs per SM of batched launches (0 = library choice: two
                             for GP_FP64, one for GP_FP32; capped by occupancy). gp_batch_autotune stores
                             its choice here.                                                          */
  int32_t locality_order;  /* tensor-core forms: start the grouped trailing updates that share a packed operand
                             group back to back when their longest-path rank is within 10 % of the best
                             ready task's (they then read the shared operand from L2): 0 or 1 = on (the
                             default), -1 = off (longest-path order only)                              */
  double shift;           /* GP_TF32 / GP_BF16 only: the factorised matrix is K + shift I (the stored FP64 K
                             keeps K itself, and the GMRES-refined mean solves with K): > 0 fixed; 0 =
                             automatic, u sqrt(n) max K_ii (u = 2^-11 / 2^-8) times 8 after each
                             non-positive pivot, at most five tries (gp_cholesky then waits for the
                             stream); < 0 = no shift. A factor that carries a shift serves the mean
                             only: gp_predict_full_cov, gp_predict_var and gp_logdet return
                             GP_ERR_INVALID_ARG for it, and gp_nlml_grad needs shift < 0          */
  int32_t tile_variant;    /* GP_FP64 Cholesky graph (Sec. 3.2 names the three tile-algorithm variants):
                             0 = right-looking (each column's trailing updates as separate tasks, longest-
                             path order; the default), 1 = left-looking, 2 = top-looking (all updates of a
                             tile fused into one task before its POTRF/TRSM, dispatched column by column /
                             row by row). The tensor-core forms always run right-looking.              */
} gp_config;

typedef struct gp_ctx gp_ctx;
typedef struct gp_factor gp_factor;

/* Creates a context on `device` that enqueues on `cuda_stream` (a cudaStream_t; NULL = the legacy
 * default stream). `cfg` may be NULL (all defaults). */
gp_status gp_create(gp_ctx** ctx, int32_t device, void* cuda_stream, const gp_config* cfg);
gp_status gp_destroy(gp_ctx* ctx);
/* Replaces the stream used by later calls. */
gp_status gp_set_stream(gp_ctx* ctx, void* cuda_stream);

/* Eq. (1) on the lower tiles of K (Sec. 3.2 stores only tiles on or below the diagonal). X is a
 * device n x D row-major FP64 array and must stay valid for gp_predict_* and gp_nlml* calls on the
 * factor. *K_out: if NULL a factor is allocated; if it already holds a factor of the same n, D and
 * configuration it is reused without allocating. Tiles are T x T row-major, packed tile (I, J) at
 * index I(I+1)/2 + J; n is padded to a multiple of T with an identity block, which leaves L, alpha
 * and the log-determinant of the leading n x n part unchanged. */
gp_status gp_assemble(gp_ctx* ctx, const double* X, int64_t n, int32_t D, gp_hyper h, gp_factor** K_out);

/* Tiled right-looking Cholesky (Sec. 3.2, Fig. 1) in place: K -> L, as one persistent kernel that
 * walks the task DAG of POTRF/TRSM/SYRK/GEMM tile operations. A non-positive pivot ends it with
 * GP_ERR_NOT_PD (reported by gp_sync, info = 1-based column of the n x n matrix). */
gp_status gp_cholesky(gp_ctx* ctx, gp_factor* K);

/* Eq. (2): mean[0..m) = K_{Xs,X} K^{-1} y, using the factor L from gp_cholesky. y and Xs are device
 * arrays (n and m x D). With the reduced forms the solve is refined in FP64 against the stored FP64
 * K (classic refinement for GP_FP32, GP_BF16X6, GP_BF16X3; GMRES for GP_TF32, GP_BF16); *ir_iters_out
 * (host, may be NULL) receives the refinement steps (GMRES: preconditioned matrix-vector products),
 * which makes this call wait for the stream. The refined forms wait for the stream at every step (the
 * host reads the backward error); they stop refining at the first device error (left in the status
 * word for gp_sync) and return GP_ERR_NONFINITE for a non-finite residual without one. GP_FP64 and
 * GP_FP64_OZAKI do not refine. alpha = K^{-1} y stays in the factor for gp_nlml_grad and gp_alpha. */
gp_status gp_predict_mean(gp_ctx* ctx, gp_factor* L, const double* y, const double* Xs, int64_t m,
                          double* mean_out, int32_t* ir_iters_out);

/* Eq. (3): cov (m x m, both triangles written) = K_{Xs,Xs} - V^T V with L V = K_{X,Xs}.
 * GP_ERR_INVALID_ARG for a factor of K + shift I (single-product forms with a shift). */
gp_status gp_predict_full_cov(gp_ctx* ctx, gp_factor* L, const double* Xs, int64_t m, double* cov_out);

/* Predictive variances only, the diagonal of Eq. (3) (the paper notes that the diagonal of the
 * posterior covariance holds the predictive variances, Sec. 3.1): var[j] = k(xs_j, xs_j) - ||V_:,j||^2
 * with L V = K_{X,Xs}, without forming V^T V. var_out: device, m. GP_ERR_INVALID_ARG for a factor of
 * K + shift I. */
gp_status gp_predict_var(gp_ctx* ctx, gp_factor* L, const double* Xs, int64_t m, double* var_out);

/* log det K = 2 sum log L_ii of the factor (host output; waits for the stream). GP_ERR_INVALID_ARG for
 * a factor of K + shift I. */
gp_status gp_logdet(gp_ctx* ctx, gp_factor* L, double* out);

/* Negative log marginal likelihood and its gradient w.r.t. (l, v, s2) at h, for device X (n x D) and
 * y (n): assembles K, factors it, solves for alpha, then runs the blocked Cholesky adjoint to obtain
 * Kbar = 1/2 (K^{-1} - alpha alpha^T) tile by tile and contracts it with dK/dtheta recomputed from X
 * (dK is never stored). Host outputs; waits for the stream. GP_TF32 / GP_BF16 need cfg.shift < 0 (an
 * unshifted factor of K), else GP_ERR_INVALID_ARG. */
gp_status gp_nlml_grad(gp_ctx* ctx, const double* X, const double* y, int64_t n, int32_t D, gp_hyper h,
                       double* nlml_out, double grad_out[3]);

/* Copies rows [row0, row0 + nrows) of the n x n lower-triangular matrix held by the factor (K after
 * gp_assemble, L after gp_cholesky) to out (device, nrows x n row-major; entries above the diagonal
 * are written as 0). Asynchronous. */
gp_status gp_factor_rows(gp_ctx* ctx, const gp_factor* f, int64_t row0, int64_t nrows, double* out);

/* Refinement record of a factor (host, 4 doubles): {shift the factorised matrix carried (single-product
 * forms), normwise backward error reached by the last gp_predict_mean, its refinement steps (GMRES:
 * preconditioned matrix-vector products), precision form}. Host only; no wait. */
gp_status gp_factor_stats(gp_ctx* ctx, const gp_factor* f, double out[4]);

/* Copies alpha = K^{-1} y from the last gp_predict_mean on the factor to out (device, n). */
gp_status gp_alpha(gp_ctx* ctx, const gp_factor* f, double* out);

/* x = (L L^T)^{-1} b with the stored factor L (of K, or of K + shift I for the single-product forms), by
 * the two blocked substitutions of Eq. 2 and no refinement: b, x device arrays of n doubles (they may be
 * the same array). GP_FP64 and GP_FP64_OZAKI solve in FP64; the refined forms (FP32-accurate factors)
 * solve with the factor's FP32 copy in FP32 arithmetic at tile edges 128 and 256 (their correction
 * solves), in FP64 at other tile edges. Asynchronous; a device wait that expires is reported by gp_sync
 * as GP_ERR_TIMEOUT. GP_ERR_INVALID_ARG before gp_cholesky. */
gp_status gp_solve(gp_ctx* ctx, gp_factor* f, const double* b, double* x);

gp_status gp_factor_free(gp_ctx* ctx, gp_factor* f);

/* Waits for the context's stream, then returns and clears the first device-side error
 * (GP_OK if none). *info (host, may be NULL) receives its detail (failing column for NOT_PD). */
gp_status gp_sync(gp_ctx* ctx, int64_t* info);

/* ---------------------------------------------------------------- batches of independent GPs
 * Many independent GPs of uneven size are assembled, factored and predicted together: one batched
 * assembly kernel, ONE persistent task-DAG launch running every GP's tiled Cholesky (Sec. 3.2), mean
 * solve (Eq. 2) and covariance solve (Eq. 3) in a single list-scheduled order, and one output kernel,
 * captured once into a CUDA graph. Not in the paper (its GPs are solved one at a time). */
typedef struct {
  const double* X;   /* device, n x D       */
  const double* y;   /* device, n           */
  const double* Xs;  /* device, m x D       */
  int64_t n, m;
  int32_t D;
  int32_t tile;      /* tile edge for this GP (multiple of 32); 0 = library choice by n       */
  gp_hyper h;
  double* mean_out;  /* device, m                                                               */
  double* cov_out;   /* device, m x m (both triangles), or NULL for the mean only              */
} gp_batch_desc;

typedef struct gp_batch gp_batch;

/* Allocates the batch's workspace, builds its task order and captures its CUDA graph. The device
 * pointers in descs are baked into the graph: they must stay valid (their contents may change)
 * until gp_batch_free. Precision follows the context: GP_FP32 runs the FP32 trailing updates of
 * the mixed mode without the refinement step. */
gp_status gp_batch_create(gp_ctx* ctx, int32_t B, const gp_batch_desc* descs, gp_batch** out);
/* Launches the captured graph on the context's stream (asynchronous; errors via gp_sync, where a
 * NOT_PD info holds the GP index in its high 32 bits and the column in the low 32 bits). */
gp_status gp_batch_run(gp_ctx* ctx, gp_batch* b);
gp_status gp_batch_free(gp_ctx* ctx, gp_batch* b);
/* One-shot batch: gp_batch_create, one gp_batch_run and gp_batch_free, then the device status as
 * gp_sync returns it (and clears it), its detail in *info (host, may be NULL; for GP_ERR_NOT_PD the GP
 * index in the high 32 bits and the column in the low 32 bits). An error still pending from an earlier
 * call on the context is returned first, with its detail, and then nothing of the batch runs. With
 * want_cov = 0 only the means are computed (the descriptors' cov_out are ignored). Synchronous; for
 * repeated solves of the same shapes keep a gp_batch instead (its graph is captured once). */
gp_status gp_batch_predict(gp_ctx* ctx, int32_t B, const gp_batch_desc* descs, int32_t want_cov,
                           int64_t* info);

/* Sets the schedule of later gp_batch_create calls: cfg.batch_order (0 or 1) and
 * cfg.batch_ctas_per_sm (0..2), as gp_create validates them (GP_ERR_INVALID_ARG otherwise). For a
 * schedule chosen earlier by gp_batch_autotune and kept by the caller (the Python binding's JSON
 * cache). Host only. */
gp_status gp_set_batch_schedule(gp_ctx* ctx, int32_t order, int32_t ctas_per_sm);

/* Autotuner of the batched path (not in the paper, whose tile count is fixed per run): chooses each
 * GP's tile edge and the batch's schedule by timing them on this GPU.
 *   1. The GPs are split into `classes` size classes of equal count by n. For each class a sample of
 *      up to `sample` GPs (evenly spaced in n) is run as a batch of its own with every candidate tile
 *      edge (candidates more than twice the class's largest n are skipped); the fastest edge wins.
 *   2. With those edges, the whole batch is run under every schedule (cfg.batch_order 0 and 1, and
 *      for GP_FP64 one and two CTAs per SM); the fastest wins.
 *   3. The batch under the library's own tile rule and schedule is timed too; if it is faster, it is
 *      the choice (descs[g].tile = 0, order 0, residency 0).
 * Each trial is one gp_batch_create, one untimed run and `reps` runs timed with CUDA events (the
 * best is kept). On return descs[g].tile holds the chosen edge of GP g, the context's
 * cfg.batch_order / cfg.batch_ctas_per_sm hold the chosen schedule (used by later gp_batch_create
 * calls), and *result (host, may be NULL) reports the choices and timings. The trials write the
 * outputs of the GPs they run (the caller's mean_out / cov_out arrays). Synchronous. */
typedef struct {
  int32_t tiles[6];  /* candidate tile edges (multiples of 32, <= 1024); all 0 = {32, 64, 128, 256} */
  int32_t classes;   /* size classes, 1..8 (0 = 3)                                                  */
  int32_t sample;    /* GPs timed per class (0 = 24)                                                */
  int32_t reps;      /* timed runs per trial (0 = 2)                                                */
  int32_t reserved;
} gp_autotune_opts;

typedef struct {
  int32_t nclass;
  int32_t class_tile[8];     /* chosen tile edge per class                                         */
  int64_t class_nmax[8];     /* class k holds the GPs with class_nmax[k-1] < n <= class_nmax[k]       */
  double class_seconds[8];   /* best time of the class's sample (s)                                */
  int32_t order;             /* chosen cfg.batch_order                                             */
  int32_t ctas_per_sm;       /* chosen cfg.batch_ctas_per_sm                                       */
  int32_t trials;            /* batches built and timed                                            */
  int32_t reserved;
  double seconds_tuned;      /* the whole batch with the chosen tiles and schedule (s, best run)    */
  double seconds_default;    /* the whole batch with the library's own tile rule and schedule (s)   */
  double seconds_spent;      /* wall time of the whole search (s)                                  */
} gp_autotune_result;

gp_status gp_batch_autotune(gp_ctx* ctx, int32_t B, gp_batch_desc* descs, const gp_autotune_opts* opts,
                            gp_autotune_result* result);

/* Predictive mean (Eq. 2) of a small GP, end to end, without allocating anything -- no
 * counterpart in the paper; it exists for callers that cannot call cudaMalloc (a real-time loop that
 * must not touch the device allocator, a process whose device memory is fixed up front, or a host
 * application that owns all device memory and lends the library only its inputs and outputs).
 * X (n x D), y (n), Xs (m x D) and mean_out (m) are the caller's device arrays; nothing else is
 * needed: no context, no factor. The library's workspace is one file-scope device array of about
 * 4.5 MB (tiles of edge 64, counters, task lists, status word) that every GPU loading the library
 * holds until the process exits. Set-up: the first call made on a device (with that device current)
 * looks the array's device address up and keeps it; a later call looks it up again only if the
 * device's CUDA context has changed since (for example after cudaDeviceReset). Make that first call
 * before any stream capture. n must be <= 1024 (larger n returns GP_ERR_INVALID_ARG).
 * Runs on `cuda_stream` of the current device and waits for it, then returns the device status
 * (GP_ERR_NOT_PD with *info = failing column, GP_ERR_TIMEOUT; info may be NULL). Every call shares
 * the one array and leaves its contents behind; each call clears what must start at zero, but calls
 * that overlap on the GPU (other streams or host threads) race on it. */
gp_status gp_predict_mean_noalloc(const double* X, const double* y, int64_t n, int32_t D, gp_hyper h,
                                  const double* Xs, int64_t m, double* mean_out, void* cuda_stream,
                                  int64_t* info);

/* Host-only introspection of the persistent kernel's dispatch order: writes the task list of graph
 * `graph` (0 = tiled Cholesky, 1 = covariance solve, 2 = mean solve, 3 = reverse sweep of the tiled
 * Cholesky used by gp_nlml_grad, 4 = the V solve of gp_predict_var) for Mt tile rows, Mc covariance
 * tile columns, tile edge T, `workers` CTAs and the cost model of precision `mixed` (0 = FP64,
 * 1 = GP_FP32 with the locality order off; 3 = GP_FP32 with it on; 4 / 5 = GP_FP64 with cfg.tile_variant 1 / 2) as int32 quadruples {kind, p, q, r} (kinds as in the
 * library's task table: 0 POTRF(J), 1 TRSM(I,J), 2 UPDATE(I,K,J), 3 VTRSM(J,c), 4 VGEMM(I,J,c),
 * 5 WSYRK(a,b,J), 6 FSOLVE(J), 7 FGEMV(I,J,ch), 8 BSOLVE(J), 9 BGEMV(J,I,ch), 10 RUPD(P,K,J),
 * 11 RTRSM(P,J), 12 RDIAG(P,J), 13 RPOTRF(J), 14 TRTRI(J): the FP64 inverse of the factored diagonal tile
 * J, which the vector solves of gp_predict_mean apply as a matrix-vector product, 15 VGEMM(I,c,J0|J1<<16)
 * and 16 WSYRK(a,b,J0|J1<<16): products of columns J0..J1-1 applied in one pass, mixed mode with
 * 128-multiple tiles; 17 FSOLVE(J,ch) and 18 BSOLVE(J,ch): 32-row chunk ch of the diagonal-block solve of
 * the mean graph, a product with the stored inverse of the diagonal tile; 19 UPDATE2(I,K,J0|J1<<16):
 * the grouped updates of tiles (I,K) and (I+1,K) in one pass over the shared L_KJ, mixed mode with
 * tile edge 128) into out (host, room for cap tasks). Returns the task count, or -1 on bad
 * arguments. Needs no GPU. */
int64_t gp_schedule_tasks(int32_t graph, int32_t Mt, int32_t Mc, int32_t T, int32_t workers, int32_t mixed,
                          int32_t* out, int64_t cap);

/* Task trace of the last persistent-kernel launch on this context (cfg.trace = 1): for each task in
 * dispatch order, {kind, p, q, r} as gp_schedule_tasks describes them (batched launches carry the GP
 * index in kind's bits 5 and up) followed by {CTA, t_taken, t_ready, t_done} in ns of %globaltimer,
 * 8 int64 per task, into out (host, room for cap tasks). Waits for the stream. Returns the task
 * count, or -1 when tracing is off or nothing was traced. */
int64_t gp_trace(gp_ctx* ctx, int64_t* out, int64_t cap);

/* Human-readable name of a status code (static string). */
const char* gp_status_string(gp_status s);

/* Number of kernel launches the library has enqueued on this context so far. */
int64_t gp_launch_count(const gp_ctx* ctx);

/* TEST HOOK (host-side fault injection): counting device allocations from this call on, the k-th one
 * made by any context of the process fails as cudaMalloc would, and the entry point that needed it
 * returns GP_ERR_OOM with its objects left valid (retry after freeing memory); k <= 0 turns it off.
 * Not thread-safe against concurrent calls into the library. */
void gp_debug_fail_alloc(int64_t k);

/* TEST HOOK (no counterpart in the paper): one tensor-core tile product through the same device
 * routines the persistent kernel uses for the trailing updates (Sec. 3.2's SYRK/GEMM): A and B are
 * device 128 x K row-major FP64 arrays (K a multiple of 32, at most 1024; at most 512 for
 * GP_FP64_OZAKI), packed in the operand format of `precision` (GP_FP32 = 3xTF32, GP_TF32, GP_BF16,
 * GP_BF16X3, GP_BF16X6, GP_FP64_OZAKI), then C (device 128 x 128 row-major FP64) -= A B^T (store != 0:
 * C = A B^T; lower != 0: only entries with column <= row change), repeated `reps` times on the
 * context's stream in one CTA. Needs cfg.tensor_cores = 0. Synchronous; returns the device status. */
gp_status gp_debug_tile_product(gp_ctx* ctx, int32_t precision, const double* A, const double* B, double* C,
                                int32_t K, int32_t store, int32_t lower, int32_t reps);

/* TEST HOOK: out[i] = the covariance assembly's exponential of x[i] (device arrays of n doubles; the
 * assembly only evaluates x <= 0): a table-driven evaluation after Tang (ACM TOMS 1989), x < -745.2
 * giving +0 and NaN staying NaN. Asynchronous. */
gp_status gp_debug_exp_neg(gp_ctx* ctx, const double* x, int64_t n, double* out);

/* TEST HOOK (host only, no GPU needed): the work items, in order, of CTA `cta` of the FP32 correction
 * solve's persistent kernel run with `ctas` CTAs on Mt tile rows, as {kind, I, J} int32 triples in out
 * (host, 3 x cap). Kinds: 0 forward tile (I, J), 1 forward chain step of block I (J = I - 1), 2 forward
 * y product of block I, 3 the first forward block (0), 4-7 the same for the backward sweep (the chain
 * step of block J carries I = J + 1). Returns the number of items (out may be null), -1 on invalid
 * arguments. */
int64_t gp_debug_solve_items(int32_t Mt, int32_t ctas, int32_t cta, int32_t* out, int64_t cap);

/* TEST HOOK (host only): the covariance assembly's squared distance from fixed-point coordinates,
 * sum_d (qa[d] - qb[d])^2 2^-twoF rounded once to FP64 by the same integer routines the kernels run.
 * qa, qb: host arrays of D values with |q| < 2^58; 1 <= D <= 256, twoF <= 1022 (normal or zero
 * results). Writes *out; GP_ERR_INVALID_ARG outside those ranges. */
gp_status gp_debug_fx_sqdist(const int64_t* qa, const int64_t* qb, int32_t D, int32_t twoF, double* out);

#ifdef __cplusplus
}
#endif
#endif /* GP_H_ */
