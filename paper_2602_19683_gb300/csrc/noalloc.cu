// gp_predict_mean_noalloc: the whole predictive-mean path for a small GP (assembly, tiled Cholesky,
// both substitutions and the cross-covariance GEMV) without allocating any memory.
//
// Who needs it: callers that cannot call cudaMalloc -- code that runs where the device allocator is
// off limits (a real-time control loop that must not block on the allocator or fragment memory, a
// process whose memory pool is fixed up front, an embedding application that owns all device memory
// and only lends the library its inputs and outputs). Such a caller passes its device inputs and
// output and gets the mean back; the library's own workspace (tiles, counters, task lists, status
// word) lives in one file-scope device array that every GPU loading the library holds until exit.
//
// Limits and sharing: n <= kNoAllocMaxN training points (tile edge 64, at most 16 x 16 tiles; the
// array is about 4.5 MB). Every call uses the same array and leaves the last call's contents in it;
// each call clears what must start at zero (counters, status word, padding of the solve vector), so
// consecutive calls are independent, but calls that overlap on the GPU (two streams, two host threads)
// race on the array and give wrong results.
#include <cuda.h>

#include <climits>
#include <cstring>
#include <mutex>

#include "../../include/gp.h"
#include "kernels.h"

namespace {

constexpr long long kNoAllocMaxN = 1024;
constexpr int kT = 64;                                 // tile edge
constexpr int kMtMax = (int)(kNoAllocMaxN / kT);       // 16 tile rows
constexpr int kTilesMax = kMtMax * (kMtMax + 1) / 2;  // 136 lower tiles
constexpr int kNch = kT / 32;
// Task counts of the in-order task lists at Mt tile rows (upper bounds at kMtMax).
constexpr int kCholTasksMax = kMtMax + kMtMax * (kMtMax - 1) / 2 + (kMtMax - 1) * kMtMax * (kMtMax + 1) / 6;
constexpr int kMeanTasksMax = 2 * kMtMax + kMtMax * (kMtMax - 1) * kNch;

struct Scratch {
  double tiles[(size_t)kTilesMax * kT * kT];
  double bvec[kMtMax * kT];
  gpk::DevStatus status;
  int cK[kTilesMax];
  int cMean[kMtMax * kNch * 2 + kMtMax * 2];
  int4 chol_tasks[kCholTasksMax];
  int4 mean_tasks[kMeanTasksMax];
};
constexpr size_t kScratchBytes = sizeof(Scratch);

// The library's only workspace for this entry point (see the file comment).
static __device__ __align__(256) unsigned char g_gp_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
// Device address of g_gp_noalloc_scratch per device, and the id of the CUDA context it was looked up
// in: a device whose context was replaced since (cudaDeviceReset, another context made current)
// loads the module again at another address, so the lookup is redone there.
void* g_scratch_ptr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

// Id of the CUDA context current on this thread (0 if none), through the driver entry points that
// the runtime exposes (no link-time dependency on the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {  // under g_setup_mutex
    looked_up = true;
    cudaDriverEntryPointQueryResult q1, q2;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = (CtxGetCurrentFn)f1;
      get_id = (CtxGetIdFn)f2;
    }
    cudaGetLastError();
  }
  if (!get_current || !get_id) return 0;
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

// Writes the in-order task lists (a topological order of Fig. 1's tasks, and of the two
// substitutions) for Mt tile rows: one thread, a few hundred tasks.
__global__ void noalloc_tasks_kernel(int Mt, int4* chol, int4* mean) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  int c = 0;
  for (int J = 0; J < Mt; ++J) {
    chol[c++] = make_int4(gpk::TASK_POTRF, J, 0, 0);
    for (int I = J + 1; I < Mt; ++I) chol[c++] = make_int4(gpk::TASK_TRSM, I, J, 0);
    for (int I = J + 1; I < Mt; ++I)
      for (int K = J + 1; K <= I; ++K) chol[c++] = make_int4(gpk::TASK_UPD, I, K, J);
  }
  int t = 0;
  for (int J = 0; J < Mt; ++J) {
    mean[t++] = make_int4(gpk::TASK_FSOLVE, J, 0, 0);
    for (int I = J + 1; I < Mt; ++I)
      for (int ch = 0; ch < kNch; ++ch) mean[t++] = make_int4(gpk::TASK_FGEMV, I, J, ch);
  }
  for (int I = Mt - 1; I >= 0; --I) {
    mean[t++] = make_int4(gpk::TASK_BSOLVE, I, 0, 0);
    for (int J = 0; J < I; ++J)
      for (int ch = 0; ch < kNch; ++ch) mean[t++] = make_int4(gpk::TASK_BGEMV, J, I, ch);
  }
}

// Device address of the scratch array on the current device. Set-up, done by the first call made on
// a device (with that device current): cudaGetSymbolAddress, its return code checked. Later calls
// reuse the address while the device's context stays the same one.
gp_status scratch_on(int device, Scratch** out) {
  if (device < 0 || device >= kMaxDevices) return GP_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  unsigned long long ctx = current_context_id();
  if (ctx == 0) {  // no context yet on this thread: make the device's primary context current
    if (cudaSetDevice(device) != cudaSuccess) {
      cudaGetLastError();
      return GP_ERR_NO_DEVICE;
    }
    ctx = current_context_id();
  }
  if (!g_scratch_ptr[device] || ctx == 0 || ctx != g_scratch_ctx[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_gp_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      g_scratch_ptr[device] = nullptr;
      return GP_ERR_CUDA;
    }
    g_scratch_ptr[device] = p;
    g_scratch_ctx[device] = ctx;
  }
  *out = (Scratch*)g_scratch_ptr[device];
  return GP_OK;
}

}  // namespace

extern "C" gp_status gp_predict_mean_noalloc(const double* X, const double* y, int64_t n, int32_t D, gp_hyper h,
                                             const double* Xs, int64_t m, double* mean_out, void* cuda_stream,
                                             int64_t* info) {
  if (info) *info = 0;
  if (!X || !y || n < 1 || D < 1 || m < 0 || (m > 0 && (!Xs || !mean_out))) return GP_ERR_INVALID_ARG;
  if (n > kNoAllocMaxN) return GP_ERR_INVALID_ARG;  // the static workspace holds n <= 1024
  if (!(h.l > 0) || !(h.v > 0) || !(h.s2 >= 0) || h.l != h.l || h.v != h.v || h.s2 != h.s2) return GP_ERR_INVALID_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_NO_DEVICE;
  }
  Scratch* s = nullptr;
  gp_status st = scratch_on(device, &s);
  if (st != GP_OK) return st;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const int Mt = (int)((n + kT - 1) / kT);
  const int ntiles = Mt * (Mt + 1) / 2;
  const int nchol = Mt + Mt * (Mt - 1) / 2 + (Mt - 1) * Mt * (Mt + 1) / 6;
  const int nmean = 2 * Mt + Mt * (Mt - 1) * kNch;
  cudaError_t e = cudaSuccess;
#define NOALLOC_CUDA(x)          \
  do {                           \
    e = (x);                     \
    if (e != cudaSuccess) {      \
      cudaGetLastError();        \
      return GP_ERR_CUDA;        \
    }                            \
  } while (0)
  // what must start at zero: status word, counters, the solve vector (its padding)
  NOALLOC_CUDA(cudaMemsetAsync(&s->status, 0, sizeof(gpk::DevStatus), stream));
  const long long big = LLONG_MAX;
  NOALLOC_CUDA(cudaMemcpyAsync(&s->status.info, &big, sizeof(big), cudaMemcpyHostToDevice, stream));
  NOALLOC_CUDA(cudaMemsetAsync(s->cK, 0, sizeof(s->cK), stream));
  NOALLOC_CUDA(cudaMemsetAsync(s->cMean, 0, sizeof(s->cMean), stream));
  NOALLOC_CUDA(cudaMemsetAsync(s->bvec, 0, sizeof(s->bvec), stream));
  NOALLOC_CUDA(cudaMemcpyAsync(s->bvec, y, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, stream));
  noalloc_tasks_kernel<<<1, 1, 0, stream>>>(Mt, s->chol_tasks, s->mean_tasks);
  NOALLOC_CUDA(cudaGetLastError());
  NOALLOC_CUDA(gpk::launch_assemble_tiles(X, n, D, h.l, h.v, h.s2, s->tiles, kT, Mt, stream));
  gpk::DagArgs a;
  std::memset(&a, 0, sizeof(a));
  a.Kt = s->tiles;
  a.T = kT;
  a.Mt = Mt;
  a.nch = kNch;
  a.cK = s->cK;
  a.st = &s->status;
  a.timeout_ns = 10LL * 1000 * 1000 * 1000;
  a.withhold_task = -1;
  a.tasks = s->chol_tasks;
  a.ntasks = nchol;
  const int grid = 2 * sms < nchol ? 2 * sms : nchol;
  NOALLOC_CUDA(gpk::launch_dag(a, grid, false, stream));
  a.bvec = s->bvec;
  a.cF = s->cMean;
  a.cB = s->cMean + Mt * kNch;
  a.dF = s->cMean + 2 * Mt * kNch;
  a.dB = a.dF + Mt;
  a.tasks = s->mean_tasks;
  a.ntasks = nmean;
  NOALLOC_CUDA(cudaMemsetAsync(&s->status.next_task, 0, sizeof(unsigned long long), stream));
  NOALLOC_CUDA(gpk::launch_dag(a, 2 * sms < nmean ? 2 * sms : nmean, false, stream));
  if (m > 0) NOALLOC_CUDA(gpk::launch_mean_gemv(Xs, m, X, n, D, h.l, h.v, s->bvec, mean_out, stream));
  gpk::DevStatus hs;
  NOALLOC_CUDA(cudaMemcpyAsync(&hs, &s->status, sizeof(hs), cudaMemcpyDeviceToHost, stream));
  NOALLOC_CUDA(cudaStreamSynchronize(stream));
#undef NOALLOC_CUDA
  (void)ntiles;
  if (hs.code != 0 && info) *info = hs.info == LLONG_MAX ? 0 : hs.info;
  return hs.code;
}
