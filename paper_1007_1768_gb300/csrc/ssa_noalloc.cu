// ssa_ensemble_run_noalloc: the ensemble run for callers that must not
// allocate device memory.
//
// Some hosts cannot call cudaMalloc at the moment they want a result.  Examples:
// code running inside a memory pool that another runtime owns and sizes up
// front; plugins that a host process forbids from touching the allocator;
// real-time loops that must not block on allocation.  This entry point
// serves them.  It allocates nothing: no cudaMalloc, no cudaMallocAsync, no
// cudaFree, no allocating library call.  Its scratch memory (work counter,
// totals, per-grid difference sums, the uniform grid and the initial counts)
// lives in one file-scope device array of fixed size, kNoAllocScratchBytes,
// that every GPU loading the library holds until the process exits.  The
// caller passes every input and output buffer.
//
// Because every call shares that one array, calls whose work overlaps on the
// GPU (different streams, or different host threads, on the same device) race
// and give wrong results.  Calls must be serialised: issue them on one stream,
// or wait for one before starting the next.  Each call clears the parts that
// must start at zero (counter, totals, difference sums) on its own stream
// before its kernels run.
//
// The first call on a device looks up the device address of the array with
// cudaGetSymbolAddress (with that device current) and caches it.  That first
// call should therefore come before any stream capture on that device.
//
// The call moves no data from host memory: the kernel takes the model's
// small tables by value (kernel parameters), and the one table the
// finalisation reads from device memory (x0) is written into the scratch by a
// one-warp kernel from a by-value copy.  The host thread waits only when the
// caller asks for stats.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "ssa.h"
#include "ssa_internal.h"

namespace ssa_impl {
ssa_status record_error(ssa_status st, const char* msg);
void clear_error();
}  // namespace ssa_impl

using namespace ssa_impl;

namespace {

constexpr size_t kNoAllocScratchBytes = SSA_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

// The scratch array.  Host code must not use its name as an address: on the
// host it is only a stand-in for the device symbol.  The device address comes
// from cudaGetSymbolAddress in scratch_on_device().
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};
size_t g_smem_optin[kMaxDevices] = {};

ssa_status scratch_on_device(int dev, unsigned char** out, int* sms, size_t* smem_optin) {
  if (dev < 0 || dev >= kMaxDevices) return record_error(SSA_EUNSUPPORTED, "device index out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return record_error(SSA_ECUDA, "cudaGetSymbolAddress(noalloc scratch) failed");
    int n_sms = 0, smem = 0;
    e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return record_error(SSA_ECUDA, "cudaDeviceGetAttribute failed");
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
    g_sms[dev] = n_sms;
    g_smem_optin[dev] = (size_t)smem;
  }
  *out = g_scratch_ptr[dev];
  *sms = g_sms[dev];
  *smem_optin = g_smem_optin[dev];
  return SSA_OK;
}

// The initial counts, by value, for the one-warp kernel below.
struct X0Words {
  int32_t v[kSmallMax];
};

__global__ void k_put_x0(int32_t* dst, X0Words x0, int S) {
  const int s = threadIdx.x;
  if (s < S) dst[s] = x0.v[s];
}

}  // namespace

extern "C" ssa_status ssa_ensemble_run_noalloc(const ssa_model* model, int64_t n_traj, double t_end,
                                               int32_t n_grid, const double* grid, uint64_t seed,
                                               const ssa_run_opts* opts, double* mean, double* var,
                                               int64_t* sum1, int64_t* sum2, ssa_run_stats* stats) {
  clear_error();
  ssa_run_opts o;
  if (opts) o = *opts; else ssa_run_opts_init(&o);
  // a consistent copy of the model's small tables (taken under the model's
  // lock, so a concurrent ssa_model_set_rate_modifier cannot tear it)
  SmallModelCopy mc;
  if (!model || !model_small_copy(model, &mc)) return record_error(SSA_EINVAL, "model is NULL");
  if (n_traj < 1) return record_error(SSA_EINVAL, "n_traj must be >= 1");
  if (!(t_end > 0.0) || !std::isfinite(t_end)) return record_error(SSA_EINVAL, "t_end must be finite and > 0");
  if (n_grid < 1) return record_error(SSA_EINVAL, "n_grid must be >= 1");
  if (!mean || !var) return record_error(SSA_EINVAL, "mean and var must not be NULL");
  if (o.memory != SSA_MEM_DEVICE)
    return record_error(SSA_EINVAL, "ssa_ensemble_run_noalloc takes device buffers only (memory = SSA_MEM_DEVICE)");
  if (o.precision != SSA_PREC_FP64) return record_error(SSA_EUNSUPPORTED, "this entry point runs SSA_PREC_FP64 only");
  if (mc.has_mod)
    return record_error(SSA_EUNSUPPORTED,
                        "models with rate modifiers run on the warp schedule, which this entry point does not serve");
  if (o.schedule == SSA_SCHED_WARP || !mc.has_small)
    return record_error(SSA_EUNSUPPORTED, "networks with more than 16 reactions or species are not supported here");
  if (o.schedule < SSA_SCHED_AUTO || o.schedule > SSA_SCHED_WARP) return record_error(SSA_EINVAL, "bad schedule");
  if (o.reduce < SSA_REDUCE_AUTO || o.reduce > SSA_REDUCE_GLOBAL) return record_error(SSA_EINVAL, "bad reduce mode");
  if (o.block_threads < 0 || o.block_threads > 512 || (o.block_threads % 32) != 0)
    return record_error(SSA_EINVAL, "block_threads must be 0 or a multiple of 32 up to 512");
  if (o.grid_blocks < 0) return record_error(SSA_EINVAL, "grid_blocks must be >= 0");
  if (o.max_events > (int64_t)0xFFFFFFFFLL) return record_error(SSA_EINVAL, "max_events must be below 2^32");
  if (o.stream_id > 0xFFFFFFFFULL) return record_error(SSA_EINVAL, "stream_id must be below 2^32");

  // scratch layout inside the fixed array
  const size_t gs = (size_t)n_grid * (size_t)mc.S;
  auto up = [](size_t v) { return align_up(v, 256); };
  const size_t off_counter = 0;
  const size_t off_stats = up(off_counter + 8);
  const size_t off_d1 = up(off_stats + 8 * kStatCount);
  const size_t off_d2 = up(off_d1 + 8 * gs);
  const size_t off_grid = up(off_d2 + 8 * gs);
  const size_t off_x0 = up(off_grid + 8 * (size_t)n_grid);
  const size_t need = up(off_x0 + 4 * (size_t)kSmallMax);
  if (gs > ((size_t)1 << 31) || need > kNoAllocScratchBytes) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "ssa_ensemble_run_noalloc needs %zu bytes of scratch for n_grid = %d and %d species; its fixed "
             "scratch holds %zu bytes (SSA_NOALLOC_SCRATCH_BYTES)",
             need, n_grid, mc.S, kNoAllocScratchBytes);
    return record_error(SSA_EINVAL, msg);
  }

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return record_error(SSA_ECUDA, "cudaGetDevice failed");
  unsigned char* scratch = nullptr;
  int sms = 0;
  size_t smem_optin = 0;
  ssa_status st = scratch_on_device(dev, &scratch, &sms, &smem_optin);
  if (st != SSA_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(o.cuda_stream);

  // launch shape (same rule as ssa_ensemble_run)
  LaunchPlan plan;
  if (const char* msg = plan_thread_launch(mc.S, mc.M, n_grid, n_traj, sms, smem_optin, o.reduce, o.block_threads,
                                           o.grid_blocks, &plan))
    return record_error(SSA_EINVAL, msg);

  auto cuda_fail = [](cudaError_t e, const char* what) {
    char msg[256];
    snprintf(msg, sizeof msg, "%s: %s", what, cudaGetErrorString(e));
    return record_error(SSA_ECUDA, msg);
  };
  cudaError_t e = thread_kernel_set_smem(mc.M, mc.S, plan.shared_d, plan.smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  // counter, totals and difference sums start at zero on every call
  e = cudaMemsetAsync(scratch, 0, off_grid, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(scratch)");
  int32_t* d_x0 = reinterpret_cast<int32_t*>(scratch + off_x0);
  X0Words x0w = {};
  for (int s = 0; s < mc.S; ++s) x0w.v[s] = mc.small.x0[s];
  k_put_x0<<<1, 32, 0, stream>>>(d_x0, x0w, mc.S);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "initial counts kernel");
  const double* d_grid = grid;
  if (!d_grid) {
    double* g = reinterpret_cast<double*>(scratch + off_grid);
    e = launch_uniform_grid(g, n_grid, t_end, stream);
    if (e != cudaSuccess) return cuda_fail(e, "uniform grid kernel");
    d_grid = g;
  }

  RunArgs a;
  a.sm = mc.small;
  a.m = DevModel{};  // the thread kernel reads the small tables from its parameters
  a.m.S = mc.S;
  a.m.M = mc.M;
  a.m.x0 = d_x0;
  a.G = n_grid;
  a.N = n_traj;
  a.traj_offset = o.traj_offset;
  a.seed = seed;
  a.seed_word = nullptr;
  a.stream_id = o.stream_id;
  a.max_events = (o.max_events > 0) ? o.max_events : SSA_DEFAULT_MAX_EVENTS;
  a.t_end = t_end;
  a.grid = d_grid;
  a.D1 = reinterpret_cast<unsigned long long*>(scratch + off_d1);
  a.D2 = reinterpret_cast<unsigned long long*>(scratch + off_d2);
  a.counter = reinterpret_cast<unsigned long long*>(scratch + off_counter);
  a.stats = reinterpret_cast<unsigned long long*>(scratch + off_stats);
  a.traj_events = o.traj_events;
  a.traj_hash = o.traj_hash;
  a.traj_flags = o.traj_flags;
  a.device_totals = reinterpret_cast<unsigned long long*>(o.device_totals);
  a.grid_uniform = (!grid && n_grid >= 2 && n_grid <= (1 << 20) && t_end < 1e30) ? 1 : 0;
  a.grid_scale = (float)((double)(n_grid - 1) / t_end);
  a.grid_margin = (float)((double)n_grid * 0x1p-21);

  if (o.sim_event_begin) {
    e = cudaEventRecord(static_cast<cudaEvent_t>(o.sim_event_begin), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(sim_event_begin)");
  }
  e = launch_thread_kernel(a, plan.blocks, plan.threads, plan.shared_d, plan.smem, stream);
  if (e != cudaSuccess) return cuda_fail(e, "simulation kernel");
  if (o.sim_event_end) {
    e = cudaEventRecord(static_cast<cudaEvent_t>(o.sim_event_end), stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaEventRecord(sim_event_end)");
  }
  e = launch_finalize(a.D1, a.D2, n_grid, mc.S, n_traj, a.m.x0, mean, var, sum1, sum2, stream);
  if (e != cudaSuccess) return cuda_fail(e, "finalize kernel");
  if (!stats) return SSA_OK;

  unsigned long long h[kStatCount] = {};
  e = cudaMemcpyAsync(h, a.stats, sizeof h, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "reading totals");
  stats->events = (int64_t)h[kStatEvents];
  stats->truncated = (int64_t)h[kStatTruncated];
  stats->overflowed = (int64_t)h[kStatOverflowed];
  stats->max_x = (int64_t)h[kStatMaxX];
  stats->kernel_ms = 0.0;
  stats->schedule = SSA_SCHED_THREAD;
  stats->handoffs = 0;
  if (h[kStatOverflowed] > 0) return record_error(SSA_EOVERFLOW, "a trajectory stopped at the int32 state limit");
  const long double bound = (long double)n_traj * (long double)h[kStatMaxX] * (long double)h[kStatMaxX];
  if (bound >= 9.2233720368547758e18L) return record_error(SSA_EOVERFLOW, "N * max_x^2 may exceed int64 sums");
  return SSA_OK;
}
