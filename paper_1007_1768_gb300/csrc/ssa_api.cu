// C ABI of libssa (include/ssa.h): argument checks, the host planner that
// compiles a model into device tables, launch planning and buffer handling.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ssa.h"
#include "ssa_internal.h"

using namespace ssa_impl;

namespace {

thread_local std::string g_last_error;

ssa_status fail(ssa_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

#define SSA_CUDA_TRY(expr)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return fail(SSA_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

constexpr int kMaxDevices = 64;

struct DeviceInfo {
  bool ready = false;
  int sms = 0;
  size_t smem_optin = 0;
};
std::mutex g_dev_mutex;
DeviceInfo g_dev[kMaxDevices];
// Library-owned stream-ordered pools (one per device, made on first use) that
// keep freed memory for the next call instead of returning it to the driver.
cudaMemPool_t g_pool[kMaxDevices] = {};

ssa_status device_info(int dev, DeviceInfo* out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SSA_EUNSUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  if (!g_dev[dev].ready) {
    cudaDeviceProp p;
    SSA_CUDA_TRY(cudaGetDeviceProperties(&p, dev));
    g_dev[dev].sms = p.multiProcessorCount;
    g_dev[dev].smem_optin = p.sharedMemPerBlockOptin;
    g_dev[dev].ready = true;
  }
  *out = g_dev[dev];
  return SSA_OK;
}

}  // namespace

// ------------------------------------------------------------------ model
struct ssa_model {
  int32_t S = 0, M = 0;
  std::vector<int32_t> R, P;
  std::vector<double> c;
  std::vector<int32_t> x0;
  // packed tables (host image of the device copy)
  std::vector<int32_t> rinfo, nu_ptr, nu_idx, nu_val, dep_ptr, dep_idx;
  std::vector<unsigned char> image;
  size_t off_c = 0, off_rinfo = 0, off_nu_ptr = 0, off_nu_idx = 0, off_nu_val = 0, off_x0 = 0, off_dep_ptr = 0,
         off_dep_idx = 0;
  SmallModel small = {};
  bool has_small = false;
  // rate modifiers (ssa_model_set_rate_modifier); mod_f[j] = -1 when none
  std::vector<int32_t> mod_f;
  std::vector<double> mod_k, mod_lo, mod_hi;
  bool has_mod = false;
  size_t off_mod_f = 0, off_mod_k = 0, off_mod_lo = 0, off_mod_hi = 0;
  std::mutex mu;
  void* dev_image[kMaxDevices] = {};
  // event-log records per trajectory seen by earlier ssa_ensemble_avg_xy
  // calls, by (t_end, precision, schedule, max_events); guarded by mu
  std::vector<LogSize> log_sizes;
};

namespace {

size_t put(std::vector<unsigned char>& img, const void* src, size_t bytes) {
  const size_t off = align_up(img.size(), 16);
  img.resize(off + bytes + 16);
  if (bytes) std::memcpy(img.data() + off, src, bytes);
  img.resize(off + bytes);
  return off;
}

// Host planner: reactant kinds, sparse net changes and the dependency graph
// (reactions whose propensity reads a species that reaction j changes).
void plan_model(ssa_model* m) {
  const int S = m->S, M = m->M;
  m->rinfo.resize(M);
  for (int j = 0; j < M; ++j) {
    int sp[2] = {0, 0}, ns = 0, order = 0;
    for (int s = 0; s < S; ++s) {
      const int r = m->R[(size_t)j * S + s];
      order += r;
      if (r > 0) sp[ns++] = s;
    }
    int32_t w;
    if (order == 0) w = rinfo_pack(kOrder0, 0, 0);
    else if (order == 1) w = rinfo_pack(kUni, sp[0], 0);
    else if (ns == 1) w = rinfo_pack(kDimer, sp[0], 0);
    else w = rinfo_pack(kBi, sp[0], sp[1]);
    m->rinfo[j] = w;
  }
  m->nu_ptr.assign(M + 1, 0);
  m->nu_idx.clear();
  m->nu_val.clear();
  std::vector<std::vector<int>> changes(M);
  for (int j = 0; j < M; ++j) {
    for (int s = 0; s < S; ++s) {
      const int v = m->P[(size_t)j * S + s] - m->R[(size_t)j * S + s];
      if (v != 0) {
        m->nu_idx.push_back(s);
        m->nu_val.push_back(v);
        changes[j].push_back(s);
      }
    }
    m->nu_ptr[j + 1] = (int32_t)m->nu_idx.size();
  }
  // readers[s] = reactions whose propensity reads species s
  std::vector<std::vector<int>> readers(S);
  for (int k = 0; k < M; ++k)
    for (int s = 0; s < S; ++s)
      if (m->R[(size_t)k * S + s] > 0 || (m->has_mod && m->mod_f[k] == s)) readers[s].push_back(k);
  m->dep_ptr.assign(M + 1, 0);
  m->dep_idx.clear();
  std::vector<char> mark(M, 0);
  for (int j = 0; j < M; ++j) {
    std::vector<int> deps;
    for (int s : changes[j])
      for (int k : readers[s])
        if (!mark[k]) {
          mark[k] = 1;
          deps.push_back(k);
        }
    for (int k : deps) mark[k] = 0;
    std::sort(deps.begin(), deps.end());
    for (int k : deps) m->dep_idx.push_back(k);
    m->dep_ptr[j + 1] = (int32_t)m->dep_idx.size();
  }
  // by-value tables of the thread kernel (plain mass action only)
  m->has_small = (M <= kSmallMax && S <= kSmallMax && !m->has_mod);
  if (m->has_small) {
    SmallModel& sm = m->small;
    std::memset(&sm, 0, sizeof sm);
    for (int j = 0; j < M; ++j) {
      sm.rinfo[j] = m->rinfo[j];
      std::memcpy(&sm.cbits[j], &m->c[j], 8);
      uint32_t mask = 0;
      for (int q = m->dep_ptr[j]; q < m->dep_ptr[j + 1]; ++q) mask |= 1u << m->dep_idx[q];
      sm.depmask[j] = mask;
      for (int s = 0; s < S; ++s) sm.nu[j * kSmallMax + s] = m->P[(size_t)j * S + s] - m->R[(size_t)j * S + s];
    }
    for (int s = 0; s < S; ++s) sm.x0[s] = m->x0[s];
  }
  std::vector<unsigned char>& img = m->image;
  img.clear();
  m->off_c = put(img, m->c.data(), sizeof(double) * M);
  m->off_rinfo = put(img, m->rinfo.data(), sizeof(int32_t) * M);
  m->off_nu_ptr = put(img, m->nu_ptr.data(), sizeof(int32_t) * (M + 1));
  m->off_nu_idx = put(img, m->nu_idx.data(), sizeof(int32_t) * m->nu_idx.size());
  m->off_nu_val = put(img, m->nu_val.data(), sizeof(int32_t) * m->nu_val.size());
  m->off_x0 = put(img, m->x0.data(), sizeof(int32_t) * S);
  m->off_dep_ptr = put(img, m->dep_ptr.data(), sizeof(int32_t) * (M + 1));
  m->off_dep_idx = put(img, m->dep_idx.data(), sizeof(int32_t) * m->dep_idx.size());
  if (m->has_mod) {
    m->off_mod_f = put(img, m->mod_f.data(), sizeof(int32_t) * M);
    m->off_mod_k = put(img, m->mod_k.data(), sizeof(double) * M);
    m->off_mod_lo = put(img, m->mod_lo.data(), sizeof(double) * M);
    m->off_mod_hi = put(img, m->mod_hi.data(), sizeof(double) * M);
  }
  img.resize(align_up(img.size(), 16));
}

// Device copy of the model tables on `dev` (made on first use, synchronously).
ssa_status model_on_device(const ssa_model* cm, int dev, DevModel* out) {
  ssa_model* m = const_cast<ssa_model*>(cm);
  std::lock_guard<std::mutex> lk(m->mu);
  if (!m->dev_image[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, m->image.size());
    if (e != cudaSuccess) return fail(SSA_ENOMEM, "cudaMalloc(model tables): %s", cudaGetErrorString(e));
    e = cudaMemcpy(p, m->image.data(), m->image.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      cudaFree(p);
      return fail(SSA_ECUDA, "cudaMemcpy(model tables): %s", cudaGetErrorString(e));
    }
    m->dev_image[dev] = p;
  }
  const unsigned char* b = static_cast<const unsigned char*>(m->dev_image[dev]);
  out->S = m->S;
  out->M = m->M;
  out->nnz = (int32_t)m->nu_idx.size();
  out->ndep = (int32_t)m->dep_idx.size();
  out->c = reinterpret_cast<const double*>(b + m->off_c);
  out->rinfo = reinterpret_cast<const int32_t*>(b + m->off_rinfo);
  out->nu_ptr = reinterpret_cast<const int32_t*>(b + m->off_nu_ptr);
  out->nu_idx = reinterpret_cast<const int32_t*>(b + m->off_nu_idx);
  out->nu_val = reinterpret_cast<const int32_t*>(b + m->off_nu_val);
  out->x0 = reinterpret_cast<const int32_t*>(b + m->off_x0);
  out->dep_ptr = reinterpret_cast<const int32_t*>(b + m->off_dep_ptr);
  out->dep_idx = reinterpret_cast<const int32_t*>(b + m->off_dep_idx);
  out->mod_f = m->has_mod ? reinterpret_cast<const int32_t*>(b + m->off_mod_f) : nullptr;
  out->mod_k = m->has_mod ? reinterpret_cast<const double*>(b + m->off_mod_k) : nullptr;
  out->mod_lo = m->has_mod ? reinterpret_cast<const double*>(b + m->off_mod_lo) : nullptr;
  out->mod_hi = m->has_mod ? reinterpret_cast<const double*>(b + m->off_mod_hi) : nullptr;
  return SSA_OK;
}

// Workspace layout (bytes, 256-aligned pieces).
struct Workspace {
  size_t counter, stats, pool, d1, d2, grid, pool_slots, mean, var, sum1, sum2, tev, thash, tflags, total;
};

Workspace workspace_layout(int S, int G, int64_t N, const ssa_run_opts& o) {
  Workspace w;
  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t at = p;
    p = align_up(p + bytes, 256);
    return at;
  };
  const size_t gs = (size_t)G * S;
  w.counter = take(8);
  w.stats = take(8 * kStatCount);
  w.pool = take(kPoolHeaderBytes);
  w.d1 = take(8 * gs);
  w.d2 = take(8 * gs);
  w.grid = take(8 * (size_t)G);
  w.pool_slots = take(kPoolSlotBytes);
  const bool host = o.memory == SSA_MEM_HOST;
  w.mean = host ? take(8 * gs) : 0;
  w.var = host ? take(8 * gs) : 0;
  w.sum1 = host ? take(8 * gs) : 0;
  w.sum2 = host ? take(8 * gs) : 0;
  w.tev = (host && o.traj_events) ? take(8 * (size_t)N) : 0;
  w.thash = (host && o.traj_hash) ? take(8 * (size_t)N) : 0;
  w.tflags = (host && o.traj_flags) ? take(4 * (size_t)N) : 0;
  w.total = p;
  return w;
}

ssa_status check_run_args(const ssa_model* m, int64_t n_traj, double t_end, int32_t n_grid, const ssa_run_opts& o) {
  if (!m) return fail(SSA_EINVAL, "model is NULL");
  if (n_traj < 1) return fail(SSA_EINVAL, "n_traj must be >= 1 (got %lld)", (long long)n_traj);
  if (!(t_end > 0.0) || !std::isfinite(t_end)) return fail(SSA_EINVAL, "t_end must be finite and > 0");
  if (n_grid < 1) return fail(SSA_EINVAL, "n_grid must be >= 1");
  if ((size_t)n_grid * (size_t)m->S > ((size_t)1 << 31)) return fail(SSA_EINVAL, "n_grid * n_species too large");
  if (o.precision != SSA_PREC_FP64 && o.precision != SSA_PREC_FP32) return fail(SSA_EINVAL, "bad precision");
  if (o.memory != SSA_MEM_HOST && o.memory != SSA_MEM_DEVICE) return fail(SSA_EINVAL, "bad memory kind");
  if (o.schedule < SSA_SCHED_AUTO || o.schedule > SSA_SCHED_WARP) return fail(SSA_EINVAL, "bad schedule");
  if (o.reduce < SSA_REDUCE_AUTO || o.reduce > SSA_REDUCE_GLOBAL) return fail(SSA_EINVAL, "bad reduce mode");
  if (o.block_threads < 0 || o.block_threads > 512 || (o.block_threads % 32) != 0)
    return fail(SSA_EINVAL, "block_threads must be 0 or a multiple of 32 up to 512");
  if (o.grid_blocks < 0) return fail(SSA_EINVAL, "grid_blocks must be >= 0");
  if (o.max_events > (int64_t)0xFFFFFFFFLL) return fail(SSA_EINVAL, "max_events must be below 2^32");
  if (o.stream_id > 0xFFFFFFFFULL) return fail(SSA_EINVAL, "stream_id must be below 2^32");
  return SSA_OK;
}

ssa_status check_host_grid(const double* grid, int32_t G, double t_end) {
  if (!(grid[0] >= 0.0)) return fail(SSA_EINVAL, "grid[0] must be >= 0");
  for (int32_t k = 1; k < G; ++k)
    if (!(grid[k] >= grid[k - 1])) return fail(SSA_EINVAL, "grid must be ascending (index %d)", k);
  if (!(grid[G - 1] <= t_end)) return fail(SSA_EINVAL, "grid[n_grid-1] must be <= t_end");
  return SSA_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

const char* ssa_status_string(ssa_status st) {
  switch (st) {
    case SSA_OK: return "ok";
    case SSA_EINVAL: return "invalid argument";
    case SSA_ENOMEM: return "out of memory";
    case SSA_ECUDA: return "CUDA error";
    case SSA_EOVERFLOW: return "count overflow";
    case SSA_ETRUNCATED: return "trajectory truncated";
    case SSA_ETIMEOUT: return "device wait timed out";
    case SSA_EUNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* ssa_last_error(void) { return g_last_error.c_str(); }

void ssa_run_opts_init(ssa_run_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof *o);
  o->precision = SSA_PREC_FP64;
  o->schedule = SSA_SCHED_AUTO;
  o->memory = SSA_MEM_HOST;
  o->reduce = SSA_REDUCE_AUTO;
  o->max_events = SSA_DEFAULT_MAX_EVENTS;
}

ssa_status ssa_model_create(int32_t S, int32_t M, const int32_t* R, const int32_t* P, const double* c,
                            const int32_t* x0, ssa_model** out) {
  g_last_error.clear();
  if (!out) return fail(SSA_EINVAL, "out is NULL");
  *out = nullptr;
  if (S < 1 || S > 32767) return fail(SSA_EINVAL, "n_species must be in 1..32767 (got %d)", S);
  if (M < 1 || M > (1 << 20)) return fail(SSA_EINVAL, "n_reactions must be in 1..2^20 (got %d)", M);
  if (!R || !P || !c || !x0) return fail(SSA_EINVAL, "a model array is NULL");
  for (int32_t j = 0; j < M; ++j) {
    int order = 0;
    for (int32_t s = 0; s < S; ++s) {
      const int32_t r = R[(size_t)j * S + s], p = P[(size_t)j * S + s];
      if (r < 0 || r > 2) return fail(SSA_EINVAL, "reactants[%d][%d] = %d not in 0..2", j, s, r);
      if (p < 0) return fail(SSA_EINVAL, "products[%d][%d] = %d < 0", j, s, p);
      order += r;
    }
    if (order > 2) return fail(SSA_EINVAL, "reaction %d has order %d > 2", j, order);
    if (!(c[j] >= 0.0) || !std::isfinite(c[j])) return fail(SSA_EINVAL, "rates[%d] must be finite and >= 0", j);
  }
  for (int32_t s = 0; s < S; ++s)
    if (x0[s] < 0) return fail(SSA_EINVAL, "x0[%d] = %d < 0", s, x0[s]);
  ssa_model* m = new (std::nothrow) ssa_model;
  if (!m) return fail(SSA_ENOMEM, "host allocation failed");
  m->S = S;
  m->M = M;
  m->R.assign(R, R + (size_t)M * S);
  m->P.assign(P, P + (size_t)M * S);
  m->c.assign(c, c + M);
  m->x0.assign(x0, x0 + S);
  plan_model(m);
  *out = m;
  return SSA_OK;
}

ssa_status ssa_model_set_rate_modifier(ssa_model* m, int32_t reaction, int32_t species, double slope, double lo,
                                       double hi) {
  g_last_error.clear();
  if (!m) return fail(SSA_EINVAL, "model is NULL");
  if (reaction < 0 || reaction >= m->M) return fail(SSA_EINVAL, "reaction %d out of range", reaction);
  if (species < -1 || species >= m->S) return fail(SSA_EINVAL, "species %d out of range", species);
  if (!std::isfinite(slope)) return fail(SSA_EINVAL, "slope must be finite");
  if (!(lo >= 0.0) || !std::isfinite(lo) || !(hi >= lo)) return fail(SSA_EINVAL, "need 0 <= lo <= hi (hi may be +inf)");
  std::lock_guard<std::mutex> lk(m->mu);
  if (!m->has_mod) {
    m->mod_f.assign(m->M, -1);
    m->mod_k.assign(m->M, 0.0);
    m->mod_lo.assign(m->M, 0.0);
    m->mod_hi.assign(m->M, 0.0);
  }
  m->mod_f[reaction] = species;
  m->mod_k[reaction] = slope;
  m->mod_lo[reaction] = lo;
  m->mod_hi[reaction] = hi;
  m->log_sizes.clear();
  m->has_mod = false;
  for (int j = 0; j < m->M; ++j)
    if (m->mod_f[j] >= 0) m->has_mod = true;
  if (!m->has_mod) {
    m->mod_f.clear();
    m->mod_k.clear();
    m->mod_lo.clear();
    m->mod_hi.clear();
  }
  // the device copies are stale: free them (made again at the next run)
  int prev = -1;
  cudaGetDevice(&prev);
  for (int d = 0; d < kMaxDevices; ++d) {
    if (m->dev_image[d]) {
      cudaSetDevice(d);
      cudaFree(m->dev_image[d]);
      m->dev_image[d] = nullptr;
    }
  }
  if (prev >= 0) cudaSetDevice(prev);
  plan_model(m);
  return SSA_OK;
}

ssa_status ssa_release_cached_memory(void) {
  g_last_error.clear();
  std::lock_guard<std::mutex> lk(g_dev_mutex);
  for (int d = 0; d < kMaxDevices; ++d) {
    if (g_pool[d]) SSA_CUDA_TRY(cudaMemPoolTrimTo(g_pool[d], 0));
  }
  return SSA_OK;
}

ssa_status ssa_finalize_sums(int64_t n_traj, int32_t n_grid, int32_t n_species, const int64_t* sum1,
                             const int64_t* sum2, double* mean, double* var) {
  g_last_error.clear();
  if (n_traj < 1) return fail(SSA_EINVAL, "n_traj must be >= 1 (got %lld)", (long long)n_traj);
  if (n_grid < 1 || n_species < 1) return fail(SSA_EINVAL, "n_grid and n_species must be >= 1");
  if (!sum1 || !sum2 || !mean || !var) return fail(SSA_EINVAL, "sum1, sum2, mean and var must not be NULL");
  const size_t n = (size_t)n_grid * (size_t)n_species;
  const double dN = (double)n_traj;
  const double den = dN * (double)(n_traj - 1);
  for (size_t q = 0; q < n; ++q) {
    mean[q] = (double)sum1[q] / dN;
    if (n_traj < 2) {
      var[q] = std::numeric_limits<double>::quiet_NaN();
    } else {
      // N sum2 - sum1^2 in 128 bits, one rounding to double, one division
      const __int128 num = (__int128)n_traj * (__int128)sum2[q] - (__int128)sum1[q] * (__int128)sum1[q];
      var[q] = (double)num / den;
    }
  }
  return SSA_OK;
}

void ssa_model_destroy(ssa_model* m) {
  if (!m) return;
  int prev = -1;
  cudaGetDevice(&prev);
  for (int d = 0; d < kMaxDevices; ++d) {
    if (m->dev_image[d]) {
      cudaSetDevice(d);
      cudaFree(m->dev_image[d]);
    }
  }
  if (prev >= 0) cudaSetDevice(prev);
  delete m;
}

ssa_status ssa_model_info(const ssa_model* m, int32_t* S, int32_t* M) {
  if (!m) return fail(SSA_EINVAL, "model is NULL");
  if (S) *S = m->S;
  if (M) *M = m->M;
  return SSA_OK;
}

ssa_status ssa_ensemble_workspace_size(const ssa_model* m, int64_t n_traj, int32_t n_grid, const ssa_run_opts* opts,
                                       size_t* bytes) {
  ssa_run_opts o;
  if (opts) o = *opts; else ssa_run_opts_init(&o);
  if (!m || !bytes || n_grid < 1 || n_traj < 1) return fail(SSA_EINVAL, "bad arguments to workspace_size");
  *bytes = workspace_layout(m->S, n_grid, n_traj, o).total;
  return SSA_OK;
}

ssa_status ssa_ensemble_run(const ssa_model* m, int64_t n_traj, double t_end, int32_t n_grid, const double* grid,
                            uint64_t seed, const ssa_run_opts* opts, double* mean, double* var, int64_t* sum1,
                            int64_t* sum2, ssa_run_stats* stats) {
  g_last_error.clear();
  ssa_run_opts o;
  if (opts) o = *opts; else ssa_run_opts_init(&o);
  ssa_status st = check_run_args(m, n_traj, t_end, n_grid, o);
  if (st != SSA_OK) return st;
  if (!mean || !var) return fail(SSA_EINVAL, "mean and var must not be NULL");
  const bool host = o.memory == SSA_MEM_HOST;
  if (grid && host) {
    st = check_host_grid(grid, n_grid, t_end);
    if (st != SSA_OK) return st;
  }
  const bool fp32 = o.precision == SSA_PREC_FP32;
  if (m->has_mod && (fp32 || o.schedule == SSA_SCHED_THREAD))
    return fail(SSA_EUNSUPPORTED, "models with rate modifiers run FP64 on the warp schedule");
  if (fp32) {
    if (o.schedule == SSA_SCHED_THREAD)
      return fail(SSA_EUNSUPPORTED, "the FP32-propensity mode runs on the warp schedule");
    for (int32_t j = 0; j < m->M; ++j)
      if (m->c[j] > 3.4028234663852886e38)
        return fail(SSA_EINVAL, "rates[%d] exceeds the binary32 range of the FP32-propensity mode", j);
  }
  // AUTO: one trajectory per thread when the network fits its registers
  // (FP64 mode), else one per warp
  const bool use_warp =
      o.schedule == SSA_SCHED_WARP || (o.schedule == SSA_SCHED_AUTO && (!m->has_small || fp32));
  if (!use_warp && !m->has_small)
    return fail(SSA_EUNSUPPORTED, "the thread schedule takes at most %d reactions and %d species", kThreadMaxM,
                kThreadMaxS);
  if (use_warp && warp_max_chunk(m->M) == 0)
    return fail(SSA_EUNSUPPORTED, "the warp schedule takes at most %d reactions", kWarpMaxM);
  const int64_t max_events = (o.max_events > 0) ? o.max_events : SSA_DEFAULT_MAX_EVENTS;

  int dev = 0;
  SSA_CUDA_TRY(cudaGetDevice(&dev));
  DeviceInfo di;
  st = device_info(dev, &di);
  if (st != SSA_OK) return st;
  DevModel dm;
  st = model_on_device(m, dev, &dm);
  if (st != SSA_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(o.cuda_stream);

  // launch shape
  const int S = m->S, G = n_grid;
  LaunchPlan plan;
  if (use_warp) {
    if (o.block_threads > 256) return fail(SSA_EINVAL, "the warp schedule takes at most 256 threads per CTA");
    plan.threads = o.block_threads ? o.block_threads : 256;
    plan.shared_d = false;
    plan.smem = warp_kernel_smem(m->M, S, (int)m->nu_idx.size(), plan.threads);
    if (plan.smem > di.smem_optin)
      return fail(SSA_EUNSUPPORTED, "the warp kernel needs %zu bytes of shared memory per CTA (%zu available)",
                  plan.smem, di.smem_optin);
    int per_sm = 0;
    SSA_CUDA_TRY(warp_kernel_prepare(m->M, fp32, plan.smem, plan.threads, &per_sm));
    if (per_sm < 1) return fail(SSA_EUNSUPPORTED, "the warp kernel cannot be resident with this shape");
    const int64_t want = (n_traj + plan.threads / 32 - 1) / (plan.threads / 32);
    const int64_t cap = (int64_t)di.sms * per_sm;
    plan.blocks = o.grid_blocks ? o.grid_blocks : (int)(want < cap ? want : cap);
  } else {
    if (const char* msg = plan_thread_launch(S, m->M, G, n_traj, di.sms, di.smem_optin, o.reduce, o.block_threads,
                                             o.grid_blocks, &plan, true))
      return fail(SSA_EINVAL, "%s", msg);
    SSA_CUDA_TRY(thread_kernel_set_smem(m->M, S, plan.shared_d, plan.smem));
  }

  // workspace
  const Workspace wl = workspace_layout(S, G, n_traj, o);
  unsigned char* ws = static_cast<unsigned char*>(o.workspace);
  bool own_ws = false;
  if (ws) {
    if (o.workspace_bytes < wl.total)
      return fail(SSA_EINVAL, "workspace of %zu bytes is smaller than the %zu needed", o.workspace_bytes, wl.total);
  } else {
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(&ws), wl.total, stream);
    if (e != cudaSuccess) return fail(SSA_ENOMEM, "workspace allocation: %s", cudaGetErrorString(e));
    own_ws = true;
  }
  auto release = [&]() {
    if (own_ws) cudaFreeAsync(ws, stream);
  };
#define SSA_RUN_TRY(expr)                                                                      \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      release();                                                                               \
      return fail(SSA_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_));                         \
    }                                                                                          \
  } while (0)

  SSA_RUN_TRY(cudaMemsetAsync(ws, 0, wl.grid, stream));  // counter, stats, hand-off counters, D1, D2
  const double* d_grid;
  double* ws_grid = reinterpret_cast<double*>(ws + wl.grid);
  if (!grid) {
    SSA_RUN_TRY(launch_uniform_grid(ws_grid, G, t_end, stream));
    d_grid = ws_grid;
  } else if (host) {
    SSA_RUN_TRY(cudaMemcpyAsync(ws_grid, grid, sizeof(double) * G, cudaMemcpyHostToDevice, stream));
    d_grid = ws_grid;
  } else {
    d_grid = grid;
  }

  RunArgs a;
  a.sm = m->small;
  a.m = dm;
  a.G = G;
  a.N = n_traj;
  a.traj_offset = o.traj_offset;
  a.seed = seed;
  a.seed_word = nullptr;
  a.stream_id = o.stream_id;
  a.max_events = max_events;
  a.t_end = t_end;
  a.grid = d_grid;
  a.D1 = reinterpret_cast<unsigned long long*>(ws + wl.d1);
  a.D2 = reinterpret_cast<unsigned long long*>(ws + wl.d2);
  a.counter = reinterpret_cast<unsigned long long*>(ws + wl.counter);
  a.pool = use_warp ? nullptr : reinterpret_cast<unsigned long long*>(ws + wl.pool);
  a.pool_slots = use_warp ? nullptr : reinterpret_cast<unsigned long long*>(ws + wl.pool_slots);
  a.stats = reinterpret_cast<unsigned long long*>(ws + wl.stats);
  a.traj_events = host ? (o.traj_events ? reinterpret_cast<int64_t*>(ws + wl.tev) : nullptr) : o.traj_events;
  a.traj_hash = host ? (o.traj_hash ? reinterpret_cast<uint64_t*>(ws + wl.thash) : nullptr) : o.traj_hash;
  a.traj_flags = host ? (o.traj_flags ? reinterpret_cast<int32_t*>(ws + wl.tflags) : nullptr) : o.traj_flags;
  a.device_totals = reinterpret_cast<unsigned long long*>(o.device_totals);
  const bool uniform = !grid || (host && host_grid_is_uniform(grid, G, t_end));
  a.grid_uniform = (uniform && G >= 2 && G <= (1 << 20) && t_end < 1e30) ? 1 : 0;
  a.grid_scale = (float)((double)(G - 1) / t_end);
  a.grid_margin = (float)((double)G * 0x1p-21);

  double* d_mean = host ? reinterpret_cast<double*>(ws + wl.mean) : mean;
  double* d_var = host ? reinterpret_cast<double*>(ws + wl.var) : var;
  int64_t* d_s1 = host ? (sum1 ? reinterpret_cast<int64_t*>(ws + wl.sum1) : nullptr) : sum1;
  int64_t* d_s2 = host ? (sum2 ? reinterpret_cast<int64_t*>(ws + wl.sum2) : nullptr) : sum2;

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  if (stats) {
    SSA_RUN_TRY(cudaEventCreate(&ev0));
    SSA_RUN_TRY(cudaEventCreate(&ev1));
    SSA_RUN_TRY(cudaEventRecord(ev0, stream));
  }
  if (o.sim_event_begin) SSA_RUN_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.sim_event_begin), stream));
  if (use_warp)
    SSA_RUN_TRY(launch_warp_kernel(a, fp32, plan.blocks, plan.threads, plan.smem, stream));
  else
    SSA_RUN_TRY(launch_thread_kernel(a, plan.blocks, plan.threads, plan.shared_d, plan.smem, stream));
  if (o.sim_event_end) SSA_RUN_TRY(cudaEventRecord(static_cast<cudaEvent_t>(o.sim_event_end), stream));
  SSA_RUN_TRY(launch_finalize(a.D1, a.D2, G, S, n_traj, dm.x0, d_mean, d_var, d_s1, d_s2, stream));
  if (stats) SSA_RUN_TRY(cudaEventRecord(ev1, stream));

  unsigned long long hstats[kStatCount] = {};
  const size_t gs = (size_t)G * S;
  if (host) {
    SSA_RUN_TRY(cudaMemcpyAsync(mean, d_mean, 8 * gs, cudaMemcpyDeviceToHost, stream));
    SSA_RUN_TRY(cudaMemcpyAsync(var, d_var, 8 * gs, cudaMemcpyDeviceToHost, stream));
    if (sum1) SSA_RUN_TRY(cudaMemcpyAsync(sum1, d_s1, 8 * gs, cudaMemcpyDeviceToHost, stream));
    if (sum2) SSA_RUN_TRY(cudaMemcpyAsync(sum2, d_s2, 8 * gs, cudaMemcpyDeviceToHost, stream));
    if (o.traj_events)
      SSA_RUN_TRY(cudaMemcpyAsync(o.traj_events, a.traj_events, 8 * (size_t)n_traj, cudaMemcpyDeviceToHost, stream));
    if (o.traj_hash)
      SSA_RUN_TRY(cudaMemcpyAsync(o.traj_hash, a.traj_hash, 8 * (size_t)n_traj, cudaMemcpyDeviceToHost, stream));
    if (o.traj_flags)
      SSA_RUN_TRY(cudaMemcpyAsync(o.traj_flags, a.traj_flags, 4 * (size_t)n_traj, cudaMemcpyDeviceToHost, stream));
  }
  const bool wait = host || stats;
  if (wait) SSA_RUN_TRY(cudaMemcpyAsync(hstats, a.stats, sizeof hstats, cudaMemcpyDeviceToHost, stream));
  release();
  if (!wait) return SSA_OK;
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(SSA_ECUDA, "cudaStreamSynchronize: %s", cudaGetErrorString(e));
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    stats->events = (int64_t)hstats[kStatEvents];
    stats->truncated = (int64_t)hstats[kStatTruncated];
    stats->overflowed = (int64_t)hstats[kStatOverflowed];
    stats->max_x = (int64_t)hstats[kStatMaxX];
    stats->kernel_ms = ms;
    stats->schedule = use_warp ? SSA_SCHED_WARP : SSA_SCHED_THREAD;
    stats->handoffs = (int64_t)hstats[kStatHandoffs];
  }
  if (hstats[kStatPoolError] > 0)
    return fail(SSA_ETIMEOUT, "%llu hand-off waits between warps ran out", hstats[kStatPoolError]);
  if (hstats[kStatOverflowed] > 0)
    return fail(SSA_EOVERFLOW, "%llu trajectories stopped at the int32 state limit", hstats[kStatOverflowed]);
  // sum x^2 over N trajectories must stay below 2^63
  const long double bound = (long double)n_traj * (long double)hstats[kStatMaxX] * (long double)hstats[kStatMaxX];
  if (bound >= 9.2233720368547758e18L)
    return fail(SSA_EOVERFLOW, "N * max_x^2 = %.3Le may exceed int64 sums", bound);
  return SSA_OK;
#undef SSA_RUN_TRY
}

}  // extern "C"

// ------------------------------------------------------------------ internal accessors
// Used by entry points defined in other translation units (ssa_noalloc.cu).
namespace ssa_impl {

ssa_status record_error(ssa_status st, const char* msg) { return fail(st, "%s", msg); }

int set_error(int status, const char* msg) { return (int)fail((ssa_status)status, "%s", msg); }

int model_device_tables(const ssa_model* m, int dev, DevModel* out) {
  if (dev < 0 || dev >= kMaxDevices) return (int)fail(SSA_EUNSUPPORTED, "device index %d out of range", dev);
  return (int)model_on_device(m, dev, out);
}

const double* model_rates(const ssa_model* m) { return m->c.data(); }

bool model_log_size_get(const ssa_model* m, const LogSize& key, double* per_traj) {
  ssa_model* mm = const_cast<ssa_model*>(m);
  std::lock_guard<std::mutex> lk(mm->mu);
  for (const LogSize& e : mm->log_sizes) {
    if (e.t_end == key.t_end && e.precision == key.precision && e.schedule == key.schedule &&
        e.max_events == key.max_events) {
      *per_traj = e.per_traj;
      return true;
    }
  }
  return false;
}

void model_log_size_put(const ssa_model* m, const LogSize& v) {
  ssa_model* mm = const_cast<ssa_model*>(m);
  std::lock_guard<std::mutex> lk(mm->mu);
  for (LogSize& e : mm->log_sizes) {
    if (e.t_end == v.t_end && e.precision == v.precision && e.schedule == v.schedule &&
        e.max_events == v.max_events) {
      e.per_traj = v.per_traj;
      return;
    }
  }
  if (mm->log_sizes.size() >= 16) mm->log_sizes.erase(mm->log_sizes.begin());
  mm->log_sizes.push_back(v);
}

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lk(g_dev_mutex);
    if (!g_pool[dev]) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof props);
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t np;
      if ((e = cudaMemPoolCreate(&np, &props)) != cudaSuccess) return e;
      unsigned long long keep = ~0ULL;
      if ((e = cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess) {
        cudaMemPoolDestroy(np);
        return e;
      }
      g_pool[dev] = np;
    }
    pool = g_pool[dev];
  }
  return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void clear_error() { g_last_error.clear(); }

bool model_small_copy(const ssa_model* m, SmallModelCopy* out) {
  if (!m || !out) return false;
  ssa_model* mm = const_cast<ssa_model*>(m);
  std::lock_guard<std::mutex> lk(mm->mu);
  out->S = m->S;
  out->M = m->M;
  out->has_small = m->has_small;
  out->has_mod = m->has_mod;
  out->small = m->small;
  return true;
}

bool model_image_view(const ssa_model* m, ModelImageView* v) {
  if (!m || !v) return false;
  v->S = m->S;
  v->M = m->M;
  v->nnz = (int32_t)m->nu_idx.size();
  v->ndep = (int32_t)m->dep_idx.size();
  v->image = m->image.data();
  v->bytes = m->image.size();
  v->off_c = m->off_c;
  v->off_rinfo = m->off_rinfo;
  v->off_nu_ptr = m->off_nu_ptr;
  v->off_nu_idx = m->off_nu_idx;
  v->off_nu_val = m->off_nu_val;
  v->off_x0 = m->off_x0;
  v->off_dep_ptr = m->off_dep_ptr;
  v->off_dep_idx = m->off_dep_idx;
  v->small = m->has_small ? &m->small : nullptr;
  v->has_mod = m->has_mod;
  return true;
}

}  // namespace ssa_impl
