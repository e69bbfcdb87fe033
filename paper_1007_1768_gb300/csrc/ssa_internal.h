// Internal structures shared by the C-ABI layer (ssa_api.cu) and the kernels.
#ifndef SSA_INTERNAL_H_
#define SSA_INTERNAL_H_

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace ssa_impl {

// Reaction kinds of a mass-action propensity h_j(x):
//   kOrder0: 1; kUni: x_a; kBi: x_a * x_b (a != b); kDimer: x_a (x_a - 1) / 2.
enum : int32_t { kOrder0 = 0, kUni = 1, kBi = 2, kDimer = 3 };

// rinfo word of one reaction: kind in bits 0..1, species a in 2..16, species b in 17..31.
__host__ __device__ inline int32_t rinfo_kind(int32_t w) { return w & 3; }
__host__ __device__ inline int32_t rinfo_a(int32_t w) { return (w >> 2) & 0x7FFF; }
__host__ __device__ inline int32_t rinfo_b(int32_t w) { return (int32_t)(((uint32_t)w >> 17) & 0x7FFF); }
inline int32_t rinfo_pack(int32_t kind, int32_t a, int32_t b) {
  return (int32_t)((uint32_t)kind | ((uint32_t)a << 2) | ((uint32_t)b << 17));
}

// Device copy of a model: one allocation, this layout (all 8-byte aligned):
//   double  c[M]
//   int32   rinfo[M]
//   int32   nu_ptr[M + 1]        CSR of the nonzero net changes per reaction
//   int32   nu_idx[nnz]          species
//   int32   nu_val[nnz]          change
//   int32   x0[S]
//   int32   dep_ptr[M + 1]       CSR: reactions whose propensity reads a species j changes
//   int32   dep_idx[ndep]
struct DevModel {
  int32_t S, M, nnz, ndep;
  const double* c;
  const int32_t* rinfo;
  const int32_t* nu_ptr;
  const int32_t* nu_idx;
  const int32_t* nu_val;
  const int32_t* x0;
  const int32_t* dep_ptr;
  const int32_t* dep_idx;
  // rate modifiers (null when the model has none): reaction j with
  // mod_f[j] >= 0 has rate min(max(c_j + mod_k[j] x_{mod_f[j]}, mod_lo[j]), mod_hi[j])
  const int32_t* mod_f;
  const double* mod_k;
  const double* mod_lo;
  const double* mod_hi;
};

// Slots of the per-run device totals.
enum { kStatEvents = 0, kStatTruncated = 1, kStatOverflowed = 2, kStatMaxX = 3, kStatPoolError = 4, kStatHandoffs = 5,
       kStatCount = 8 };

// Hand-off pool of the thread kernel.  In the cooperative tail a warp that
// still runs two or more trajectories passes one, between batches, to a warp
// that has none left (anywhere in the launch), so that the last long
// trajectories do not share a warp or an SM that others have left.  The pool
// is a ring of trajectory states with four counters, each on its own
// 128-byte line: registrations of waiting warps not yet claimed by a
// producer (avail), states taken (head), states claimed for writing (tail)
// and warps that may still hand off (multi); then one sequence word per
// slot (p + 1 once state p is written, p + 1 + 2^62 once it is read).  The
// counters and sequence words start at zero on every launch; the slots need
// no initialisation.
constexpr int kPoolSlots = 4096;
constexpr int kPoolSlotWords = 16;
constexpr int kPoolAvail = 0, kPoolHead = 16, kPoolTail = 32, kPoolMulti = 48, kPoolSeq = 64;
constexpr size_t kPoolHeaderBytes = 8 * (size_t)(kPoolSeq + kPoolSlots);      // counters + sequence words
constexpr size_t kPoolSlotBytes = 8 * (size_t)kPoolSlotWords * kPoolSlots;    // states

// Small-network tables passed by value to the thread kernel (M <= 16,
// S <= 16): reads with a per-reaction constant index come straight from the
// kernel's parameter space.
constexpr int kSmallMax = 16;
struct SmallModel {
  int32_t rinfo[kSmallMax];
  unsigned long long cbits[kSmallMax];   // rates as double bit patterns
  int32_t x0[kSmallMax];
  uint32_t depmask[kSmallMax];           // reactions to recompute after j fires
  int32_t nu[kSmallMax * kSmallMax];     // dense net change [j][s]
};

// Arguments of the simulation kernels.
struct RunArgs {
  SmallModel sm;
  DevModel m;
  int32_t G;
  int64_t N;
  uint64_t traj_offset;
  uint64_t seed;
  const unsigned long long* seed_word;  // device word holding the seed (batch graphs), or null: use seed
  uint64_t stream_id;
  int64_t max_events;
  double t_end;
  const double* grid;                 // [G]
  unsigned long long* D1;             // [G * S] per-grid sums of count changes (global)
  unsigned long long* D2;             // [G * S] per-grid sums of square changes (global)
  unsigned long long* counter;        // next trajectory index
  unsigned long long* pool = nullptr;  // hand-off counters and sequence words (zeroed), or null: no hand-off
  unsigned long long* pool_slots = nullptr;  // [kPoolSlots * kPoolSlotWords] hand-off states
  unsigned long long* stats;          // [kStatCount]
  int64_t* traj_events;               // [N] or null
  uint64_t* traj_hash;                // [N] or null
  int32_t* traj_flags;                // [N] or null
  unsigned long long* device_totals;  // [4] or null (caller's running totals)
  int32_t grid_uniform;               // grid is g_k = k t_end / (G - 1): index found by estimate + exact fix
  float grid_scale;                   // (G - 1) / t_end, for the estimate only
  float grid_margin;                  // estimates closer than this to an integer are checked against the grid
};

// Shared-memory layout of the thread-per-trajectory kernel (bytes): log
// cells, the dense net-change rows and dependency masks (read with the fired
// reaction's index), and the difference sums when they fit.
constexpr int kLogCells = 512;
struct ThreadSmem {
  size_t log_inv, log_lnf, nu, depmask, rmask, rinfo, cbits, d1, d2, total;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline ThreadSmem thread_smem_layout(int maxm, int maxs, int S, int G, bool shared_d) {
  ThreadSmem L;
  size_t o = 0;
  L.log_inv = o; o += kLogCells * 8;
  L.log_lnf = o; o += kLogCells * 8;
  L.nu = o; o += align_up((size_t)maxm * maxs * 4, 16);
  L.depmask = o; o += align_up((size_t)maxm * 4, 16);
  L.rmask = o; o += align_up((size_t)maxs * 4, 16);
  L.rinfo = o; o += align_up((size_t)maxm * 4, 16);
  L.cbits = o; o += align_up((size_t)maxm * 8, 16);
  if (shared_d) {
    L.d1 = o; o += (size_t)G * S * 8;
    L.d2 = o; o += (size_t)G * S * 8;
  } else {
    L.d1 = L.d2 = 0;
  }
  L.total = o;
  return L;
}

// True when a host grid is the uniform grid bit for bit,
// g_k = RN(RN(k t_end) / (G - 1)) (what k_uniform_grid writes), so the
// kernels may locate grid cells by the estimate of the uniform case.
inline bool host_grid_is_uniform(const double* g, int G, double t_end) {
  if (G < 2) return false;
  for (int k = 0; k < G; ++k) {
    const double v = ((double)k * t_end) / (double)(G - 1);
    if (!(g[k] == v)) return false;
  }
  return true;
}

// Template buckets of the thread kernel: M rounded up to an even number, S to 4, 8 or 16.
__host__ __device__ inline int bucket_m(int M) { return (M + 1) / 2 * 2; }
__host__ __device__ inline int bucket_s(int S) { return S <= 4 ? 4 : (S <= 8 ? 8 : 16); }

// Launch helpers (ssa_kernels.cu).  Return cudaSuccess or the launch error.
cudaError_t launch_thread_kernel(const RunArgs& a, int blocks, int threads, bool shared_d,
                                 size_t smem_bytes, cudaStream_t stream);
// per-S-bucket launchers (ssa_thread_s4.cu, ssa_thread_s8.cu, ssa_thread_s16.cu)
cudaError_t launch_thread_s4(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem, cudaStream_t st);
cudaError_t launch_thread_s8(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem, cudaStream_t st);
cudaError_t launch_thread_s16(const RunArgs& a, int blocks, int threads, bool shared_d, size_t smem, cudaStream_t st);
cudaError_t set_smem_s4(int M, bool shared_d, size_t smem);
cudaError_t set_smem_s8(int M, bool shared_d, size_t smem);
cudaError_t set_smem_s16(int M, bool shared_d, size_t smem);
// logging variants for the Avg-XY pipeline (ssa_thread_log_s{4,8,16}.cu)
struct EventLog;
cudaError_t launch_thread_log_s4(const RunArgs& a, const EventLog& lg, int blocks, int threads, size_t smem,
                                 cudaStream_t st);
cudaError_t launch_thread_log_s8(const RunArgs& a, const EventLog& lg, int blocks, int threads, size_t smem,
                                 cudaStream_t st);
cudaError_t launch_thread_log_s16(const RunArgs& a, const EventLog& lg, int blocks, int threads, size_t smem,
                                  cudaStream_t st);
cudaError_t set_smem_log_s4(int M, size_t smem);
cudaError_t set_smem_log_s8(int M, size_t smem);
cudaError_t set_smem_log_s16(int M, size_t smem);
// by S bucket (ssa_kernels.cu)
cudaError_t launch_thread_log_kernel(const RunArgs& a, const EventLog& lg, int blocks, int threads, size_t smem,
                                     cudaStream_t stream);
cudaError_t thread_log_kernel_set_smem(int M, int S, size_t smem);
cudaError_t launch_finalize(const unsigned long long* D1, const unsigned long long* D2, int G, int S,
                            int64_t N, const int32_t* x0, double* mean, double* var, int64_t* sum1,
                            int64_t* sum2, cudaStream_t stream);
cudaError_t launch_uniform_grid(double* grid, int G, double t_end, cudaStream_t stream);
// One network's finalisation inputs and outputs (device pointers).
struct FinalizeNet {
  const unsigned long long* D1;
  const unsigned long long* D2;
  const int32_t* x0;
  double* mean;
  double* var;
  int64_t* sum1;  // may be null
  int64_t* sum2;  // may be null
  int32_t G, S;
  int64_t N;
};
// Finalises n_nets networks in one launch: cta_begin[b] = sum of S over
// networks before b (n_nets + 1 entries, device), total_ctas = sum of S.
cudaError_t launch_finalize_batch(const FinalizeNet* nets, const int* cta_begin, int n_nets, int total_ctas,
                                  int max_G, cudaStream_t stream);
// Largest M and S the thread kernel is instantiated for.
constexpr int kThreadMaxM = 16;
constexpr int kThreadMaxS = 16;
cudaError_t thread_kernel_set_smem(int M, int S, bool shared_d, size_t smem_bytes);

// Event log of the warp kernel (selective memory along the time axis): one
// record per (kept event, species it changes), handed out in per-warp chunks.
constexpr int kLogChunk = 256;       // slots a warp of the warp kernel takes at a time
constexpr int kThreadLogChunk = 32;  // slots a lane of the thread kernel takes at a time
constexpr unsigned long long kLogSentinel = 0xFFFFFFFFFFFFFFFFULL;  // key of an unused slot
// What a record carries besides its time key (16 bytes: one load).
struct __align__(16) LogRec {
  int32_t species;
  int32_t change;  // v
  long long d2;    // (2 x_old + v) v
};
struct EventLog {
  unsigned long long* key;       // [capacity] bits of the event time
  LogRec* rec;                   // [capacity]
  unsigned long long* counter;   // slots handed out (in chunks)
  unsigned long long* padded;    // unused slots (sentinel keys)
  unsigned long long* overflow;  // nonzero when the capacity ran out
  unsigned long long* needed;    // records of every event, written or not (sized a retry)
  unsigned long long capacity;
};

// Warp-per-trajectory kernel (ssa_warp_kernel.cu), schedule W32.  Chunk
// bound of the instantiation serving M reactions (0 when M > 512).
int warp_max_chunk(int M);
constexpr int kWarpMaxM = 512;
// Dynamic shared memory of one CTA of `threads` threads.
size_t warp_kernel_smem(int M, int S, int nnz, int threads);
// Sets the kernel's shared-memory limit and reports resident CTAs per SM.
// fp32 selects the FP32-propensity instantiation.
cudaError_t warp_kernel_prepare(int M, bool fp32, size_t smem, int threads, int* blocks_per_sm);
cudaError_t launch_warp_kernel(const RunArgs& a, bool fp32, int blocks, int threads, size_t smem,
                               cudaStream_t stream);
// The same kernel writing the event log.
cudaError_t warp_log_kernel_prepare(int M, bool fp32, size_t smem, int threads, int* blocks_per_sm);
cudaError_t launch_warp_log_kernel(const RunArgs& a, const EventLog& lg, bool fp32, int blocks, int threads,
                                   size_t smem, cudaStream_t stream);

// Host image of a model's device tables (see DevModel for the layout), for
// entry points that place the tables themselves.
struct ModelImageView {
  int32_t S, M, nnz, ndep;
  const unsigned char* image;
  size_t bytes;
  size_t off_c, off_rinfo, off_nu_ptr, off_nu_idx, off_nu_val, off_x0, off_dep_ptr, off_dep_idx;
  const SmallModel* small;  // filled when M <= 16, S <= 16 and no rate modifiers
  bool has_mod;             // rate modifiers present (warp schedule, FP64 only)
};

// Launch shape of the thread kernel.
struct LaunchPlan {
  int blocks, threads;
  bool shared_d;
  size_t smem;
};

// Chooses the launch shape: threads per CTA from the trajectories per SM
// (64..512, multiples of 32) unless given.  With hand-off between warps
// (`handoff`), more than 256 trajectories per SM take full 512-thread CTAs,
// at least one per SM: the warps left without a trajectory wait for handed-off
// ones from the start.  The difference sums go to global
// memory by default (fire-and-forget reductions that never stall a warp,
// measured faster than shared-memory atomics here); SSA_REDUCE_SHARED stages
// them per CTA in shared memory instead.
// Returns nullptr or an error message.
inline const char* plan_thread_launch(int S, int M, int G, int64_t N, int sms, size_t smem_optin, int reduce,
                                      int block_threads, int grid_blocks, LaunchPlan* p, bool handoff = false) {
  int threads = block_threads;
  const int64_t per_sm = (N + sms - 1) / sms;
  if (threads == 0) {
    const int64_t t = (per_sm + 31) / 32 * 32;
    threads = (int)(t < 64 ? 64 : (t > 512 ? 512 : t));
    if (handoff && per_sm > 256) threads = 512;
  }
  const int mb = bucket_m(M), sb = bucket_s(S);
  const ThreadSmem sh = thread_smem_layout(mb, sb, S, G, true);
  bool shared_d;
  if (reduce == 1) {  // SSA_REDUCE_SHARED
    if (sh.total > smem_optin) return "the difference sums do not fit in shared memory";
    shared_d = true;
  } else if (reduce == 2) {  // SSA_REDUCE_GLOBAL
    shared_d = false;
  } else {
    shared_d = false;
  }
  const ThreadSmem lay = shared_d ? sh : thread_smem_layout(mb, sb, S, G, false);
  int blocks = grid_blocks;
  if (blocks == 0) {
    const int64_t want = (N + threads - 1) / threads;
    int ctas_per_sm = 1;
    if (!shared_d) {
      ctas_per_sm = (int)(smem_optin / (lay.total > 0 ? lay.total : 1));
      ctas_per_sm = ctas_per_sm < 1 ? 1 : (ctas_per_sm > 4 ? 4 : ctas_per_sm);
    }
    const int64_t cap = (int64_t)sms * ctas_per_sm;
    blocks = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    if (handoff && block_threads == 0 && blocks < sms) blocks = sms;
  }
  p->blocks = blocks;
  p->threads = threads;
  p->shared_d = shared_d;
  p->smem = lay.total;
  return nullptr;
}

}  // namespace ssa_impl

struct ssa_model;

namespace ssa_impl {
// Event-log records per trajectory of an earlier Avg-XY call, by its key.
struct LogSize {
  double t_end;
  int32_t precision, schedule;
  int64_t max_events;
  double per_traj;
};
// Accessors implemented in ssa_api.cu.
bool model_log_size_get(const ssa_model* m, const LogSize& key, double* per_traj);
void model_log_size_put(const ssa_model* m, const LogSize& v);
// Stream-ordered allocation from the library's pool on the current device
// (freed memory stays in the pool for the next call; cudaFreeAsync frees,
// ssa_release_cached_memory returns it to the driver).
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st);
bool model_image_view(const ssa_model* m, ModelImageView* v);
// A copy of a model's sizes and small tables, taken under the model's lock.
struct SmallModelCopy {
  int32_t S, M;
  bool has_small;  // M <= 16 and S <= 16 and no rate modifiers: `small` is filled
  bool has_mod;    // rate modifiers present
  SmallModel small;
};
bool model_small_copy(const ssa_model* m, SmallModelCopy* out);
// The model's device tables on `dev` (copied there on first use); returns
// SSA_OK or an error status with the thread's message set.
int model_device_tables(const ssa_model* m, int dev, DevModel* out);
// Rates of the model (host copy, [M]).
const double* model_rates(const ssa_model* m);
// Sets the calling thread's error message and returns `status`.
int set_error(int status, const char* msg);
}  // namespace ssa_impl

#endif  // SSA_INTERNAL_H_
