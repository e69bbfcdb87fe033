// Batched ensembles (include/ssa.h, ssa_batch_*): many networks of uneven
// size and trajectory count -- the parametric copies and sweeps of Sec. 3.2
// (StochRxn_ff) -- in persistent launches captured once in a CUDA graph.
//
// Layout.  Every network of the batch gets, in one device slab: its grid,
// its difference sums D1 / D2, its results (mean, var, sum1, sum2), its
// per-lane dependency bits and binary32 rates; a descriptor table (one
// BatchNetDev per network, in launch order) points at these and at the
// model's own device tables.  Trajectory work items are numbered network
// after network in launch order; work_begin[p] is the first item of the
// network at position p.
//
// Launches.  Networks are ordered by descending chunk bucket (ceil(M / 32)
// rounded to 1, 2, 4, 8, 16), then by descending M: the costliest steps
// first.  "Split" grouping runs one
// persistent kernel per bucket (register use fits the bucket), the kernels
// on parallel graph branches so that CTAs of one fill the SMs the tail of
// another frees; "single" grouping runs one kernel for all networks at the
// largest bucket.  A warp takes the next item from its launch's counter,
// finds the item's network by binary search over work_begin, and runs the
// trajectory with the same step as the single-network warp kernel
// (ssa_warp_step.cuh).  Results do not depend on the grouping, the block
// size or the order: each trajectory is fixed by (seed, id, stream id) and
// the sums are integers.
//
// Graph.  memset of the counters, sums and stats; the simulation kernels;
// one batched finalisation kernel.  The seed is read from device memory,
// written by a one-thread kernel enqueued before each replay, so one graph
// serves every seed.
//
// Autotuner (ssa_batch_tune).  Times every candidate launch shape -- block
// size 64, 128 or 256 threads, split or single grouping -- on a sample of
// the batch (the first ceil(N_b / 8) trajectories of every network, a fixed
// seed), keeps the fastest and re-captures at the next launch.
#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "ssa.h"
#include "ssa_internal.h"
#include "ssa_warp_step.cuh"

namespace ssa_impl {
namespace {

struct BatchNetDev {
  WarpNet net;
  long long N;
};

struct BatchLaunch {
  const BatchNetDev* nets;         // by position
  const long long* work_begin;     // by position, n + 1 entries
  int pos_lo, pos_hi;              // positions this launch serves
  unsigned long long* counter;
  unsigned long long* stats;       // [n * 4] by position: events, truncated, overflowed, max x
  const unsigned long long* seed;  // device word
  unsigned long long traj_offset;
  long long max_events;
  int smax;                        // largest S of the launch (per-warp state slots)
};

// FP32 instantiations are held to 85 registers (three CTAs of 256 threads per
// SM): more resident warps hide the step's latencies better than the
// registers it gives up (measured on the uneven 256-network batch: 1.71 ->
// 1.55 s per step at 1/16 of its trajectories); FP64 ones keep 128.
template <int MAXCH, bool F32>
__global__ void __launch_bounds__(256, F32 ? 3 : 2) k_ssa_batch(const BatchLaunch L) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* s_inv = reinterpret_cast<uint64_t*>(smem);
  uint64_t* s_lnf = s_inv + kLogCells;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int32_t* xs = reinterpret_cast<int32_t*>(s_lnf + kLogCells) + (size_t)warp * L.smax;
  // per-warp pre-event counts of a batch, after every warp's state slots
  int32_t* xrec = reinterpret_cast<int32_t*>(reinterpret_cast<unsigned char*>(s_lnf + kLogCells) +
                                             align_up((size_t)(blockDim.x >> 5) * L.smax * 4, 16)) +
                  (size_t)warp * 32 * kRecPerEvent;
  for (int i = tid; i < kLogCells; i += blockDim.x) {
    s_inv[i] = d_log_tables.inv[i];
    s_lnf[i] = d_log_tables.lnf[i];
  }
  __syncthreads();
  const unsigned long long seed = *L.seed;
  const uint32_t key0 = (uint32_t)seed, key1 = (uint32_t)(seed >> 32);
  const long long first = L.work_begin[L.pos_lo], end = L.work_begin[L.pos_hi];
  for (;;) {
    unsigned long long next = 0;
    if (lane == 0) next = atomicAdd(L.counter, 1ULL);
    next = __shfl_sync(kFullMask, next, 0);
    const long long item = first + (long long)next;
    if (item >= end) break;
    int lo = L.pos_lo, hi = L.pos_hi;  // last position p with work_begin[p] <= item
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (L.work_begin[mid] <= item) lo = mid; else hi = mid;
    }
    const WarpNet net = L.nets[lo].net;
    const unsigned long long id = L.traj_offset + (unsigned long long)(item - L.work_begin[lo]);
    const WarpTraj r = warp_trajectory<MAXCH, F32>(net, xs, xrec, id, key0, key1, L.max_events, s_inv, s_lnf);
    if (lane == 0) {
      unsigned long long* st = L.stats + (size_t)lo * 4;
      atomicAdd(st + 0, (unsigned long long)r.n);
      if (r.flags & kWarpFlagTruncated) atomicAdd(st + 1, 1ULL);
      if (r.flags & kWarpFlagOverflow) atomicAdd(st + 2, 1ULL);
      atomicMax(st + 3, (unsigned long long)r.maxx);
    }
    __syncwarp();
  }
}

__global__ void k_set_word(unsigned long long* p, unsigned long long v) { *p = v; }

// The most species any reaction of a model changes (from its host tables).
int model_nnz_max(const ssa_model* m) {
  ModelImageView mv;
  if (!model_image_view(m, &mv)) return 1 << 30;
  const int32_t* ptr = reinterpret_cast<const int32_t*>(mv.image + mv.off_nu_ptr);
  int mx = 0;
  for (int j = 0; j < mv.M; ++j) mx = std::max(mx, ptr[j + 1] - ptr[j]);
  return mx;
}

// Per-network tables the batch derives on the device: dependency bits for
// the warp layout and the binary32 rates.
__global__ void k_batch_tables(const DevModel m, uint16_t* depw, float* c32) {
  const int ch = (m.M + 31) / 32;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.M * 32; i += gridDim.x * blockDim.x) {
    depw[i] = depw_entry(m.dep_ptr, m.dep_idx, ch, i >> 5, i & 31);
    if ((i & 31) == 0) c32[i >> 5] = __double2float_rn(m.c[i >> 5]);
  }
}

template <int MAXCH, bool F32>
cudaError_t launch_batch_ch(const BatchLaunch& L, int blocks, int threads, size_t smem, cudaStream_t st) {
  k_ssa_batch<MAXCH, F32><<<blocks, threads, smem, st>>>(L);
  return cudaGetLastError();
}

template <int MAXCH, bool F32>
cudaError_t prepare_batch_ch(size_t smem, int threads, int* per_sm) {
  cudaError_t e =
      cudaFuncSetAttribute(k_ssa_batch<MAXCH, F32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_ssa_batch<MAXCH, F32>, threads, smem);
}

template <bool F32>
cudaError_t batch_dispatch(int bucket, bool launch, const BatchLaunch* L, int blocks, int threads, size_t smem,
                           cudaStream_t st, int* per_sm) {
  switch (bucket) {
    case 1: return launch ? launch_batch_ch<1, F32>(*L, blocks, threads, smem, st)
                          : prepare_batch_ch<1, F32>(smem, threads, per_sm);
    case 2: return launch ? launch_batch_ch<2, F32>(*L, blocks, threads, smem, st)
                          : prepare_batch_ch<2, F32>(smem, threads, per_sm);
    case 4: return launch ? launch_batch_ch<4, F32>(*L, blocks, threads, smem, st)
                          : prepare_batch_ch<4, F32>(smem, threads, per_sm);
    case 8: return launch ? launch_batch_ch<8, F32>(*L, blocks, threads, smem, st)
                          : prepare_batch_ch<8, F32>(smem, threads, per_sm);
    case 16: return launch ? launch_batch_ch<16, F32>(*L, blocks, threads, smem, st)
                           : prepare_batch_ch<16, F32>(smem, threads, per_sm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t batch_kernel(bool fp32, int bucket, bool launch, const BatchLaunch* L, int blocks, int threads,
                         size_t smem, cudaStream_t st, int* per_sm) {
  return fp32 ? batch_dispatch<true>(bucket, launch, L, blocks, threads, smem, st, per_sm)
              : batch_dispatch<false>(bucket, launch, L, blocks, threads, smem, st, per_sm);
}

size_t batch_smem(int threads, int smax) {
  return (size_t)kLogCells * 16 + align_up((size_t)(threads / 32) * smax * 4, 16) +
         (size_t)(threads / 32) * 32 * kRecPerEvent * 4;
}

}  // namespace
}  // namespace ssa_impl

using namespace ssa_impl;

struct ssa_batch {
  int n = 0;
  int dev = 0, sms = 0;
  bool fp32 = false;
  ssa_run_opts opts{};
  std::vector<const ssa_model*> models;
  std::vector<int64_t> N;
  std::vector<int32_t> G, S, M;
  std::vector<double> t_end;
  std::vector<int> order;  // position -> network index (warp-schedule networks first)
  std::vector<int> pos;    // network index -> position
  // schedules (SSA_SCHED_THREAD / SSA_SCHED_WARP) by network index; networks
  // that fit the thread kernel (FP64, at most 16 reactions and species, no
  // rate modifiers) may take either, which ssa_batch_tune decides by timing
  // unless opts->schedule fixed it
  std::vector<int> sched;
  std::vector<char> thread_ok;
  bool sched_fixed = false;
  int n_warp = 0;          // positions [0, n_warp) run on the warp schedule
  int smem_optin = 0;
  // per network index: the warp layout's descriptor and finalisation entry
  // (slab pointers), the device tables and the small-network tables
  std::vector<WarpNet> wnets;
  std::vector<FinalizeNet> fnets;
  std::vector<DevModel> dms;
  std::vector<SmallModelCopy> smalls;
  // thread-schedule networks by position - n_warp: launch arguments for the
  // full run and for the tuner's sample, with their launch shapes
  struct ThreadNet {
    RunArgs full, sample;
    LaunchPlan plan_full, plan_sample;
  };
  std::vector<ThreadNet> tnets;
  // device slab and the offsets of each network's pieces (by network index)
  unsigned char* slab = nullptr;
  std::vector<size_t> off_grid, off_d1, off_d2, off_mean, off_var, off_s1, off_s2, off_depw, off_c32;
  size_t off_nets = 0, off_fin = 0, off_cta = 0, off_work = 0, off_work_sample = 0, off_counters = 0,
         off_stats = 0, off_seed = 0, zero_begin = 0, zero_bytes = 0;
  static constexpr int kGroupCounters = 32;  // counters of the warp groups; thread networks follow
  int total_ctas = 0, max_G = 0;
  // launch plan
  int threads = 128;
  bool split = true;
  double tuned_ms = 0.0;
  struct Group {
    int bucket, pos_lo, pos_hi, smax, blocks;
    size_t smem;
  };
  std::vector<Group> groups;
  // graph
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> forks;
  std::vector<cudaEvent_t> evs;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  std::vector<unsigned long long> host_stats;
};

namespace {

#define SSA_B_TRY(expr)                                                           \
  do {                                                                            \
    cudaError_t e_ = (expr);                                                      \
    if (e_ != cudaSuccess) return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

int bucket_of(int M) { return warp_max_chunk(M); }

// Plans the groups for the current (threads, split) choice.
ssa_status plan_groups(ssa_batch* b) {
  b->groups.clear();
  auto add = [&](int bucket, int lo, int hi) -> ssa_status {
    ssa_batch::Group g;
    g.bucket = bucket;
    g.pos_lo = lo;
    g.pos_hi = hi;
    g.smax = 1;
    for (int p = lo; p < hi; ++p) g.smax = std::max(g.smax, b->S[b->order[p]]);
    g.smem = batch_smem(b->threads, g.smax);
    int per_sm = 0;
    cudaError_t e = batch_kernel(b->fp32, bucket, false, nullptr, 0, b->threads, g.smem, nullptr, &per_sm);
    if (e != cudaSuccess) return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
    if (per_sm < 1) return (ssa_status)set_error(SSA_EUNSUPPORTED, "batch kernel cannot be resident with this shape");
    g.blocks = b->sms * per_sm;
    b->groups.push_back(g);
    return SSA_OK;
  };
  // warp-schedule networks only (positions [0, n_warp))
  const int nw = b->n_warp;
  if (nw == 0) return SSA_OK;
  if (b->split) {
    int p = 0;
    while (p < nw) {
      const int bk = bucket_of(b->M[b->order[p]]);
      int q = p;
      while (q < nw && bucket_of(b->M[b->order[q]]) == bk) ++q;
      const ssa_status st = add(bk, p, q);
      if (st != SSA_OK) return st;
      p = q;
    }
  } else {
    int bk = 1;
    for (int p = 0; p < nw; ++p) bk = std::max(bk, bucket_of(b->M[b->order[p]]));
    const ssa_status st = add(bk, 0, nw);
    if (st != SSA_OK) return st;
  }
  return SSA_OK;
}

// Enqueues one full pass (zeroing, simulation, finalisation) on `st`: the
// warp groups and the thread-schedule networks each on a fork stream.
// sample: the tuner's sample (the first ceil(N / 8) trajectories of each
// network, no finalisation).
ssa_status enqueue_pass(ssa_batch* b, cudaStream_t st, bool sample) {
  unsigned char* s = b->slab;
  SSA_B_TRY(cudaMemsetAsync(s + b->zero_begin, 0, b->zero_bytes, st));
  const int ng = (int)b->groups.size();
  const int nt = (int)b->tnets.size();
  SSA_B_TRY(cudaEventRecord(b->evs[0], st));
  for (int t = 0; t < nt; ++t) {
    const ssa_batch::ThreadNet& tn = b->tnets[t];
    const LaunchPlan& pl = sample ? tn.plan_sample : tn.plan_full;
    cudaStream_t fs = b->forks[ng + t];
    SSA_B_TRY(cudaStreamWaitEvent(fs, b->evs[0], 0));
    SSA_B_TRY(launch_thread_kernel(sample ? tn.sample : tn.full, pl.blocks, pl.threads, false, pl.smem, fs));
    SSA_B_TRY(cudaEventRecord(b->evs[1 + ng + t], fs));
    SSA_B_TRY(cudaStreamWaitEvent(st, b->evs[1 + ng + t], 0));
  }
  for (int g = 0; g < ng; ++g) {
    const ssa_batch::Group& gr = b->groups[g];
    cudaStream_t fs = b->forks[g];
    SSA_B_TRY(cudaStreamWaitEvent(fs, b->evs[0], 0));
    BatchLaunch L;
    L.nets = reinterpret_cast<const BatchNetDev*>(s + b->off_nets);
    L.work_begin = reinterpret_cast<const long long*>(s + (sample ? b->off_work_sample : b->off_work));
    L.pos_lo = gr.pos_lo;
    L.pos_hi = gr.pos_hi;
    L.counter = reinterpret_cast<unsigned long long*>(s + b->off_counters) + g;
    L.stats = reinterpret_cast<unsigned long long*>(s + b->off_stats);
    L.seed = reinterpret_cast<const unsigned long long*>(s + b->off_seed);
    L.traj_offset = b->opts.traj_offset;
    L.max_events = b->opts.max_events;
    L.smax = gr.smax;
    SSA_B_TRY(batch_kernel(b->fp32, gr.bucket, true, &L, gr.blocks, b->threads, gr.smem, fs, nullptr));
    SSA_B_TRY(cudaEventRecord(b->evs[1 + g], fs));
    SSA_B_TRY(cudaStreamWaitEvent(st, b->evs[1 + g], 0));
  }
  if (!sample)
    SSA_B_TRY(launch_finalize_batch(reinterpret_cast<const FinalizeNet*>(s + b->off_fin),
                                    reinterpret_cast<const int*>(s + b->off_cta), b->n, b->total_ctas, b->max_G, st));
  return SSA_OK;
}

ssa_status ensure_streams(ssa_batch* b) {
  const size_t need = b->groups.size() + b->tnets.size();
  if (!b->cap) SSA_B_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  while (b->forks.size() < need) {
    cudaStream_t f;
    SSA_B_TRY(cudaStreamCreateWithFlags(&f, cudaStreamNonBlocking));
    b->forks.push_back(f);
  }
  while (b->evs.size() < need + 1) {
    cudaEvent_t e;
    SSA_B_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->evs.push_back(e);
  }
  return SSA_OK;
}

void drop_graph(ssa_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

ssa_status capture(ssa_batch* b) {
  drop_graph(b);
  ssa_status st = ensure_streams(b);
  if (st != SSA_OK) return st;
  SSA_B_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  st = enqueue_pass(b, b->cap, false);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (st != SSA_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
  b->graph = g;
  SSA_B_TRY(cudaGraphInstantiate(&b->exec, g, 0));
  return SSA_OK;
}

// Writes the seed word the graph's kernels read (a one-thread launch: its
// argument is captured at launch, so nothing on the host must outlive it).
ssa_status set_seed(ssa_batch* b, uint64_t seed, cudaStream_t st) {
  k_set_word<<<1, 1, 0, st>>>(reinterpret_cast<unsigned long long*>(b->slab + b->off_seed), seed);
  SSA_B_TRY(cudaGetLastError());
  return SSA_OK;
}

// The thread-schedule launches of network i (full run and the tuner's
// sample), with the counter kGroupCounters + p and the stats slot of
// position p, and their launch shapes.
ssa_status thread_net(ssa_batch* b, int i, int p, ssa_batch::ThreadNet* tn) {
  const int div = 8;
  unsigned char* s = b->slab;
  const WarpNet& w = b->wnets[i];
  RunArgs& a = tn->full;
  a.sm = b->smalls[i].small;
  a.m = b->dms[i];
  a.G = b->G[i];
  a.N = b->N[i];
  a.traj_offset = b->opts.traj_offset;
  a.seed = 0;
  a.seed_word = reinterpret_cast<const unsigned long long*>(s + b->off_seed);
  a.stream_id = b->opts.stream_id + (uint64_t)i;
  a.max_events = b->opts.max_events;
  a.t_end = b->t_end[i];
  a.grid = w.grid;
  a.D1 = w.D1;
  a.D2 = w.D2;
  a.counter = reinterpret_cast<unsigned long long*>(s + b->off_counters) + ssa_batch::kGroupCounters + p;
  a.stats = reinterpret_cast<unsigned long long*>(s + b->off_stats) + 4 * (size_t)p;
  a.traj_events = nullptr;
  a.traj_hash = nullptr;
  a.traj_flags = nullptr;
  a.device_totals = nullptr;
  a.grid_uniform = w.grid_uniform;
  a.grid_scale = w.grid_scale;
  a.grid_margin = w.grid_margin;
  tn->sample = a;
  tn->sample.N = (b->N[i] + div - 1) / div;
  const char* msg = plan_thread_launch(b->S[i], b->M[i], b->G[i], tn->full.N, b->sms, (size_t)b->smem_optin,
                                       SSA_REDUCE_GLOBAL, 0, 0, &tn->plan_full);
  if (!msg)
    msg = plan_thread_launch(b->S[i], b->M[i], b->G[i], tn->sample.N, b->sms, (size_t)b->smem_optin,
                             SSA_REDUCE_GLOBAL, 0, 0, &tn->plan_sample);
  if (msg) return (ssa_status)set_error(SSA_EUNSUPPORTED, msg);
  SSA_B_TRY(thread_kernel_set_smem(b->M[i], b->S[i], false, std::max(tn->plan_full.smem, tn->plan_sample.smem)));
  return SSA_OK;
}

// Device time of network i's sample on one schedule alone (the second of two
// passes; the first warms up), on the capture stream.
ssa_status time_schedule(ssa_batch* b, int i, bool thread, double* ms_out) {
  const int p = b->pos[i];
  unsigned char* s = b->slab;
  ssa_batch::ThreadNet tn;
  BatchLaunch L;
  int blocks = 0;
  size_t smem = 0;
  if (thread) {
    const ssa_status st = thread_net(b, i, p, &tn);
    if (st != SSA_OK) return st;
  } else {
    L.nets = reinterpret_cast<const BatchNetDev*>(s + b->off_nets);
    L.work_begin = reinterpret_cast<const long long*>(s + b->off_work_sample);
    L.pos_lo = p;
    L.pos_hi = p + 1;
    L.counter = reinterpret_cast<unsigned long long*>(s + b->off_counters) + (ssa_batch::kGroupCounters - 1);
    L.stats = reinterpret_cast<unsigned long long*>(s + b->off_stats);
    L.seed = reinterpret_cast<const unsigned long long*>(s + b->off_seed);
    L.traj_offset = b->opts.traj_offset;
    L.max_events = b->opts.max_events;
    L.smax = std::max(1, b->S[i]);
    smem = batch_smem(b->threads, L.smax);
    int per_sm = 0;
    SSA_B_TRY(batch_kernel(b->fp32, bucket_of(b->M[i]), false, nullptr, 0, b->threads, smem, nullptr, &per_sm));
    if (per_sm < 1) return (ssa_status)set_error(SSA_EUNSUPPORTED, "batch kernel cannot be resident with this shape");
    blocks = b->sms * per_sm;
  }
  float ms = 0.f;
  for (int rep = 0; rep < 2; ++rep) {
    SSA_B_TRY(cudaMemsetAsync(s + b->zero_begin, 0, b->zero_bytes, b->cap));
    SSA_B_TRY(cudaEventRecord(b->t0, b->cap));
    if (thread) {
      SSA_B_TRY(launch_thread_kernel(tn.sample, tn.plan_sample.blocks, tn.plan_sample.threads, false,
                                     tn.plan_sample.smem, b->cap));
    } else {
      SSA_B_TRY(batch_kernel(b->fp32, bucket_of(b->M[i]), true, &L, blocks, b->threads, smem, b->cap, nullptr));
    }
    SSA_B_TRY(cudaEventRecord(b->t1, b->cap));
    SSA_B_TRY(cudaEventSynchronize(b->t1));
    SSA_B_TRY(cudaEventElapsedTime(&ms, b->t0, b->t1));
  }
  *ms_out = ms;
  return SSA_OK;
}

// Orders the networks -- warp-schedule ones first, by register bucket and M
// descending (the costliest steps first, so that in one kernel for all
// networks the largest networks' trajectories do not start last), then
// thread-schedule ones, most trajectories first -- writes the by-position
// descriptor tables into the slab and prepares the thread-schedule launches
// (network i uses the counter kGroupCounters + its position and its stats
// slot).  Synchronous.
ssa_status upload_tables(ssa_batch* b) {
  const int n = b->n;
  b->order.resize(n);
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
    const bool tx = b->sched[x] == SSA_SCHED_THREAD, ty = b->sched[y] == SSA_SCHED_THREAD;
    if (tx != ty) return !tx;
    if (tx) return b->N[x] > b->N[y];
    const int bx = bucket_of(b->M[x]), by = bucket_of(b->M[y]);
    if (bx != by) return bx > by;
    return b->M[x] > b->M[y];
  });
  b->pos.resize(n);
  b->n_warp = 0;
  for (int p = 0; p < n; ++p) {
    b->pos[b->order[p]] = p;
    if (b->sched[b->order[p]] != SSA_SCHED_THREAD) ++b->n_warp;
  }
  std::vector<BatchNetDev> nets(n);
  std::vector<FinalizeNet> fin(n);
  std::vector<int> cta(n + 1, 0);
  std::vector<long long> work(n + 1, 0), work_s(n + 1, 0);
  const int div = 8;
  unsigned char* s = b->slab;
  b->tnets.clear();
  for (int p = 0; p < n; ++p) {
    const int i = b->order[p];
    nets[p].net = b->wnets[i];
    nets[p].N = b->N[i];
    fin[p] = b->fnets[i];
    work[p + 1] = work[p] + b->N[i];
    work_s[p + 1] = work_s[p] + (b->N[i] + div - 1) / div;
    cta[p + 1] = cta[p] + b->S[i];
    if (b->sched[i] != SSA_SCHED_THREAD) continue;
    ssa_batch::ThreadNet tn;
    const ssa_status st = thread_net(b, i, p, &tn);
    if (st != SSA_OK) return st;
    b->tnets.push_back(tn);
  }
  SSA_B_TRY(cudaMemcpy(s + b->off_nets, nets.data(), sizeof(BatchNetDev) * n, cudaMemcpyHostToDevice));
  SSA_B_TRY(cudaMemcpy(s + b->off_fin, fin.data(), sizeof(FinalizeNet) * n, cudaMemcpyHostToDevice));
  SSA_B_TRY(cudaMemcpy(s + b->off_cta, cta.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice));
  SSA_B_TRY(cudaMemcpy(s + b->off_work, work.data(), 8 * (size_t)(n + 1), cudaMemcpyHostToDevice));
  SSA_B_TRY(cudaMemcpy(s + b->off_work_sample, work_s.data(), 8 * (size_t)(n + 1), cudaMemcpyHostToDevice));
  SSA_B_TRY(cudaDeviceSynchronize());
  return SSA_OK;
}

}  // namespace

extern "C" {

ssa_status ssa_batch_create(int32_t n_models, const ssa_model* const* models, const int64_t* n_traj,
                            const double* t_end, const int32_t* n_grid, const double* const* grids,
                            const ssa_run_opts* opts, ssa_batch** out) {
  if (!out) return (ssa_status)set_error(SSA_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_models < 1 || !models || !n_traj || !t_end || !n_grid)
    return (ssa_status)set_error(SSA_EINVAL, "n_models must be >= 1 and the per-network arrays non-NULL");
  ssa_run_opts o;
  if (opts) o = *opts; else ssa_run_opts_init(&o);
  if (o.precision != SSA_PREC_FP64 && o.precision != SSA_PREC_FP32)
    return (ssa_status)set_error(SSA_EINVAL, "bad precision");
  if (o.memory != SSA_MEM_HOST && o.memory != SSA_MEM_DEVICE) return (ssa_status)set_error(SSA_EINVAL, "bad memory kind");
  if (o.schedule < SSA_SCHED_AUTO || o.schedule > SSA_SCHED_WARP) return (ssa_status)set_error(SSA_EINVAL, "bad schedule");
  if (o.block_threads != 0 && o.block_threads != 64 && o.block_threads != 128 && o.block_threads != 256)
    return (ssa_status)set_error(SSA_EINVAL, "batch block_threads must be 0, 64, 128 or 256");
  if (o.max_events <= 0) o.max_events = SSA_DEFAULT_MAX_EVENTS;
  if (o.max_events > (int64_t)0xFFFFFFFFLL) return (ssa_status)set_error(SSA_EINVAL, "max_events must be below 2^32");
  if (o.stream_id + (uint64_t)n_models > 0x100000000ULL)
    return (ssa_status)set_error(SSA_EINVAL, "stream_id + n_models must not exceed 2^32");
  ssa_batch* b = new (std::nothrow) ssa_batch;
  if (!b) return (ssa_status)set_error(SSA_ENOMEM, "host allocation failed");
  b->n = n_models;
  b->opts = o;
  b->fp32 = o.precision == SSA_PREC_FP32;
  auto bail = [&](int st) {
    ssa_batch_destroy(b);
    return (ssa_status)st;
  };
  for (int i = 0; i < n_models; ++i) {
    const ssa_model* m = models[i];
    if (!m) return bail(set_error(SSA_EINVAL, "a model is NULL"));
    int32_t S = 0, M = 0;
    ssa_model_info(m, &S, &M);
    if (warp_max_chunk(M) == 0) return bail(set_error(SSA_EUNSUPPORTED, "the warp schedule takes at most 512 reactions"));
    if (n_traj[i] < 1) return bail(set_error(SSA_EINVAL, "n_traj must be >= 1"));
    if (!(t_end[i] > 0.0) || !(t_end[i] < 1e300)) return bail(set_error(SSA_EINVAL, "t_end must be finite and > 0"));
    if (n_grid[i] < 1 || (size_t)n_grid[i] * (size_t)S > ((size_t)1 << 31))
      return bail(set_error(SSA_EINVAL, "n_grid must be >= 1 and n_grid * n_species < 2^31"));
    const double* gr = grids ? grids[i] : nullptr;
    if (gr) {
      if (!(gr[0] >= 0.0)) return bail(set_error(SSA_EINVAL, "grid[0] must be >= 0"));
      for (int k = 1; k < n_grid[i]; ++k)
        if (!(gr[k] >= gr[k - 1])) return bail(set_error(SSA_EINVAL, "grids must be ascending"));
      if (!(gr[n_grid[i] - 1] <= t_end[i])) return bail(set_error(SSA_EINVAL, "grid values must be <= t_end"));
    }
    ModelImageView mv;
    if (b->fp32 && model_image_view(m, &mv) && mv.has_mod)
      return bail(set_error(SSA_EUNSUPPORTED, "models with rate modifiers run FP64"));
    if (b->fp32) {
      const double* c = model_rates(m);
      for (int j = 0; j < M; ++j)
        if (c[j] > 3.4028234663852886e38)
          return bail(set_error(SSA_EINVAL, "a rate exceeds the binary32 range of the FP32-propensity mode"));
    }
    b->models.push_back(m);
    b->N.push_back(n_traj[i]);
    b->G.push_back(n_grid[i]);
    b->S.push_back(S);
    b->M.push_back(M);
    b->t_end.push_back(t_end[i]);
  }
  // schedules: networks that fit the thread kernel start on it under AUTO
  // (the rule of ssa_ensemble_run), until ssa_batch_tune times both
  const int n = n_models;
  b->sched.assign(n, SSA_SCHED_WARP);
  b->thread_ok.assign(n, 0);
  b->smalls.resize(n);
  b->sched_fixed = o.schedule != SSA_SCHED_AUTO;
  for (int i = 0; i < n; ++i) {
    model_small_copy(b->models[i], &b->smalls[i]);
    b->thread_ok[i] = (!b->fp32 && b->smalls[i].has_small) ? 1 : 0;
    if (o.schedule == SSA_SCHED_THREAD && !b->thread_ok[i])
      return bail(set_error(SSA_EUNSUPPORTED, "the thread schedule takes FP64 networks of at most 16 reactions and "
                                              "16 species without rate modifiers"));
    if (o.schedule != SSA_SCHED_WARP && b->thread_ok[i]) b->sched[i] = SSA_SCHED_THREAD;
  }
  cudaError_t e = cudaGetDevice(&b->dev);
  if (e != cudaSuccess) return bail(set_error(SSA_ECUDA, cudaGetErrorString(e)));
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, b->dev);
  if (e != cudaSuccess) return bail(set_error(SSA_ECUDA, cudaGetErrorString(e)));
  b->sms = prop.multiProcessorCount;
  b->smem_optin = (int)prop.sharedMemPerBlockOptin;

  // slab layout (pieces by network index)
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off = align_up(off + bytes, 256);
    return at;
  };
  b->off_nets = take(sizeof(BatchNetDev) * n);
  b->off_fin = take(sizeof(FinalizeNet) * n);
  b->off_cta = take(sizeof(int) * (n + 1));
  b->off_work = take(sizeof(long long) * (n + 1));
  b->off_work_sample = take(sizeof(long long) * (n + 1));
  b->off_seed = take(8);
  b->off_grid.resize(n);
  b->off_depw.resize(n);
  b->off_c32.resize(n);
  b->off_mean.resize(n);
  b->off_var.resize(n);
  b->off_s1.resize(n);
  b->off_s2.resize(n);
  b->off_d1.resize(n);
  b->off_d2.resize(n);
  for (int i = 0; i < n; ++i) {
    const size_t gs = (size_t)b->G[i] * b->S[i];
    b->off_grid[i] = take(8 * (size_t)b->G[i]);
    b->off_depw[i] = take(2 * (size_t)b->M[i] * 32);
    b->off_c32[i] = take(4 * (size_t)b->M[i]);
    b->off_mean[i] = take(8 * gs);
    b->off_var[i] = take(8 * gs);
    b->off_s1[i] = take(8 * gs);
    b->off_s2[i] = take(8 * gs);
  }
  // everything from here on is zeroed before every pass
  b->zero_begin = off;
  b->off_counters = take(8 * (size_t)(ssa_batch::kGroupCounters + n));
  b->off_stats = take(8 * 4 * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const size_t gs = (size_t)b->G[i] * b->S[i];
    b->off_d1[i] = take(8 * gs);
    b->off_d2[i] = take(8 * gs);
  }
  b->zero_bytes = off - b->zero_begin;
  e = cudaMalloc(reinterpret_cast<void**>(&b->slab), off);
  if (e != cudaSuccess) return bail(set_error(SSA_ENOMEM, cudaGetErrorString(e)));

  // per network: device tables, derived tables, grid, descriptors
  b->wnets.resize(n);
  b->fnets.resize(n);
  b->dms.resize(n);
  for (int i = 0; i < n; ++i) {
    DevModel& dm = b->dms[i];
    int st = model_device_tables(b->models[i], b->dev, &dm);
    if (st != SSA_OK) return bail(st);
    unsigned char* s = b->slab;
    k_batch_tables<<<(b->M[i] * 32 + 255) / 256, 256>>>(dm, reinterpret_cast<uint16_t*>(s + b->off_depw[i]),
                                                          reinterpret_cast<float*>(s + b->off_c32[i]));
    e = cudaGetLastError();
    if (e != cudaSuccess) return bail(set_error(SSA_ECUDA, cudaGetErrorString(e)));
    double* dgrid = reinterpret_cast<double*>(s + b->off_grid[i]);
    const double* gr = grids ? grids[i] : nullptr;
    if (gr) {
      e = cudaMemcpy(dgrid, gr, 8 * (size_t)b->G[i], cudaMemcpyHostToDevice);
    } else {
      e = launch_uniform_grid(dgrid, b->G[i], b->t_end[i], nullptr);
    }
    if (e != cudaSuccess) return bail(set_error(SSA_ECUDA, cudaGetErrorString(e)));
    WarpNet& w = b->wnets[i];
    w.rinfo = dm.rinfo;
    w.cbits = reinterpret_cast<const unsigned long long*>(dm.c);
    w.c32 = reinterpret_cast<const float*>(s + b->off_c32[i]);
    w.nu_ptr = dm.nu_ptr;
    w.nu_idx = dm.nu_idx;
    w.nu_val = dm.nu_val;
    w.depw = reinterpret_cast<const uint16_t*>(s + b->off_depw[i]);
    w.x0 = dm.x0;
    w.grid = dgrid;
    w.D1 = reinterpret_cast<unsigned long long*>(s + b->off_d1[i]);
    w.D2 = reinterpret_cast<unsigned long long*>(s + b->off_d2[i]);
    w.mod_f = dm.mod_f;
    w.mod_k = dm.mod_k;
    w.mod_lo = dm.mod_lo;
    w.mod_hi = dm.mod_hi;
    double te = b->t_end[i];
    std::memcpy(&w.t_end_bits, &te, 8);
    w.S = b->S[i];
    w.M = b->M[i];
    w.G = b->G[i];
    w.nnz_max = model_nnz_max(b->models[i]);
    const bool uniform = !gr || host_grid_is_uniform(gr, b->G[i], te);
    w.grid_uniform = (uniform && b->G[i] >= 2 && b->G[i] <= (1 << 20) && te < 1e30) ? 1 : 0;
    w.grid_scale = (float)((double)(b->G[i] - 1) / te);
    w.grid_margin = (float)((double)b->G[i] * 0x1p-21);
    w.sid = (uint32_t)(o.stream_id + (uint64_t)i);
    FinalizeNet& f = b->fnets[i];
    f.D1 = w.D1;
    f.D2 = w.D2;
    f.x0 = dm.x0;
    f.mean = reinterpret_cast<double*>(s + b->off_mean[i]);
    f.var = reinterpret_cast<double*>(s + b->off_var[i]);
    f.sum1 = reinterpret_cast<int64_t*>(s + b->off_s1[i]);
    f.sum2 = reinterpret_cast<int64_t*>(s + b->off_s2[i]);
    f.G = b->G[i];
    f.S = b->S[i];
    f.N = b->N[i];
    b->max_G = std::max(b->max_G, b->G[i]);
  }
  for (int i = 0; i < n; ++i) b->total_ctas += b->S[i];
  ssa_status ust = upload_tables(b);
  if (ust != SSA_OK) return bail(ust);

  b->threads = o.block_threads ? o.block_threads : 128;
  b->split = true;
  const ssa_status pst = plan_groups(b);
  if (pst != SSA_OK) return bail(pst);
  if ((e = cudaEventCreate(&b->t0)) != cudaSuccess || (e = cudaEventCreate(&b->t1)) != cudaSuccess)
    return bail(set_error(SSA_ECUDA, cudaGetErrorString(e)));
  b->host_stats.assign(4 * (size_t)n, 0);
  *out = b;
  return SSA_OK;
}

ssa_status ssa_batch_tune(ssa_batch* b, int32_t* block_threads, int32_t* split, double* sample_ms) {
  if (!b) return (ssa_status)set_error(SSA_EINVAL, "batch is NULL");
  const int cand_threads[3] = {64, 128, 256};
  double best = 1e300;
  int best_t = b->threads;
  bool best_split = b->split;
  ssa_status st = SSA_OK;
  // thread versus warp for every network that fits both (unless opts fixed
  // the schedule): each timed alone on its sample, the faster kept and
  // recorded; the batch's results then follow the recorded schedules
  if (!b->sched_fixed) {
    bool any = false;
    for (int i = 0; i < b->n; ++i) any = any || b->thread_ok[i];
    if (any) {
      if ((st = ensure_streams(b)) != SSA_OK) return st;
      if ((st = set_seed(b, 0x5eedULL ^ 0xA5A5A5A5ULL, b->cap)) != SSA_OK) return st;
      for (int i = 0; i < b->n; ++i) {
        if (!b->thread_ok[i]) continue;
        double t_thread = 0.0, t_warp = 0.0;
        if ((st = time_schedule(b, i, true, &t_thread)) != SSA_OK) return st;
        if ((st = time_schedule(b, i, false, &t_warp)) != SSA_OK) return st;
        b->sched[i] = (t_thread <= t_warp) ? SSA_SCHED_THREAD : SSA_SCHED_WARP;
      }
      if ((st = upload_tables(b)) != SSA_OK) return st;
      drop_graph(b);
    }
  }
  for (int sp = 0; sp < 2; ++sp) {
    for (int ti = 0; ti < 3; ++ti) {
      b->threads = cand_threads[ti];
      b->split = sp == 0;
      if ((st = plan_groups(b)) != SSA_OK) return st;
      if ((st = ensure_streams(b)) != SSA_OK) return st;
      if ((st = set_seed(b, 0x5eedULL ^ 0xA5A5A5A5ULL, b->cap)) != SSA_OK) return st;
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // the first pass warms up
        SSA_B_TRY(cudaEventRecord(b->t0, b->cap));
        if ((st = enqueue_pass(b, b->cap, true)) != SSA_OK) return st;
        SSA_B_TRY(cudaEventRecord(b->t1, b->cap));
        SSA_B_TRY(cudaEventSynchronize(b->t1));
        SSA_B_TRY(cudaEventElapsedTime(&ms, b->t0, b->t1));
      }
      if (ms < best) {
        best = ms;
        best_t = b->threads;
        best_split = b->split;
      }
    }
  }
  b->threads = best_t;
  b->split = best_split;
  b->tuned_ms = best;
  if ((st = plan_groups(b)) != SSA_OK) return st;
  drop_graph(b);
  if (block_threads) *block_threads = best_t;
  if (split) *split = best_split ? 1 : 0;
  if (sample_ms) *sample_ms = best;
  return SSA_OK;
}

ssa_status ssa_batch_launch(ssa_batch* b, uint64_t seed, double* const* means, double* const* vars,
                            int64_t* const* sums1, int64_t* const* sums2, ssa_run_stats* stats) {
  if (!b) return (ssa_status)set_error(SSA_EINVAL, "batch is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(b->opts.cuda_stream);
  ssa_status rc;
  if (!b->exec && (rc = capture(b)) != SSA_OK) return rc;
  if ((rc = set_seed(b, seed, st)) != SSA_OK) return rc;
  if (stats) SSA_B_TRY(cudaEventRecord(b->t0, st));
  SSA_B_TRY(cudaGraphLaunch(b->exec, st));
  if (stats) SSA_B_TRY(cudaEventRecord(b->t1, st));
  const bool host = b->opts.memory == SSA_MEM_HOST;
  const cudaMemcpyKind kind = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  unsigned char* s = b->slab;
  for (int i = 0; i < b->n; ++i) {
    const size_t bytes = 8 * (size_t)b->G[i] * b->S[i];
    if (means && means[i]) SSA_B_TRY(cudaMemcpyAsync(means[i], s + b->off_mean[i], bytes, kind, st));
    if (vars && vars[i]) SSA_B_TRY(cudaMemcpyAsync(vars[i], s + b->off_var[i], bytes, kind, st));
    if (sums1 && sums1[i]) SSA_B_TRY(cudaMemcpyAsync(sums1[i], s + b->off_s1[i], bytes, kind, st));
    if (sums2 && sums2[i]) SSA_B_TRY(cudaMemcpyAsync(sums2[i], s + b->off_s2[i], bytes, kind, st));
  }
  const bool wait = stats || (host && (means || vars || sums1 || sums2));
  if (!wait) return SSA_OK;
  SSA_B_TRY(cudaMemcpyAsync(b->host_stats.data(), s + b->off_stats, 8 * 4 * (size_t)b->n, cudaMemcpyDeviceToHost, st));
  SSA_B_TRY(cudaStreamSynchronize(st));
  unsigned long long ev = 0, tr = 0, ov = 0, mx = 0;
  int bad = -1;
  for (int p = 0; p < b->n; ++p) {
    const unsigned long long* h = &b->host_stats[4 * (size_t)p];
    ev += h[0];
    tr += h[1];
    ov += h[2];
    mx = std::max(mx, h[3]);
    const int i = b->order[p];
    const long double bound = (long double)b->N[i] * (long double)h[3] * (long double)h[3];
    if (h[2] > 0 || bound >= 9.2233720368547758e18L) bad = i;
  }
  if (stats) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->t0, b->t1);
    stats->events = (int64_t)ev;
    stats->truncated = (int64_t)tr;
    stats->overflowed = (int64_t)ov;
    stats->max_x = (int64_t)mx;
    stats->kernel_ms = ms;
    int common = b->sched[0];
    for (int i = 1; i < b->n; ++i) common = (b->sched[i] == common) ? common : SSA_SCHED_AUTO;
    stats->schedule = common;
    stats->handoffs = 0;
  }
  if (bad >= 0) {
    char msg[128];
    snprintf(msg, sizeof msg, "network %d: a count reached the int32 limit or N * max_x^2 may exceed int64", bad);
    return (ssa_status)set_error(SSA_EOVERFLOW, msg);
  }
  return SSA_OK;
}

ssa_status ssa_batch_result(const ssa_batch* b, int32_t index, const double** mean, const double** var,
                            const int64_t** sum1, const int64_t** sum2) {
  if (!b || index < 0 || index >= b->n) return (ssa_status)set_error(SSA_EINVAL, "bad batch or index");
  const unsigned char* s = b->slab;
  if (mean) *mean = reinterpret_cast<const double*>(s + b->off_mean[index]);
  if (var) *var = reinterpret_cast<const double*>(s + b->off_var[index]);
  if (sum1) *sum1 = reinterpret_cast<const int64_t*>(s + b->off_s1[index]);
  if (sum2) *sum2 = reinterpret_cast<const int64_t*>(s + b->off_s2[index]);
  return SSA_OK;
}

ssa_status ssa_batch_network_stats(const ssa_batch* b, int32_t index, ssa_run_stats* out) {
  if (!b || !out || index < 0 || index >= b->n) return (ssa_status)set_error(SSA_EINVAL, "bad batch, index or out");
  const unsigned long long* h = &b->host_stats[4 * (size_t)b->pos[index]];
  out->events = (int64_t)h[0];
  out->truncated = (int64_t)h[1];
  out->overflowed = (int64_t)h[2];
  out->max_x = (int64_t)h[3];
  out->kernel_ms = 0.0;
  out->schedule = b->sched[index];
  out->handoffs = 0;
  return SSA_OK;
}

void ssa_batch_destroy(ssa_batch* b) {
  if (!b) return;
  drop_graph(b);
  for (cudaStream_t f : b->forks) cudaStreamDestroy(f);
  for (cudaEvent_t e : b->evs) cudaEventDestroy(e);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->t0) cudaEventDestroy(b->t0);
  if (b->t1) cudaEventDestroy(b->t1);
  if (b->slab) cudaFree(b->slab);
  delete b;
}

ssa_status ssa_batch_run(int32_t n_models, const ssa_model* const* models, const int64_t* n_traj,
                         const double* t_end, const int32_t* n_grid, const double* const* grids, uint64_t seed,
                         const ssa_run_opts* opts, double* const* means, double* const* vars) {
  ssa_batch* b = nullptr;
  ssa_status st = ssa_batch_create(n_models, models, n_traj, t_end, n_grid, grids, opts, &b);
  if (st != SSA_OK) return st;
  st = ssa_batch_launch(b, seed, means, vars, nullptr, nullptr, nullptr);
  if (st == SSA_OK) {
    const cudaError_t e = cudaStreamSynchronize(static_cast<cudaStream_t>(b->opts.cuda_stream));
    if (e != cudaSuccess) st = (ssa_status)set_error(SSA_ECUDA, cudaGetErrorString(e));
  }
  ssa_batch_destroy(b);
  return st;
}

}  // extern "C"
