/*
 * ssa.h — C ABI of libssa: ensembles of Gillespie direct-method trajectories of
 * a mass-action reaction network on one sm_103a GPU, with every trajectory's
 * state aligned on a common simulation-time grid and reduced across
 * trajectories into exact int64 sums, mean and variance.
 *
 * Paper: Aldinucci, Bracciali, Lio, Sorathiya, Torquati, "StochKit-FF:
 * Efficient Systems Biology on Multicore Architectures" (arXiv:1007.1768).
 *   - Sec. 2: the direct method picks the next transition and its time from
 *     the CTMC's law and updates the state; one such run is a trajectory.
 *   - Sec. 3.2 (model files): a model is an integer state vector, an integer
 *     stoichiometric matrix, a propensity vector following mass action, the
 *     rate constants and the simulated duration.
 *   - Sec. 3.2 (StochRxn_ff): many copies of one simulation, or a parameter
 *     sweep, run in parallel.
 *   - Sec. 3.2.1 and Fig. 3 ("selective memory"): points of different
 *     trajectories are aligned by simulation time and reduced by associative,
 *     commutative functions; Sec. 4 uses average and variance.
 *
 * Conventions for every call:
 *   - No call throws; each returns an ssa_status.  On failure a message for
 *     the calling thread is available from ssa_last_error().
 *   - Arrays are dense, row-major, C order.  "G x S" means index k * S + s.
 *   - The library copies every input it keeps (models); the caller owns every
 *     output buffer.
 *   - opts->memory selects where grid and output arrays live: SSA_MEM_HOST
 *     (plain host memory; the call copies in and out and is synchronous) or
 *     SSA_MEM_DEVICE (device memory of the current CUDA device; the call only
 *     enqueues work on opts->cuda_stream and returns, unless `stats` is
 *     non-NULL, in which case it waits for the stream).
 *   - The current CUDA device at the time of the call is used.
 */
#ifndef SSA_H_
#define SSA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum ssa_status {
  SSA_OK = 0,
  SSA_EINVAL = 1,       /* an argument is out of its documented range */
  SSA_ENOMEM = 2,       /* a device or host allocation failed */
  SSA_ECUDA = 3,        /* a CUDA runtime call failed */
  SSA_EOVERFLOW = 4,    /* a count would leave int32, or sum x^2 could leave int64 */
  SSA_ETRUNCATED = 5,   /* reserved: some trajectory hit max_events (reported in stats) */
  SSA_ETIMEOUT = 6,     /* a bounded device wait ran out (hand-off between warps) */
  SSA_EUNSUPPORTED = 7  /* valid request this build does not implement */
} ssa_status;

/* Precision of the propensity arithmetic.  Time is FP64 in every mode.
 *   SSA_PREC_FP64: a_j = c_j * (double)h_j; a0 and the selection prefix sums
 *     are FP64 sums in the schedule's order.
 *   SSA_PREC_FP32: a_j = (float)c_j * (float)h_j in binary32; the selection
 *     prefix sums are binary32 sums (schedule W32) with total A32; a0 is
 *     formed anew at every event in FP64: each lane's chunk is summed in
 *     binary32 with its rounding errors carried (cascaded TwoSum), the two
 *     parts widened and added in FP64, and the 32 lane values combined by
 *     the W32 scan in FP64; tau = -ln(r1) / a0 and t in FP64; the reaction
 *     is the first j with a_j > 0 and (double)prefix_j > r2 * (double)A32.
 *     Runs one trajectory per warp; rates must lie in the binary32 range. */
enum { SSA_PREC_FP64 = 0, SSA_PREC_FP32 = 1 };
/* Kernel shape and summation order:
 *   SSA_SCHED_THREAD: one trajectory per thread, sums left to right
 *     (schedule L); networks of at most 16 reactions and 16 species.
 *   SSA_SCHED_WARP: one trajectory per warp, schedule W32: lane l owns the
 *     reactions l*c .. l*c + c - 1 (c = ceil(M / 32)) and sums them left to
 *     right; the 32 lane sums are combined by an inclusive Kogge-Stone scan
 *     (offsets 1, 2, 4, 8, 16); prefix_j = (scan of the lanes before j's
 *     lane) + (running sum inside j's chunk); a0 = the scan's last value.
 *     Networks of at most 512 reactions.
 *   SSA_SCHED_AUTO: THREAD for FP64 networks that fit it, else WARP. */
enum { SSA_SCHED_AUTO = 0, SSA_SCHED_THREAD = 1, SSA_SCHED_WARP = 2 };
/* Where grid / outputs live. */
enum { SSA_MEM_HOST = 0, SSA_MEM_DEVICE = 1 };
/* Where the per-CTA difference arrays of the reduction live. */
enum { SSA_REDUCE_AUTO = 0, SSA_REDUCE_SHARED = 1, SSA_REDUCE_GLOBAL = 2 };

/* Largest state count; an event that would exceed it is not fired and the
 * trajectory stops with the overflow flag. */
#define SSA_STATE_MAX 2147483647
#define SSA_DEFAULT_MAX_EVENTS ((int64_t)100000000)

/* Per-trajectory flag bits (opts->traj_flags). */
#define SSA_TRAJ_TRUNCATED 1
#define SSA_TRAJ_OVERFLOW 2

typedef struct ssa_model ssa_model; /* opaque, owned by the library */

/* Options of one ensemble run.  Initialise with ssa_run_opts_init(). */
typedef struct ssa_run_opts {
  int32_t precision;      /* SSA_PREC_FP64 (bit-exact with the oracle) or SSA_PREC_FP32 */
  int32_t schedule;       /* SSA_SCHED_* */
  int32_t memory;         /* SSA_MEM_HOST or SSA_MEM_DEVICE */
  int32_t reduce;         /* SSA_REDUCE_* */
  int32_t block_threads;  /* threads per CTA; 0 = choose */
  int32_t grid_blocks;    /* CTAs; 0 = choose */
  int64_t max_events;     /* events per trajectory before it is truncated, < 2^32; <= 0: SSA_DEFAULT_MAX_EVENTS */
  uint64_t traj_offset;   /* id of the first trajectory; ids are traj_offset .. traj_offset + n_traj - 1 */
  uint64_t stream_id;     /* fourth word of the random counter, < 2^32 (e.g. a network index) */
  void* cuda_stream;      /* cudaStream_t to run on; NULL = the legacy default stream */
  void* workspace;        /* device scratch of workspace_bytes; NULL = taken from the library's stream-ordered
                           * pool and returned to it (ssa_release_cached_memory) */
  size_t workspace_bytes;
  /* Optional per-trajectory outputs, [n_traj] each, in opts->memory's space; NULL to skip:
   * events fired, a 64-bit hash of the (reaction index, event time bits) sequence, flag bits.
   * (ssa_ensemble_grad reads traj_events as an input: the forward's counts.) */
  int64_t* traj_events;
  uint64_t* traj_hash;
  int32_t* traj_flags;
  /* Optional device int64[4] (device memory even with SSA_MEM_HOST): the run
   * adds its event, truncated and overflowed counts to [0], [1], [2] and
   * raises [3] to its largest count, without waiting for the stream. */
  int64_t* device_totals;
  /* Optional cudaEvent_t handles recorded on the stream immediately before and
   * after the simulation kernel (for timing it alone); NULL to skip. */
  void* sim_event_begin;
  void* sim_event_end;
  /* ssa_ensemble_avg_xy only: capacity of the event log in records; 0 = the
   * records per trajectory of an earlier call on the same model (same t_end,
   * precision, max_events) scaled with a margin, else the event count of a
   * pilot of up to 4,096 trajectories scaled with a quarter to spare.  Too
   * small a value costs one more logging run. */
  int64_t log_records;
} ssa_run_opts;

/* Totals of one run (host struct). */
typedef struct ssa_run_stats {
  int64_t events;       /* reaction events fired over all trajectories */
  int64_t truncated;    /* trajectories stopped by max_events */
  int64_t overflowed;   /* trajectories stopped by SSA_STATE_MAX */
  int64_t max_x;        /* largest count seen in any trajectory */
  double kernel_ms;     /* device time of the simulation + reduction kernels */
  int32_t schedule;     /* SSA_SCHED_THREAD or SSA_SCHED_WARP: the schedule that ran (for a
                           whole batch SSA_SCHED_AUTO; per network see ssa_batch_network_stats) */
  int64_t handoffs;     /* trajectories one warp passed to another during the run (thread
                           schedule of ssa_ensemble_run; 0 elsewhere); results do not depend on it */
} ssa_run_stats;

/* Text for a status code (static storage). */
const char* ssa_status_string(ssa_status status);

/* Message of the last failed call on this thread ("" if none). */
const char* ssa_last_error(void);

/* Returns the device memory that the library keeps between calls (its
 * stream-ordered pools hold the workspaces of finished calls for reuse) to
 * the driver.  Call when no library work is in flight.  Errors: SSA_ECUDA. */
ssa_status ssa_release_cached_memory(void);

/*
 * ssa_finalize_sums — the average and variance of Sec. 4 from int64 grid sums
 * (step A8) on the host, for sums added across shards: trajectories are
 * fixed by (seed, id, stream id), so runs over contiguous id ranges
 * (opts->traj_offset) add up to the sums of one run bit for bit.
 *   sum1, sum2: [n_grid x n_species] row-major host arrays of sum x and
 *     sum x^2 over n_traj trajectories (sum1, sum2 of ssa_ensemble_run);
 *   mean, var: [n_grid x n_species] host outputs (caller-owned).
 * mean = sum1 / N; var = (N sum2 - sum1^2) / (N (N - 1)) with the numerator
 * exact in 128 bits and rounded once; NaN when N = 1.  The values are
 * bit-identical to what the device finalisation writes for a single run.
 * Errors: SSA_EINVAL (n_traj < 1, n_grid < 1, n_species < 1, NULL arrays).
 */
ssa_status ssa_finalize_sums(int64_t n_traj, int32_t n_grid, int32_t n_species, const int64_t* sum1,
                             const int64_t* sum2, double* mean, double* var);

/* Fills *opts with the defaults: FP64, AUTO schedule and reduction, host
 * memory, default max_events, offset 0, stream id 0, default CUDA stream,
 * library-managed workspace, no per-trajectory outputs. */
void ssa_run_opts_init(ssa_run_opts* opts);

/*
 * Creates a model (Sec. 3.2 model files).
 *   n_species S >= 1, n_reactions M >= 1.
 *   reactants [M x S]: multiplicity of species s consumed by reaction j,
 *     entries 0..2 with row sum <= 2 (mass-action orders 0, 1, 2).
 *   products  [M x S]: molecules of s produced by j, entries 0..SSA_STATE_MAX.
 *   rates     [M]: stochastic rate constants c_j, finite and >= 0.
 *   x0        [S]: initial counts, 0..SSA_STATE_MAX.
 * The propensity of j in state x is c_j * prod_s C(x_s, reactants[j][s]);
 * the state change of j is products[j] - reactants[j].
 * All arrays are host memory and are copied.  *out receives the model.
 * Errors: SSA_EINVAL (bad sizes or entries), SSA_ENOMEM.
 */
ssa_status ssa_model_create(int32_t n_species, int32_t n_reactions, const int32_t* reactants,
                            const int32_t* products, const double* rates, const int32_t* x0,
                            ssa_model** out);

/*
 * Makes the rate of `reaction` state dependent (the paper's TNF-dependent
 * infectivities, Sec. 2.1: beta_R5 = beta - K F clamped to [0, beta],
 * beta_X4 = beta + K F):
 *   rate = min(max(c + slope * x_species, lo), hi)      (FP64: product, sum, clamp)
 * where c is the reaction's rate constant; the propensity is rate * h(x).
 * species = -1 removes the modifier.  0 <= lo <= hi, lo finite (hi may be
 * +infinity); slope finite.  Models with modifiers run FP64 on the warp
 * schedule (ssa_ensemble_run, ssa_ensemble_avg_xy, FP64 batches); the
 * thread schedule, FP32 mode, ssa_ensemble_grad and ssa_ensemble_run_noalloc
 * refuse them (SSA_EUNSUPPORTED).  Not thread-safe against runs of the same
 * model in flight.
 * Errors: SSA_EINVAL.
 */
ssa_status ssa_model_set_rate_modifier(ssa_model* model, int32_t reaction, int32_t species, double slope, double lo,
                                       double hi);

/* Releases a model and its device copies.  NULL is ignored.  No run using the
 * model may be pending on any stream. */
void ssa_model_destroy(ssa_model* model);

/* Sizes of a model. */
ssa_status ssa_model_info(const ssa_model* model, int32_t* n_species, int32_t* n_reactions);

/* Device scratch bytes ssa_ensemble_run needs for these arguments (the
 * per-grid difference sums, the work counter and the totals). */
ssa_status ssa_ensemble_workspace_size(const ssa_model* model, int64_t n_traj, int32_t n_grid,
                                       const ssa_run_opts* opts, size_t* bytes);

/*
 * Runs n_traj independent trajectories (Sec. 2) of `model` from its x0 over
 * [0, t_end] and reduces them on the grid (Sec. 3.2.1):
 *   sum1[k][s] = sum_i X_i,s(g_k),  sum2[k][s] = sum_i X_i,s(g_k)^2   (int64)
 *   mean = sum1 / N,  var = (N sum2 - sum1^2) / (N (N - 1))           (FP64)
 * where X_i(g) is trajectory i's state after every event with time <= g.
 * At each event the reaction fired is the first j with a_j > 0 and
 * prefix_j > r2 * a0 (the last j with a_j > 0 if rounding leaves none), and
 * the time step is -ln(r1) / a0 (Sec. 2, direct method).
 * Event n of trajectory id = traj_offset + i draws one Philox4x32-10 block
 * with key (seed low word, seed high word) and counter (n, id low word, id
 * high word, opts->stream_id), so any trajectory can be reproduced alone and
 * shards by traj_offset add up exactly.
 *   n_traj >= 1 (var is NaN when n_traj == 1); t_end > 0 and finite;
 *   n_grid >= 1; grid [n_grid] ascending, grid[0] >= 0, grid[n_grid-1] <= t_end,
 *     or NULL for g_k = (k * t_end) / (n_grid - 1) (g_0 = t_end if n_grid == 1).
 *   mean, var [G x S] doubles; sum1, sum2 [G x S] int64 or NULL.
 *   stats: host struct or NULL.
 * The results are bit-identical to the plain CPU statement of the same
 * arithmetic (the oracle shipped with the tests) for the precision and
 * summation schedule the run uses.  On the thread schedule warps pass
 * trajectories to idle warps between batches of the cooperative tail (a pool
 * of trajectory states in the workspace; stats->handoffs counts them); which
 * warp runs which events does not change any result.
 * Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA, SSA_EUNSUPPORTED,
 * SSA_EOVERFLOW, SSA_ETIMEOUT (a bounded wait of the hand-off ran out; both
 * only detectable when the call waits: host memory or stats).
 */
ssa_status ssa_ensemble_run(const ssa_model* model, int64_t n_traj, double t_end, int32_t n_grid,
                            const double* grid, uint64_t seed, const ssa_run_opts* opts,
                            double* mean, double* var, int64_t* sum1, int64_t* sum2,
                            ssa_run_stats* stats);

/*
 * ssa_ensemble_grad -- likelihood-ratio sensitivities of a loss on the grid
 * mean with respect to the rate constants (FP64, thread schedule: networks of
 * at most 16 reactions and 16 species, every rate > 0).
 *
 * The trajectories of ssa_ensemble_run with the same model, n_traj, t_end,
 * grid, seed and opts are replayed from their Philox counters (nothing of the
 * forward pass is stored).  For reaction r the score of a path is
 *   Z_r(t) = N_r(t) / c_r - int_0^t h_r(x(s)) ds
 * (N_r: firings of r up to t), and trajectory i contributes
 *   g_ir = sum_k u_k Z_r(g_k),  u_k = sum_s dL_dmean[k][s] (x_is(g_k) - mean[k][s]).
 *   dL_drates[r]    = (1/N) sum_i g_ir
 *   dL_drates_se[r] = sample standard deviation of g_ir / sqrt(N)   (may be NULL)
 * dL_dmean, mean [G x S] and the outputs [M] live in opts->memory's space.
 * opts->workspace, when non-NULL, receives the per-trajectory contributions
 * g (M x N, column r at r * N, same memory space; workspace_bytes >= 8 M N).
 * opts->traj_events, when non-NULL, is an input here: the forward's
 * per-trajectory event counts [N] (same memory space).  When N is several
 * times the GPU's resident threads, the replay then starts the longest
 * trajectories first; the results do not depend on it (each contribution is
 * kept at its trajectory's index and reduced in index order), only the time
 * the replay's last trajectories take.
 * Host memory: synchronous.  Device memory: enqueued on opts->cuda_stream.
 * Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA, SSA_EUNSUPPORTED (FP32 mode, the
 * warp schedule, larger networks, a zero rate).
 */
ssa_status ssa_ensemble_grad(const ssa_model* model, int64_t n_traj, double t_end, int32_t n_grid,
                             const double* grid, uint64_t seed, const ssa_run_opts* opts, const double* dL_dmean,
                             const double* mean, double* dL_drates, double* dL_drates_se);

/*
 * ssa_ensemble_avg_xy -- selective memory along the time axis (Sec. 3.2.1,
 * Fig. 3): Avg-Y on the union of every trajectory's event times, reduced
 * along time into Avg-XY (adaptive sampling: more points where more events
 * happen).
 *
 * Union points T_0 = 0 < T_1 < ... < T_{U-1} are 0 and the distinct event
 * times of all n_traj trajectories (ids traj_offset + i, opts->precision);
 * the trajectories are ssa_ensemble_run's under the same opts->schedule
 * (AUTO: the thread schedule for FP64 networks of at most 16 reactions and
 * species without rate modifiers, else the warp schedule).
 * S1_m[s] and S2_m[s] are the sums over trajectories of
 * x_s(T_m) and x_s(T_m)^2 (right-continuous states).  Window p covers union
 * points [p k, min(U, (p + 1) k)) with n_p points, k = window (0: n_traj):
 *   t_out[p]         = (T_pk + ... ) / n_p      (FP64, ascending order)
 *   mean_out[p][s]   = (sum over the window of S1_m[s]) / (N n_p)
 *   msq_out[p][s]    = (sum over the window of S2_m[s]) / (N n_p)
 * window = 1 returns Avg-Y itself.  Outputs hold max_points entries (x S for
 * mean and msq) in opts->memory's space; *n_points receives the number of
 * windows P (only min(P, max_points) are written; max_points = 0 only
 * counts) and *n_union (may be NULL) the number of union points U.
 * The event log takes about 57 bytes of device memory per (event, species
 * changed); opts->log_records sizes it (0: an earlier call's count, else a
 * pilot of up to 4,096 trajectories, estimates it).  Should the log run out,
 * the logging run is repeated once with the exact record count it reports.
 * Workspaces come from the library's pool (ssa_release_cached_memory).
 * Synchronous.
 * Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA, SSA_EUNSUPPORTED (the thread
 * schedule for a network or mode it does not take, networks beyond the warp
 * schedule, more than 2^31 log records),
 * SSA_EOVERFLOW (n_traj * max_x^2 * window could leave int64).
 */
ssa_status ssa_ensemble_avg_xy(const ssa_model* model, int64_t n_traj, double t_end, uint64_t seed,
                               const ssa_run_opts* opts, int64_t window, int64_t max_points, double* t_out,
                               double* mean_out, double* msq_out, int64_t* n_points, int64_t* n_union);

/*
 * Size of the fixed device scratch used by ssa_ensemble_run_noalloc: 4 MiB,
 * held by every GPU that loads the library until the process exits.
 */
#define SSA_NOALLOC_SCRATCH_BYTES ((size_t)4 << 20)

/*
 * ssa_ensemble_run_noalloc — the same computation as ssa_ensemble_run, for
 * callers that cannot allocate device memory during the call.  The paper has
 * no counterpart; this exists for deployment.  Such callers include code whose
 * device memory is owned and pre-sized by another runtime, plugins that the
 * host process bars from the allocator, and latency-bound loops that must not
 * block on an allocation.
 *
 * It calls no cudaMalloc, cudaMallocAsync, cudaFree or other allocating
 * routine, and copies nothing from host memory: the model's tables travel as
 * kernel parameters.  Its scratch (work counter, totals, per-grid difference
 * sums, the uniform grid and the initial counts) lives in one fixed device
 * array of SSA_NOALLOC_SCRATCH_BYTES per GPU.  The caller passes all inputs
 * and outputs:
 *   opts->memory must be SSA_MEM_DEVICE; grid (NULL for the uniform grid),
 *   mean, var [G x S] and the optional sum1, sum2 [G x S] and per-trajectory
 *   outputs are device pointers on the current device.  stats is a host
 *   struct or NULL; when non-NULL the call waits for the stream (kernel_ms is
 *   reported as 0); otherwise it only enqueues work.  opts->workspace is
 *   ignored; opts->sim_event_begin / sim_event_end are recorded around the
 *   simulation kernel as in ssa_ensemble_run.
 * Limits: 16 * n_grid * n_species + 8 * n_grid + 64 bytes (plus alignment)
 * must fit in SSA_NOALLOC_SCRATCH_BYTES, else SSA_EINVAL with a message
 * giving the bytes needed.  Networks with at most 16 reactions and 16
 * species, FP64, without rate modifiers (others: SSA_EUNSUPPORTED).
 * Sharing: every call uses the same array and overwrites what the previous
 * call left there; each call clears what must start at zero on its own stream.
 * Calls whose GPU work overlaps (several streams or host threads on one
 * device) race and give wrong results, so serialise them.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current).  Make that first call
 * before any stream capture on the device.
 * Results are bit-identical to ssa_ensemble_run with the same arguments.
 */
ssa_status ssa_ensemble_run_noalloc(const ssa_model* model, int64_t n_traj, double t_end, int32_t n_grid,
                                    const double* grid, uint64_t seed, const ssa_run_opts* opts,
                                    double* mean, double* var, int64_t* sum1, int64_t* sum2,
                                    ssa_run_stats* stats);

/* ------------------------------------------------------------------ batches
 * Many networks of uneven size and trajectory count -- the parametric copies
 * and sweeps of Sec. 3.2 (StochRxn_ff) -- run together: one persistent
 * kernel per register bucket of the warp layout, on parallel branches of one
 * CUDA graph that also zeroes the sums and finalises every network.  The
 * graph is captured at the first launch and replayed for every seed.
 *
 * Network b runs n_traj[b] trajectories with ids opts->traj_offset + i and
 * Philox stream id (fourth counter word) opts->stream_id + b in
 * opts->precision, on one schedule: one trajectory per warp (W32, any
 * network) or one per thread (L, FP64 networks of at most 16 reactions and
 * 16 species without rate modifiers), each on its own branch of the graph.
 * Its results are bit-identical to ssa_ensemble_run of that network alone
 * with that schedule and stream_id = opts->stream_id + b; they do not depend
 * on the launch shape.  ssa_batch_network_stats reports the schedule.
 */
typedef struct ssa_batch ssa_batch; /* opaque, owned by the library */

/*
 * Creates a batch of n_models >= 1 networks.  Per network b (host arrays):
 *   models[b]: a model with at most 512 reactions (the batch keeps a
 *     reference: models must outlive the batch);
 *   n_traj[b] >= 1; t_end[b] > 0 and finite; n_grid[b] >= 1;
 *   grids: NULL (every grid uniform, g_k = k t_end / (n_grid - 1)) or an
 *     array of n_models host pointers, each NULL (uniform) or n_grid[b]
 *     ascending values in [0, t_end[b]] (copied).
 * opts (NULL for defaults): precision, max_events, traj_offset, stream_id
 * (stream_id + n_models <= 2^32), cuda_stream (where launches run), memory
 * (where ssa_batch_launch's output buffers live), block_threads (0 = 128
 * until ssa_batch_tune picks; else 64, 128 or 256), schedule: AUTO (networks
 * that fit the thread schedule start on it, as in ssa_ensemble_run, until
 * ssa_batch_tune times both schedules per network and keeps the faster),
 * WARP (every network per warp) or THREAD (every network per thread; each
 * must fit it, else SSA_EUNSUPPORTED); WARP and THREAD are not changed by
 * the tuner.  FP32 batches run the warp schedule (the thread schedule is
 * FP64).  Allocates one device slab for every network's grid, tables,
 * difference sums and results; synchronous.
 * Errors: SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA, SSA_EUNSUPPORTED.
 */
ssa_status ssa_batch_create(int32_t n_models, const ssa_model* const* models, const int64_t* n_traj,
                            const double* t_end, const int32_t* n_grid, const double* const* grids,
                            const ssa_run_opts* opts, ssa_batch** out);

/*
 * Autotuner, on a sample of the batch (the first ceil(n_traj[b] / 8)
 * trajectories of every network).  First, under schedule AUTO, every network
 * that fits both schedules is timed alone on each and keeps the faster (the
 * choice is recorded: ssa_batch_network_stats reports it, and later launches
 * reproduce its results exactly).  Then every launch shape of the warp
 * kernels (block size 64, 128 or 256; one kernel per register bucket or one
 * kernel for all) is timed and the fastest kept, which leaves results
 * unchanged.  Reports (each output pointer may be NULL): block_threads, split
 * (1 = one kernel per bucket), sample_ms (device time of the chosen shape on
 * the sample).  Synchronous.
 */
ssa_status ssa_batch_tune(ssa_batch* batch, int32_t* block_threads, int32_t* split, double* sample_ms);

/*
 * Runs the batch for `seed` on opts->cuda_stream.  means, vars, sums1, sums2:
 * NULL, or arrays of n_models pointers (each may be NULL) to G_b x S_b
 * buffers in opts->memory's space that receive network b's results.  The
 * results also stay in the batch's own device buffers (ssa_batch_result)
 * until the next launch.  stats: host struct or NULL (totals over all
 * networks; kernel_ms is the device time of the whole graph).  The call waits
 * for the stream when stats is non-NULL or host outputs are requested;
 * otherwise it only enqueues work.
 * Errors: SSA_EINVAL, SSA_ECUDA, SSA_EOVERFLOW (only detectable when the call
 * waits: a count reached SSA_STATE_MAX, or N * max_x^2 could leave int64).
 */
ssa_status ssa_batch_launch(ssa_batch* batch, uint64_t seed, double* const* means, double* const* vars,
                            int64_t* const* sums1, int64_t* const* sums2, ssa_run_stats* stats);

/* Device pointers to network `index`'s results of the last launch (each
 * output may be NULL); valid until the next launch or ssa_batch_destroy. */
ssa_status ssa_batch_result(const ssa_batch* batch, int32_t index, const double** mean, const double** var,
                            const int64_t** sum1, const int64_t** sum2);

/* Totals of network `index` (events, truncated, overflowed, max_x) from the
 * last launch that waited for the stream, and the schedule it runs on
 * (SSA_SCHED_THREAD or SSA_SCHED_WARP); kernel_ms is 0. */
ssa_status ssa_batch_network_stats(const ssa_batch* batch, int32_t index, ssa_run_stats* out);

/* Releases a batch.  NULL is ignored.  No launch of it may be pending. */
void ssa_batch_destroy(ssa_batch* batch);

/*
 * One-shot batch: ssa_batch_create, one ssa_batch_launch with `seed` and the
 * given means / vars (arrays of n_models pointers, opts->memory's space), a
 * wait for the stream, and ssa_batch_destroy.
 */
ssa_status ssa_batch_run(int32_t n_models, const ssa_model* const* models, const int64_t* n_traj,
                         const double* t_end, const int32_t* n_grid, const double* const* grids, uint64_t seed,
                         const ssa_run_opts* opts, double* const* means, double* const* vars);

#ifdef __cplusplus
}
#endif

#endif /* SSA_H_ */
