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
};

// Slots of the per-run device totals.
enum { kStatEvents = 0, kStatTruncated = 1, kStatOverflowed = 2, kStatMaxX = 3, kStatCount = 8 };

// Arguments of the simulation kernels.
struct RunArgs {
  DevModel m;
  int32_t G;
  int64_t N;
  uint64_t traj_offset;
  uint64_t seed;
  uint64_t stream_id;
  int64_t max_events;
  double t_end;
  const double* grid;                 // [G]
  unsigned long long* D1;             // [G * S] per-grid sums of count changes (global)
  unsigned long long* D2;             // [G * S] per-grid sums of square changes (global)
  unsigned long long* counter;        // next trajectory index
  unsigned long long* stats;          // [kStatCount]
  int64_t* traj_events;               // [N] or null
  uint64_t* traj_hash;                // [N] or null
  int32_t* traj_flags;                // [N] or null
  unsigned long long* device_totals;  // [4] or null (caller's running totals)
};

// Shared-memory layout of the thread-per-trajectory kernel (bytes).
struct ThreadSmem {
  size_t log_inv, log_lnf, c, rinfo, nu_ptr, nu_idx, nu_val, x, d1, d2, total;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline ThreadSmem thread_smem_layout(int S, int M, int nnz, int G, int threads,
                                                         bool shared_d) {
  ThreadSmem L;
  size_t o = 0;
  L.log_inv = o; o += 128 * 8;
  L.log_lnf = o; o += 128 * 8;
  L.c = o; o += align_up((size_t)M * 8, 16);
  L.rinfo = o; o += align_up((size_t)M * 4, 16);
  L.nu_ptr = o; o += align_up((size_t)(M + 1) * 4, 16);
  L.nu_idx = o; o += align_up((size_t)nnz * 4, 16);
  L.nu_val = o; o += align_up((size_t)nnz * 4, 16);
  L.x = o; o += align_up((size_t)S * threads * 4, 16);
  if (shared_d) {
    L.d1 = o; o += (size_t)G * S * 8;
    L.d2 = o; o += (size_t)G * S * 8;
  } else {
    L.d1 = L.d2 = 0;
  }
  L.total = o;
  return L;
}

// Launch helpers (ssa_kernels.cu).  Return cudaSuccess or the launch error.
cudaError_t launch_thread_kernel(const RunArgs& a, int blocks, int threads, bool shared_d,
                                 size_t smem_bytes, cudaStream_t stream);
cudaError_t launch_finalize(const unsigned long long* D1, const unsigned long long* D2, int G, int S,
                            int64_t N, const int32_t* x0, double* mean, double* var, int64_t* sum1,
                            int64_t* sum2, cudaStream_t stream);
cudaError_t launch_uniform_grid(double* grid, int G, double t_end, cudaStream_t stream);
// Largest M the thread kernel is instantiated for.
constexpr int kThreadMaxM = 16;
cudaError_t thread_kernel_set_smem(int M, bool shared_d, size_t smem_bytes);

// Host image of a model's device tables (see DevModel for the layout), for
// entry points that place the tables themselves.
struct ModelImageView {
  int32_t S, M, nnz, ndep;
  const unsigned char* image;
  size_t bytes;
  size_t off_c, off_rinfo, off_nu_ptr, off_nu_idx, off_nu_val, off_x0, off_dep_ptr, off_dep_idx;
};

}  // namespace ssa_impl

struct ssa_model;

namespace ssa_impl {
// Accessors implemented in ssa_api.cu.
bool model_image_view(const ssa_model* m, ModelImageView* v);
}  // namespace ssa_impl

#endif  // SSA_INTERNAL_H_
