// Latency of the step's parts and of pairs of them in one block (one warp, clock64).
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>
#include "../ssa_thread_kernel.cuh"

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)
constexpr int ITER = 512;
using namespace ssa_impl;

__device__ __forceinline__ double quotient_nb(unsigned long long Eb, double a0, bool& okall) {
  bool ok;
  const unsigned long long qb = ssa_sf::div_pos(Eb, (unsigned long long)obits(a0), ok);
  okall &= ok;
  return __longlong_as_double((long long)qb);
}

template <int MODE>
__global__ void kprobe(long long* cyc, unsigned long long* out) {
  __shared__ uint64_t inv[512], lnf[512];
  for (int i = threadIdx.x; i < 512; i += blockDim.x) { inv[i] = d_log_tables.inv[i]; lnf[i] = d_log_tables.lnf[i]; }
  __syncthreads();
  Traj<10, 4> q;
  for (int j = 0; j < 10; ++j) q.av[j] = 0x3FF0000000000000ULL + (unsigned long long)(j + threadIdx.x) * 12345ULL;
  unsigned long long E = 0x4000123456789ABCULL + threadIdx.x;
  double a0s = 3.5;
  unsigned long long acc = 0;
  uint32_t n = threadIdx.x;
  long long t0 = clock64();
  for (int it = 0; it < ITER; ++it) {
    double a0new = a0s;
    if (MODE == 5 || MODE == 6) {
      bool okall = true;
      const double tau = quotient_nb(E, a0s, okall);
      E ^= (unsigned long long)obits(tau) & 0xFFFULL;
      acc += (unsigned long long)obits(tau) + (okall ? 0 : 1);
    }
    if (MODE == 6) {
      const double a0 = prefix_sums(10, q);
      q.av[it % 10] ^= (unsigned long long)obits(a0) & 0xFULL;
      acc += (unsigned long long)obits(a0);
      a0new = a0;
    }
    if (MODE == 7 || MODE == 8) {   // prefix + 60 dependent-pair ALU ops (xor/add/shift), no multiplies
      unsigned w0 = (unsigned)E, w1 = (unsigned)(E >> 32);
#pragma unroll
      for (int u = 0; u < 30; ++u) { w0 = (w0 ^ (w1 >> 3)) + 0x9e3779b9u; w1 = (w1 ^ (w0 << 5)) + 0x7f4a7c15u; }
      E = ((unsigned long long)w1 << 32) | w0;
      acc += E;
    }
    if (MODE == 8 || MODE == 9) {
      const double a0 = prefix_sums(10, q);
      q.av[it % 10] ^= (unsigned long long)obits(a0) & 0xFULL;
      acc += (unsigned long long)obits(a0);
      a0new = a0;
    }
    if (MODE == 9 || MODE == 10) {
      const EventRandom r = event_random(n, 77ULL, 0, 123, 456, inv, lnf);
      n += (uint32_t)(r.E & 1ULL) + 1;
      acc += r.u2;
    }
    if (MODE == 1 || MODE == 2 || MODE == 3) {   // uses last iteration's a0: independent of this prefix
      const double tau = quotient(E, a0s);
      E ^= (unsigned long long)obits(tau) & 0xFFFULL;
      acc += (unsigned long long)obits(tau);
    }
    if (MODE == 0 || MODE == 2 || MODE == 3) {
      const double a0 = prefix_sums(10, q);
      q.av[it % 10] ^= (unsigned long long)obits(a0) & 0xFULL;   // loop-carried
      acc += (unsigned long long)obits(a0);
      a0new = a0;
    }
    a0s = (MODE == 1 || MODE == 5) ? a0s : a0new;
    if (MODE == 3 || MODE == 4) {
      const EventRandom r = event_random(n, 77ULL, 0, 123, 456, inv, lnf);
      n += (uint32_t)(r.E & 1ULL) + 1;
      acc += r.u2;
    }
  }
  long long t1 = clock64();
  if (threadIdx.x == 0) cyc[0] = t1 - t0;
  out[threadIdx.x] = acc + q.av[3];
}

template <int MODE>
int run(const char* name, long long* dc, unsigned long long* dout) {
  kprobe<MODE><<<1, 32>>>(dc, dout);
  CK(cudaGetLastError());
  CK(cudaDeviceSynchronize());
  long long h; CK(cudaMemcpy(&h, dc, 8, cudaMemcpyDeviceToHost));
  printf("%-40s %8.1f cycles per iteration\n", name, (double)h / ITER);
  return 0;
}

int main() {
  long long* dc; unsigned long long* dout;
  CK(cudaMalloc(&dc, 64)); CK(cudaMalloc(&dout, 8 * 64));
  run<0>("prefix chain (9 DADD)", dc, dout);
  run<1>("integer quotient", dc, dout);
  run<2>("prefix + quotient", dc, dout);
  run<3>("prefix + quotient + event_random", dc, dout);
  run<4>("event_random", dc, dout);
  run<5>("quotient, no fallback branch", dc, dout);
  run<6>("prefix + quotient (no branch)", dc, dout);
  run<7>("60 ALU ops", dc, dout);
  run<8>("prefix + 60 ALU ops", dc, dout);
  run<9>("prefix + event_random", dc, dout);
  return 0;
}
