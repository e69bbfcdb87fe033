// Latency / lane-activity probes of the FP64 and integer pipes: dependent chains
// timed with clock64 by one warp per SM, with all 32 lanes or only lane 0 active;
// full grid where only one lane per warp works.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

constexpr int CHAIN = 2048;

// mode: 0 dadd, 1 dmul, 2 ddiv, 3 iadd32, 4 imad32, 5 umul64hi, 6 dfma,
// 7 two independent dadd chains (cycles per pair)
template <int MODE>
__device__ __forceinline__ void chain(double& d, unsigned long long& u, unsigned& w) {
  if (MODE == 0) { d = __dadd_rn(d, 1.0000000001); }
  if (MODE == 1) { d = __dmul_rn(d, 0.9999999999); }
  if (MODE == 2) { d = __ddiv_rn(1.0000001, d) ; }
  if (MODE == 3) { w = w + 0x9e3779b9u; w ^= (w >> 3); }
  if (MODE == 4) { w = w * 2654435761u + 1u; }
  if (MODE == 5) { u = __umul64hi(u, 0x9E3779B97F4A7C15ull) + u; }
  if (MODE == 6) { d = __fma_rn(d, 0.9999999, 1e-9); }
  if (MODE == 7) {
    d = __dadd_rn(d, 1.0000000001);
    u = (unsigned long long)__double_as_longlong(__dadd_rn(__longlong_as_double((long long)u), 1.5));
  }
}

template <int MODE>
__global__ void k_lat(long long* cycles, double* out, int active_lanes) {
  const int lane = threadIdx.x & 31;
  double d = 1.0 + lane;
  unsigned long long u = (MODE == 7) ? (unsigned long long)__double_as_longlong(2.0 + lane) : 12345ULL + lane;
  unsigned w = 777 + lane;
  long long t0 = 0, t1 = 0;
  if (lane < active_lanes) {
    t0 = clock64();
    for (int i = 0; i < CHAIN; ++i) chain<MODE>(d, u, w);
    t1 = clock64();
  }
  __syncwarp();
  if (lane == 0) cycles[blockIdx.x] = t1 - t0;
  out[blockIdx.x * blockDim.x + threadIdx.x] = d + (double)u + (double)w;
}

// throughput with `active_lanes` lanes per warp working, 8 independent chains each
template <int MODE>
__global__ void k_thr(double* out, int active_lanes) {
  const int lane = threadIdx.x & 31;
  double d0 = 1.0 + lane, d1 = d0 + 1, d2 = d0 + 2, d3 = d0 + 3;
  unsigned long long u0 = lane, u1 = lane + 1, u2 = lane + 2, u3 = lane + 3;
  unsigned w0 = lane, w1 = lane + 1, w2 = lane + 2, w3 = lane + 3;
  if (lane < active_lanes) {
    for (int i = 0; i < CHAIN / 4; ++i) {
      chain<MODE>(d0, u0, w0); chain<MODE>(d1, u1, w1); chain<MODE>(d2, u2, w2); chain<MODE>(d3, u3, w3);
    }
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = d0 + d1 + d2 + d3 + (double)(u0 ^ u1 ^ u2 ^ u3) + (double)(w0 ^ w1 ^ w2 ^ w3);
}

template <int MODE>
int run(const char* name, int sms, long long* d_cyc, double* d_out, cudaEvent_t e0, cudaEvent_t e1) {
  long long h[1024];
  for (int act : {32, 1}) {
    k_lat<MODE><<<sms, 32>>>(d_cyc, d_out, act);
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(h, d_cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost));
    long long mx = 0; for (int i = 0; i < sms; ++i) mx = h[i] > mx ? h[i] : mx;
    printf("%-10s latency  active=%2d : %7.2f cycles/op (1 warp per SM)\n", name, act, (double)mx / CHAIN);
  }
  for (int act : {32, 1}) {
    float best = 1e30f;
    for (int r = 0; r < 3; ++r) {
      CK(cudaEventRecord(e0));
      k_thr<MODE><<<sms * 16, 256>>>(d_out, act);
      CK(cudaGetLastError());
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      float ms; CK(cudaEventElapsedTime(&ms, e0, e1)); if (ms < best) best = ms;
    }
    double warp_instr = (double)sms * 16 * 256 / 32 * CHAIN;
    printf("%-10s throughput active=%2d : %8.3f ms, %8.3f warp-instr/clk/SM @2.0GHz, lane-ops %.3g/s\n", name, act, best,
           warp_instr / (best * 1e-3) / sms / 2.0e9, warp_instr * act / (best * 1e-3));
  }
  return 0;
}

int main() {
  cudaDeviceProp p; CK(cudaGetDeviceProperties(&p, 0));
  int sms = p.multiProcessorCount;
  long long* d_cyc; double* d_out;
  CK(cudaMalloc(&d_cyc, sizeof(long long) * 1024));
  CK(cudaMalloc(&d_out, sizeof(double) * sms * 16 * 256));
  cudaEvent_t e0, e1; CK(cudaEventCreate(&e0)); CK(cudaEventCreate(&e1));
  if (run<0>("DADD", sms, d_cyc, d_out, e0, e1)) return 1;
  if (run<1>("DMUL", sms, d_cyc, d_out, e0, e1)) return 1;
  if (run<6>("DFMA", sms, d_cyc, d_out, e0, e1)) return 1;
  if (run<7>("2xDADD", sms, d_cyc, d_out, e0, e1)) return 1;
  if (run<2>("DDIV", sms, d_cyc, d_out, e0, e1)) return 1;
  if (run<3>("IADD+SHF", sms, d_cyc, d_out, e0, e1)) return 1;
  if (run<4>("IMAD", sms, d_cyc, d_out, e0, e1)) return 1;
  if (run<5>("UMUL64HI", sms, d_cyc, d_out, e0, e1)) return 1;
  return 0;
}
