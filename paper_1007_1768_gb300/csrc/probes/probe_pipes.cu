// Throughput probes for the ALU pipes the SSA step uses (measured peaks of the roofline).
// Every kernel: bounded loops, one store per thread into an output buffer of
// exactly grid*block elements.
#include <cstdio>
#include <cstdint>
#include <cuda_runtime.h>

#define CK(x) do { cudaError_t e = (x); if (e != cudaSuccess) { printf("CUDA %s at %d\n", cudaGetErrorString(e), __LINE__); return 1; } } while (0)

constexpr int ITERS = 4096;

__global__ void k_dadd(double* out, double s) {
  double a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    a0 = __dadd_rn(a0, s); a1 = __dadd_rn(a1, s); a2 = __dadd_rn(a2, s); a3 = __dadd_rn(a3, s);
    a4 = __dadd_rn(a4, s); a5 = __dadd_rn(a5, s); a6 = __dadd_rn(a6, s); a7 = __dadd_rn(a7, s);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
__global__ void k_dmul(double* out, double s) {
  double a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    a0 = __dmul_rn(a0, s); a1 = __dmul_rn(a1, s); a2 = __dmul_rn(a2, s); a3 = __dmul_rn(a3, s);
    a4 = __dmul_rn(a4, s); a5 = __dmul_rn(a5, s); a6 = __dmul_rn(a6, s); a7 = __dmul_rn(a7, s);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
__global__ void k_dfma(double* out, double s) {
  double a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    a0 = __fma_rn(a0, s, s); a1 = __fma_rn(a1, s, s); a2 = __fma_rn(a2, s, s); a3 = __fma_rn(a3, s, s);
    a4 = __fma_rn(a4, s, s); a5 = __fma_rn(a5, s, s); a6 = __fma_rn(a6, s, s); a7 = __fma_rn(a7, s, s);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
__global__ void k_ffma(double* out, float s) {
  float a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    a0 = __fmaf_rn(a0, s, s); a1 = __fmaf_rn(a1, s, s); a2 = __fmaf_rn(a2, s, s); a3 = __fmaf_rn(a3, s, s);
    a4 = __fmaf_rn(a4, s, s); a5 = __fmaf_rn(a5, s, s); a6 = __fmaf_rn(a6, s, s); a7 = __fmaf_rn(a7, s, s);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}
// int64 -> double conversion
__global__ void k_i2d(double* out, long long s) {
  long long b = threadIdx.x;
  double acc0 = 0, acc1 = 0;
  long long v0 = b, v1 = b + 1, v2 = b + 2, v3 = b + 3;
  unsigned r0 = 0, r1 = 0, r2 = 0, r3 = 0;
  for (int i = 0; i < ITERS; ++i) {
    double d0 = __ll2double_rn(v0 + i), d1 = __ll2double_rn(v1 + i), d2 = __ll2double_rn(v2 + i), d3 = __ll2double_rn(v3 + i);
    r0 ^= __double2hiint(d0); r1 ^= __double2hiint(d1); r2 ^= __double2hiint(d2); r3 ^= __double2hiint(d3);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)(r0 ^ r1 ^ r2 ^ r3) + acc0 + acc1;
}
// double division
__global__ void k_ddiv(double* out, double s) {
  double a0 = threadIdx.x + 1.0, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  for (int i = 0; i < ITERS / 8; ++i) {
    a0 = __ddiv_rn(s, a0) + 1.0; a1 = __ddiv_rn(s, a1) + 1.0; a2 = __ddiv_rn(s, a2) + 1.0; a3 = __ddiv_rn(s, a3) + 1.0;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = a0 + a1 + a2 + a3;
}
// 32-bit integer multiply-add
__global__ void k_imad(double* out, unsigned s) {
  unsigned a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    a0 = a0 * s + 7u; a1 = a1 * s + 7u; a2 = a2 * s + 7u; a3 = a3 * s + 7u;
    a4 = a4 * s + 7u; a5 = a5 * s + 7u; a6 = a6 * s + 7u; a7 = a7 * s + 7u;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)(a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7);
}
// 32x32 -> hi 32
__global__ void k_umulhi(double* out, unsigned s) {
  unsigned a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    a0 = __umulhi(a0, s) ^ a0; a1 = __umulhi(a1, s) ^ a1; a2 = __umulhi(a2, s) ^ a2; a3 = __umulhi(a3, s) ^ a3;
    a4 = __umulhi(a4, s) ^ a4; a5 = __umulhi(a5, s) ^ a5; a6 = __umulhi(a6, s) ^ a6; a7 = __umulhi(a7, s) ^ a7;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)(a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7);
}
// 64x64 -> hi 64
__global__ void k_umul64hi(double* out, unsigned long long s) {
  unsigned long long a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  for (int i = 0; i < ITERS; ++i) {
    a0 = __umul64hi(a0, s) ^ (a0 + 1); a1 = __umul64hi(a1, s) ^ (a1 + 1); a2 = __umul64hi(a2, s) ^ (a2 + 1); a3 = __umul64hi(a3, s) ^ (a3 + 1);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)(a0 ^ a1 ^ a2 ^ a3);
}
// logical ops
__global__ void k_lop(double* out, unsigned s) {
  unsigned a0 = threadIdx.x, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5, a6 = a0 + 6, a7 = a0 + 7;
  for (int i = 0; i < ITERS; ++i) {
    a0 = (a0 ^ s) + a1; a1 = (a1 ^ s) + a2; a2 = (a2 ^ s) + a3; a3 = (a3 ^ s) + a4;
    a4 = (a4 ^ s) + a5; a5 = (a5 ^ s) + a6; a6 = (a6 ^ s) + a7; a7 = (a7 ^ s) + a0;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)(a0 ^ a1 ^ a2 ^ a3 ^ a4 ^ a5 ^ a6 ^ a7);
}
// shared-memory int64 atomics, distinct addresses per lane
__global__ void k_satom(double* out, unsigned long long s) {
  __shared__ unsigned long long buf[4096];
  for (int i = threadIdx.x; i < 4096; i += blockDim.x) buf[i] = 0;
  __syncthreads();
  unsigned idx = threadIdx.x;
  for (int i = 0; i < ITERS / 4; ++i) {
    atomicAdd(&buf[(idx + 0 * 1024u + (unsigned)i * 33u) & 4095u], s);
    atomicAdd(&buf[(idx + 1 * 1024u + (unsigned)i * 33u) & 4095u], s);
    atomicAdd(&buf[(idx + 2 * 1024u + (unsigned)i * 33u) & 4095u], s);
    atomicAdd(&buf[(idx + 3 * 1024u + (unsigned)i * 33u) & 4095u], s);
  }
  __syncthreads();
  out[blockIdx.x * blockDim.x + threadIdx.x] = (double)buf[threadIdx.x & 4095u];
}

typedef void (*launcher)(int, int, double*);

int main() {
  int dev = 0;
  CK(cudaSetDevice(dev));
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, dev));
  int clk_khz = 0;
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
  printf("device %s SMs %d cc %d.%d clock(attr) %d kHz smemPerBlockOptin %zu regsPerSM %d\n",
         p.name, p.multiProcessorCount, p.major, p.minor, clk_khz, p.sharedMemPerBlockOptin, p.regsPerMultiprocessor);
  const int sms = p.multiProcessorCount;
  const int block = 256;
  const int grid = sms * 8;
  double* out = nullptr;
  CK(cudaMalloc(&out, sizeof(double) * grid * block));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  struct T { const char* name; double ops_per_thread; int which; };
  T tests[] = {
    {"DADD", 8.0 * ITERS, 0}, {"DMUL", 8.0 * ITERS, 1}, {"DFMA", 8.0 * ITERS, 2}, {"FFMA", 8.0 * ITERS, 3},
    {"I2F.F64(+hi xor)", 4.0 * ITERS, 4}, {"DDIV(+DADD)", 4.0 * (ITERS / 8), 5}, {"IMAD32", 8.0 * ITERS, 6},
    {"UMULHI32(+xor)", 8.0 * ITERS, 7}, {"UMUL64HI(+xor,add)", 4.0 * ITERS, 8}, {"XOR+ADD32", 8.0 * ITERS, 9},
    {"ATOMS.ADD.64 shared", 4.0 * (ITERS / 4), 10},
  };
  for (auto& t : tests) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      CK(cudaEventRecord(e0));
      switch (t.which) {
        case 0: k_dadd<<<grid, block>>>(out, 1.0000001); break;
        case 1: k_dmul<<<grid, block>>>(out, 0.9999999); break;
        case 2: k_dfma<<<grid, block>>>(out, 0.5); break;
        case 3: k_ffma<<<grid, block>>>(out, 0.5f); break;
        case 4: k_i2d<<<grid, block>>>(out, 3); break;
        case 5: k_ddiv<<<grid, block>>>(out, 3.0); break;
        case 6: k_imad<<<grid, block>>>(out, 2654435761u); break;
        case 7: k_umulhi<<<grid, block>>>(out, 2654435761u); break;
        case 8: k_umul64hi<<<grid, block>>>(out, 0x9E3779B97F4A7C15ull); break;
        case 9: k_lop<<<grid, block>>>(out, 0x5bd1e995u); break;
        case 10: k_satom<<<grid, block>>>(out, 3ull); break;
      }
      CK(cudaGetLastError());
      CK(cudaEventRecord(e1));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best) best = ms;
    }
    double total = t.ops_per_thread * (double)grid * block;
    double rate = total / (best * 1e-3);
    printf("%-24s %9.3f ms  %10.3f Gop/s  per-SM-per-clk@1.9GHz %8.3f\n", t.name, best, rate * 1e-9,
           rate / sms / 1.9e9);
  }
  CK(cudaFree(out));
  return 0;
}
