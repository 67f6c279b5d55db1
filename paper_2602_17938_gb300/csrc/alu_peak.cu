// Min/max throughput microbenchmark: the ALU-pipe peak that the median
// kernels are measured against.  Each thread runs compare-exchange chains on
// eight independent register pairs (no memory traffic in the loop), so the
// kernel is bound by the min/max issue rate alone.  Separate from the
// detect-and-clean library; only the benchmark loads it.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) minmax_f32(float* out, int iters, float seed) {
  float a[8], b[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    a[j] = seed * (threadIdx.x + j);
    b[j] = seed * (blockIdx.x - j);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float lo = fminf(a[j], b[(j + r) & 7]);
        const float hi = fmaxf(a[j], b[(j + r) & 7]);
        a[j] = lo;
        b[(j + r) & 7] = hi;
      }
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j] - b[j];
  if (s == 12345.0f) out[blockIdx.x] = s;  // keeps the chains live
}

__device__ __forceinline__ uint32_t vmin2(uint32_t x, uint32_t y) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(y));
  return r;
}
__device__ __forceinline__ uint32_t vmax2(uint32_t x, uint32_t y) {
  uint32_t r;
  asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(y));
  return r;
}

__global__ void __launch_bounds__(kThreads) minmax_u16x2(uint32_t* out, int iters, uint32_t seed) {
  uint32_t a[8], b[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    a[j] = seed * (threadIdx.x + 3 * j + 1);
    b[j] = seed ^ (blockIdx.x * 7919u + j);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t lo = vmin2(a[j], b[(j + r) & 7]);
        const uint32_t hi = vmax2(a[j], b[(j + r) & 7]);
        a[j] = lo;
        b[(j + r) & 7] = hi;
      }
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s ^= a[j] + b[j];
  if (s == 0x12345u) out[blockIdx.x] = s;
}

template <class Launch>
int time_kernel(Launch launch, double ops, double* gops) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
  launch();  // warm-up
  float best = 1e30f;
  for (int rep = 0; rep < 5; ++rep) {
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *gops = ops / (best * 1e-3) / 1e9;
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace

extern "C" {

// Measured min/max throughput on `device`, in 10^9 two-input min/max
// operations per second: f32 (one element per op) and u16x2 (two elements
// per op, reported per instruction).  Returns 0 on success.
int alu_minmax_peak(int device, double* f32_gops, double* u16x2_gops) {
  if (cudaSetDevice(device) != cudaSuccess) return -1;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int blocks = sms * 8;
  const int iters = 2048;
  const double ops = (double)blocks * kThreads * iters * 8 * 8 * 2;
  void* buf = nullptr;
  if (cudaMalloc(&buf, blocks * sizeof(uint32_t)) != cudaSuccess) return -1;
  int rc = time_kernel([&] { minmax_f32<<<blocks, kThreads>>>((float*)buf, iters, 1.0001f); },
                       ops, f32_gops);
  if (rc == 0)
    rc = time_kernel([&] { minmax_u16x2<<<blocks, kThreads>>>((uint32_t*)buf, iters, 2654435761u); },
                     ops, u16x2_gops);
  cudaFree(buf);
  return rc;
}

}  // extern "C"
