// The core kernel's selection networks, each run alone: how many instructions
// (per pipe) one unit of work executes and how close the network comes to the
// ALU pipe's peak when nothing else competes for the SM.  A unit is what one
// thread of core_kernel does in one go:
//   0  a pair of 4x2 med5 blocks on packed uint16 (16 outputs, 8 pixels wide),
//   1  a pair of 8x2 med3 blocks on packed uint16 (32 outputs),
//   2  one 5x5 median of float S (an S' item),
//   3  one 7x7 median of int keys of uint16 med3 values (an F item),
//   4  one masked 5x5 median of a uint16 frame (a replaced pixel, ~3% flagged),
//   5  the loop and load around a unit, nothing else.
// Inputs are sky-like uint16 values (300..499) staged in shared memory with
// the core kernel's row pitch; units walk the array in the same index
// pattern as the kernel's.  Every access stays inside the staged rows (the
// unit ranges are bounded below).  A stand-alone diagnostic, not part of the
// library: compile with nvcc for sm_103a and run under ncu for the per-pipe
// instruction counts; it prints the CUDA-event time of each network.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "lacos_kernels.cuh"

namespace {
using namespace lacos;

constexpr int kW = 80;     // X row pitch (R6 of a 32x64 tile)
constexpr int kWS = 68;    // S row pitch (R2)
constexpr int kRows = 48;  // staged rows

template <int MODE>
__global__ void __launch_bounds__(256, 4) net_unit(const uint16_t* __restrict__ g, unsigned* sink, int iters) {
  __shared__ __align__(16) uint16_t X[kRows * kW];
  __shared__ __align__(16) float S[kRows * kWS];
  __shared__ __align__(16) uint8_t Mb[kRows * kW];
  for (int i = threadIdx.x; i < kRows * kW; i += blockDim.x) {
    const uint16_t v = g[(blockIdx.x * 977u + i) & 0xfffffu];
    X[i] = v;
    Mb[i] = (v & 31) == 0;
  }
  for (int i = threadIdx.x; i < kRows * kWS; i += blockDim.x)
    S[i] = (float)g[(blockIdx.x * 531u + i) & 0xfffffu] * 0.37f;
  __syncthreads();
  unsigned acc = 0;
  for (int it = 0; it < iters; ++it) {
    const int u = (threadIdx.x + it * 37) % 153;
    if (MODE == 0) {  // rows ly0 .. ly0 + 5 + 18 <= 39, columns lx0 .. lx0 + 7 <= 71
      const int ly0 = (u / 17) * 2, lx0 = (u % 17) * 4;
      const QuadLoaderU16<8, 18, kW> ld{X + ly0 * kW + lx0};
      U16x2 m5[8];
      blk_med5_4x2_ld<U16x2>(ld, m5);
#pragma unroll
      for (int e = 0; e < 8; ++e) acc ^= m5[e].v;
    } else if (MODE == 1) {  // rows .. ly0 + 3 + 20 <= 41, columns .. lx0 + 11 <= 75
      const int v = u % 90;
      const int ly0 = (v / 9) * 2, lx0 = (v % 9) * 8;
      const QuadLoaderU16<10, 20, kW> ld{X + ly0 * kW + lx0};
      U16x2 m3[16];
      blk_med3_8x2_ld<U16x2>(ld, m3);
#pragma unroll
      for (int e = 0; e < 16; ++e) acc ^= m3[e].v;
    } else if (MODE == 2) {  // rows .. 22, columns .. 64 of a 68-wide row
      const int y = 2 + (u / 16) * 2, x = 2 + (u % 16) * 4;
      const float* wb = S + (y - 2) * kWS + x - 2;
      const auto ld5 = [&](int e) { return wb[(e / 5) * kWS + e % 5]; };
      float m;
      med5x5_ld<float>(ld5, &m);
      acc ^= __float_as_uint(m);
    } else if (MODE == 3) {  // rows .. 24, columns .. 66
      const int y = 3 + (u / 16) * 2, x = 3 + (u % 16) * 4;
      const uint16_t* w7 = X + (y - 3) * kW + x - 3;
      const auto ld7 = [&](int e) { return (int)w7[(e / 7) * kW + e % 7]; };
      int m7;
      med7x7_ld<int>(ld7, &m7);
      acc ^= (unsigned)m7;
    } else if (MODE == 4) {  // rows .. 22, columns .. 64
      const int y = 2 + (u / 16) * 2, x = 2 + (u % 16) * 4;
      uint16_t o = 0;
      maskmed5<uint16_t>(X, Mb, kW, y * kW + x, o);
      acc ^= o;
    } else {
      acc ^= X[(u / 17) * 2 * kW + (u % 17) * 4];
    }
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

int main(int argc, char** argv) {
  const int iters = argc > 1 ? atoi(argv[1]) : 64;
  const int blocks = 152 * 4 * 4;
  std::vector<uint16_t> h(1 << 20);
  unsigned s = 12345u;
  for (auto& v : h) {
    s = s * 1664525u + 1013904223u;
    v = (uint16_t)(300 + ((s >> 16) % 200));
  }
  uint16_t* g = nullptr;
  unsigned* sink = nullptr;
  if (cudaMalloc(&g, h.size() * 2) != cudaSuccess || cudaMalloc(&sink, (size_t)blocks * 256 * 4) != cudaSuccess) return 1;
  cudaMemcpy(g, h.data(), h.size() * 2, cudaMemcpyHostToDevice);
  const char* names[] = {"med5_4x2_pair_u16x2", "med3_8x2_pair_u16x2", "med5x5_f32", "med7x7_int",
                         "maskmed5_u16", "loop_only"};
  void (*ks[])(const uint16_t*, unsigned*, int) = {net_unit<0>, net_unit<1>, net_unit<2>,
                                                   net_unit<3>, net_unit<4>, net_unit<5>};
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const double units = (double)blocks * 256 * iters;
  for (int m = 0; m < 6; ++m) {
    ks[m]<<<blocks, 256>>>(g, sink, iters);  // warm-up
    cudaEventRecord(a);
    ks[m]<<<blocks, 256>>>(g, sink, iters);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    printf("{\"network\": \"%s\", \"ms\": %.4f, \"units\": %.0f}\n", names[m], ms, units);
  }
  const cudaError_t e = cudaDeviceSynchronize();
  cudaFree(g);
  cudaFree(sink);
  if (e != cudaSuccess) {
    fprintf(stderr, "%s\n", cudaGetErrorString(e));
    return 1;
  }
  return 0;
}
