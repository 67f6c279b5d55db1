// Device code of the L.A.Cosmic detect-and-clean iteration (sm_103a).
//
// Iteration k is two kernels:
//   core_kernel (one per frame dtype): per TH x TW tile, stages the original
//     frame X0 and the cumulative mask M_{k-1} with a 6-pixel halo and
//     rebuilds the working image I_{k-1} = R(X0, M_{k-1}) on the tile + 4
//     (step 7 of the previous iteration: unflagged pixels keep X0, flagged
//     ones take the masked median of unflagged X0, so I depends only on X0
//     and the mask); then med5(I) on the tile + 2 and med3(I) on the tile + 3
//     (register blocks of shared min/max networks), L+, N and S per pixel,
//     and S' = S - med5(S) with F and the objlim test on compacted lists of
//     the pixels where a test can pass (steps 1-5).  It writes three
//     bit-planes: S' > sigclip and S' > sigfrac*sigclip (both excluding
//     saturated pixels) and the candidates.  Levels after the first skip the
//     tiles whose inputs did not change;
//   grow_kernel: step 6 on 32-pixel words, M_k = M_{k-1} | g2, whether the
//     level found new pixels, and the tiles the next level must recompute.
// For uint16 frames 2N and 1/(2N) are read from a 65536-entry table indexed by
// med5, built once per request (ntab_kernel), S = L+/(2N) is formed from the
// reciprocal with two Markstein corrections (div_recip), and the dense
// networks run on packed pairs.  With saturated-star protection the grown
// saturated set is built once per request (satseed_kernel, satgrow_kernel).
// finalize_kernel writes the cleaned frame R(X0, M) and the uint8 mask.
//
// Every stage evaluates its own array at in-frame positions only and reads
// out-of-frame neighbours at clamped coordinates (clamp-to-edge per stage).
//
// Exactness: all float arithmetic uses the explicit round-to-nearest
// intrinsics in the same operation order as the float32 CPU definition (the
// uint16 path divides through a reciprocal form that rounds like IEEE division:
// Markstein's theorem, checked exhaustively by lacos_selftest_division), the
// translation unit is compiled with -fmad=false, and medians are selections
// (min/max networks), so results are bit-identical to it.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <type_traits>

#include "../../include/lacos.h"

namespace lacos_net {
template <class K> __device__ __forceinline__ K neg_inf();
template <class K> __device__ __forceinline__ K pos_inf();
template <> __device__ __forceinline__ float neg_inf<float>() { return -__int_as_float(0x7f800000); }
template <> __device__ __forceinline__ float pos_inf<float>() { return __int_as_float(0x7f800000); }
}  // namespace lacos_net

__device__ __forceinline__ float MN(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float MX(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ int MN(int a, int b) { return min(a, b); }
__device__ __forceinline__ int MX(int a, int b) { return max(a, b); }

// Two 16-bit keys per register: one min/max instruction compares both halves.
struct U16x2 {
  uint32_t v;
};
__device__ __forceinline__ U16x2 MN(U16x2 a, U16x2 b) {
  U16x2 r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r.v) : "r"(a.v), "r"(b.v));
  return r;
}
__device__ __forceinline__ U16x2 MX(U16x2 a, U16x2 b) {
  U16x2 r;
  asm("max.u16x2 %0, %1, %2;" : "=r"(r.v) : "r"(a.v), "r"(b.v));
  return r;
}

#include "networks.cuh"
#include "gain_math.cuh"

namespace lacos {

// Threads per CTA of the kernels other than the core kernel.
constexpr int kBlock = 256;

// Tile geometry of a core-kernel variant: TH x TW output pixels per tile, NT
// threads per CTA.  Regions grown around the tile are Reg<H, C>: H rows and
// C columns on each side, row-major in shared memory, idx(0, 0) the tile's
// first pixel.  Staged input regions carry 8 extra columns on each side
// (more than the 6 and 3 the stencils need) so that every staged row starts
// on a 16-byte boundary of both the frame and shared memory.
template <int TH_, int TW_, int NT_>
struct Geo {
  static constexpr int TH = TH_, TW = TW_, NT = NT_;
  static constexpr int TWW = TW / 32;                      // mask words per tile row
  static constexpr int MWORDS = (TW + 12 + 31) / 32 + 1;   // mask words spanning the staged columns
  template <int H, int C = H>
  struct Reg {
    static constexpr int W = TW + 2 * C;
    static constexpr int Hh = TH + 2 * H;
    static constexpr int N = W * Hh;
    __host__ __device__ static constexpr int idx(int ly, int lx) { return (ly + H) * W + (lx + C); }
  };
  using XR6 = Reg<6, 8>;  // core: X0 and M_{k-1}
  using XR3 = Reg<3, 8>;  // finalize
  static_assert(TW % 32 == 0 && TH % 8 == 0 && NT % 32 == 0, "tile geometry");
  static_assert((TH & (TH - 1)) == 0 && (TW & (TW - 1)) == 0, "tile sides are powers of two (mark_tiles shifts)");
};
// The core variants' tile shapes.
using G32x64 = Geo<32, 64, 256>;
using G64x64 = Geo<64, 64, 512>;
using G32x128 = Geo<32, 128, 512>;
using G32x32 = Geo<32, 32, 160>;
// Finalize tiles, 256 threads: 32 x 128 for requests of many tiles (twice
// the pixels of a 32 x 64 tile per staging and per barrier: 18% less time
// on a 61-Mpx frame), 32 x 64 for small requests, which the larger tiles
// would leave with too few blocks.
using FGBig = Geo<32, 128, 256>;
using FGSmall = Geo<32, 64, 256>;

constexpr unsigned ERR_NONFINITE = 1u;
constexpr unsigned ERR_TIMEOUT = 2u;
constexpr unsigned ERR_NOGAIN = 4u;  // a level's gain estimate was undefined (it used gain 1)

// Gain estimation (C15): the full pair set and up to five clipping rounds
// per level, all taken from one histogram of the pair differences d.
constexpr int kGainRounds = 6;
constexpr int kGainBins = 2 * 65535 + 1;  // d = a - b of uint16 pairs: -65535 .. 65535
constexpr int kGainSmemHalf = 512;        // per-block shared bins for -512 <= d < 512

struct FrameState {
  unsigned long long fresh[LACOS_MAX_NITER + 1];  // nonzero when iteration k flagged new pixels
  unsigned long long flagged;                      // pixels in the final mask
  unsigned long long n_sprime, n_fine, n_replace;  // sparse-work counters (profiling)
  unsigned long long n_replace_wide;               // replacements whose 5x5 window was all flagged
  unsigned long long px_core;                      // tile pixels the core kernel computed (all levels)
  unsigned long long n_sprime_net, n_fine_net;     // S' and F evaluations by the full median networks
  unsigned int err;
  int iters_run;
  // Gain estimation (frames with gain 0), per level: the range of d present
  // in the level's histogram as max(65535 - d) and max(d + 65535) over the
  // pairs (0 and 0: no pair), the sums of the full pair set, the level whose
  // core launch recomputes every tile (the gain changed), and the latest
  // level's gain.
  unsigned int g_dneg, g_dpos;
  unsigned long long g0[4];  // the level's full pair set: n, sum d (two's complement), sum d^2, sum (a + b)
  int g_all_level;
  float gain;
};

struct FrameDesc {
  const void* x0;
  int dtype;  // 0 f32, 1 u16
  int ny, nx, wpr;  // wpr: 32-bit mask words per row
  uint32_t* mbuf0;  // M_k lives in buffer k & 1 (M_0 = zeros in buffer 0)
  uint32_t* mbuf1;
  uint32_t* p_sig;   // bit-planes of the current iteration (ny x wpr words each)
  uint32_t* p_lo;
  uint32_t* p_cand;
  float2* ntab;      // uint16 frames: {2N, RN(1/(2N))} for every integer med5 value 0..65535
  unsigned int* ghist_n;          // gain 0: pairs per d (index d + 65535), zero between levels
  unsigned long long* ghist_a;    // gain 0: sum of a + b per d
  uint8_t* tflags;   // per core tile: [2][tiles] "recompute at level k" (buffer k & 1), [tiles] sticky
  uint32_t* p_sat;   // satgrow > 0: the grown saturated set (C16) as 32-pixel words, built per request
  uint8_t* mask_out;
  float* clean_out;  // the working image I, and the cleaned output
  FrameState* st;
  float gain, rn2, satlevel, sigclip, lo, thr_min, objlim;
  float rn;          // read noise (the gain estimate squares it in double)
  int gain_est;      // 1: gain estimated at every level (C15, uint16 frames)
  int niter, fnorm;
  int satgrow;       // radius of the protected region around saturated pixels (0..4)
  int sepmed;        // 1: both 5x5 detection medians taken separably (comparison mode)
  int th, tw;        // core tile shape of the request's core-kernel variant
  int tiles_x;       // core tiles per row
  unsigned int tile_begin, tile_end;    // this frame's range in the flattened core-tile list
  int ftiles_x;                         // finalize tiles per row
  unsigned int fin_begin, fin_end;      // this frame's range in the flattened finalize-tile list
  unsigned long long word_begin;        // this frame's range in the flattened word list
  unsigned int gblk_begin, gblk_x;      // growth items: this frame's first, column groups per strip
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ float load_x0(const FrameDesc& f, int gy, int gx, bool& bad) {
  const size_t q = (size_t)gy * f.nx + gx;
  if (f.dtype == 1) return (float)__ldg((const unsigned short*)f.x0 + q);
  float v = __ldg((const float*)f.x0 + q);
  if (!isfinite(v)) { bad = true; v = 0.0f; }
  return v == 0.0f ? 0.0f : v;  // -0 -> +0
}

__device__ __forceinline__ uint32_t mask_bit(const uint32_t* M, int wpr, int gy, int gx) {
  return (__ldg(M + (size_t)gy * wpr + (gx >> 5)) >> (gx & 31)) & 1u;
}

// Float -> uint32 key with the same order as the float values (no NaN).
__device__ __forceinline__ uint32_t okey(float v) {
  const uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float from_okey(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Masked median with the window widened to (2*r0+1)^2 and beyond (rare: the
// smaller windows are fully flagged).  Reads X0 and the mask from global
// memory and selects the lower median by a 32-pass radix select on order
// keys.
__device__ float maskmed_wide(const FrameDesc& f, const uint32_t* M, int gy, int gx, int r0) {
  const int rmax = max(f.ny, f.nx) + 2;
  bool bad = false;
  for (int r = r0; r <= rmax; ++r) {
    unsigned n = 0;
    for (int dy = -r; dy <= r; ++dy) {
      const int y = clampi(gy + dy, 0, f.ny - 1);
      for (int dx = -r; dx <= r; ++dx) n += mask_bit(M, f.wpr, y, clampi(gx + dx, 0, f.nx - 1)) ^ 1u;
    }
    if (n == 0) continue;
    unsigned k = (n - 1) / 2;
    uint32_t prefix = 0;
    for (int b = 31; b >= 0; --b) {
      const uint32_t hi = (b == 31) ? 0u : (0xffffffffu << (b + 1));
      unsigned cnt = 0;
      for (int dy = -r; dy <= r; ++dy) {
        const int y = clampi(gy + dy, 0, f.ny - 1);
        for (int dx = -r; dx <= r; ++dx) {
          const int x = clampi(gx + dx, 0, f.nx - 1);
          if (mask_bit(M, f.wpr, y, x)) continue;
          const uint32_t key = okey(load_x0(f, y, x, bad));
          cnt += ((key & hi) == prefix) && !((key >> b) & 1u);
        }
      }
      if (k >= cnt) { k -= cnt; prefix |= (1u << b); }
    }
    return from_okey(prefix);
  }
  return load_x0(f, gy, gx, bad);  // unreachable: a frame always keeps an unflagged pixel
}

__device__ __forceinline__ int frame_of(const FrameDesc* fr, int nframes, unsigned item) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (fr[mid].tile_begin <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int frame_of_fin(const FrameDesc* fr, int nframes, unsigned item) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (fr[mid].fin_begin <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int frame_of_word(const FrameDesc* fr, int nframes, unsigned long long w) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (fr[mid].word_begin <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ bool iteration_runs(const FrameDesc& f, int k) {
  if (k > f.niter) return false;
  return k == 1 || *(volatile unsigned long long*)&f.st->fresh[k - 1] != 0;
}

// Core tiles of a frame.
__device__ __forceinline__ unsigned tiles_of(const FrameDesc& f) { return f.tile_end - f.tile_begin; }

// Iteration count actually executed (early stop included).
__device__ __forceinline__ int run_of(const FrameDesc& f) {
  for (int k = 1; k <= f.niter; ++k)
    if (f.st->fresh[k] == 0) return k;
  return f.niter;
}

// Selection keys of the working-image types: float values are their own
// keys (finite, -0 canonicalised) with -inf/+inf as sentinels; uint16 values
// become int keys with -1 and 65536 as sentinels.
template <class XT> struct KeyOf;
template <> struct KeyOf<float> {
  using K = float;
  static __device__ __forceinline__ K lo() { return lacos_net::neg_inf<float>(); }
  static __device__ __forceinline__ K hi() { return lacos_net::pos_inf<float>(); }
  static __device__ __forceinline__ K key(float x) { return x; }
  static __device__ __forceinline__ float back(K k) { return k; }
};
template <> struct KeyOf<uint16_t> {
  using K = int;
  static __device__ __forceinline__ K lo() { return -1; }
  static __device__ __forceinline__ K hi() { return 65536; }
  static __device__ __forceinline__ K key(uint16_t x) { return (int)x; }
  static __device__ __forceinline__ uint16_t back(K k) { return (uint16_t)k; }
};

// Masked 5x5 median at shared-memory index c of X (pitch P) with flags Mb:
// the lower median of the unflagged members.  With k members flagged and
// n = 25 - k unflagged, the rank-12 element of the 25 is the rank-(n-1)/2
// unflagged value when ceil(k/2) flagged members are taken as a low sentinel
// and the other floor(k/2) as a high one.  Which flagged members get which
// does not matter (the rank is a function of the multiset), so the i-th
// flagged member in row-major order takes the low sentinel for even i and
// the high one for odd i: bit j of `odd`, the parity of the flagged members
// before j, is an exclusive prefix XOR of the flag bits, with no running
// count.  Returns false when no member is unflagged.
template <class XT>
__device__ __forceinline__ bool maskmed5(const XT* X, const uint8_t* Mb, int P, int c, XT& out) {
  using KT = KeyOf<XT>;
  using K = typename KT::K;
  uint32_t b = 0;  // bit j: window member j (row-major) is flagged
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) b |= (uint32_t)(Mb[c + dy * P + dx] != 0) << ((dy + 2) * 5 + dx + 2);
  if (b == 0x1ffffffu) return false;
  uint32_t x = b;  // inclusive prefix XOR
  x ^= x << 1;
  x ^= x << 2;
  x ^= x << 4;
  x ^= x << 8;
  x ^= x << 16;
  const uint32_t odd = x << 1;  // exclusive
  K v[25];
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      const int j = (dy + 2) * 5 + dx + 2;
      const K s = ((odd >> j) & 1u) ? KT::hi() : KT::lo();
      v[j] = ((b >> j) & 1u) ? s : KT::key(X[c + dy * P + dx]);
    }
  K o;
  med5x5<K>(v, &o);
  out = KT::back(o);
  return true;
}

// Masked 7x7 median (the first widening): the same sentinel scheme with the
// rank-24 element of 49.  Returns false when no member is unflagged.
template <class XT>
__device__ __forceinline__ bool maskmed7(const XT* X, const uint8_t* Mb, int P, int c, XT& out) {
  using KT = KeyOf<XT>;
  using K = typename KT::K;
  int n = 0;
#pragma unroll
  for (int dy = -3; dy <= 3; ++dy)
#pragma unroll
    for (int dx = -3; dx <= 3; ++dx) n += Mb[c + dy * P + dx] ? 0 : 1;
  if (n == 0) return false;
  const int plo = 24 - (n - 1) / 2;
  K v[49];
  int seen = 0;
#pragma unroll
  for (int dy = -3; dy <= 3; ++dy)
#pragma unroll
    for (int dx = -3; dx <= 3; ++dx) {
      const int q = c + dy * P + dx;
      const bool fl = Mb[q] != 0;
      const K s = (seen < plo) ? KT::lo() : KT::hi();
      seen += fl ? 1 : 0;
      v[(dy + 3) * 7 + dx + 3] = fl ? s : KT::key(X[q]);
    }
  K o;
  med7x7<K>(v, &o);
  out = KT::back(o);
  return true;
}

// ---- core: steps 1-4 on a tile --------------------------------------------

// Stages X0 and the mask M (clamped coordinates) on region H of a tile:
// X (Reg<H>-indexed floats), Mb (bytes), via the mask words of the rows.
template <class G, int H, class XT>
__device__ __forceinline__ void stage_x0_mask(const FrameDesc& f, const uint32_t* M, int oy, int ox,
                                              XT* X, uint8_t* Mb, uint32_t (*Mw)[G::MWORDS],
                                              bool& bad) {
  constexpr int TH = G::TH, TW = G::TW, NT = G::NT, MWORDS = G::MWORDS;
  using R = typename G::template Reg<H, 8>;
  constexpr int C = 8;
  const int ny = f.ny, nx = f.nx;
  const int w0 = clampi(ox - C, 0, nx - 1) >> 5;
  // Columns ox-8 .. ox+TW+7 all inside the frame, rows 16-byte aligned:
  // 16-byte loads of 16 / sizeof(XT) pixels (rows are still clamped).
  constexpr int V = 16 / (int)sizeof(XT);  // pixels per 16-byte chunk
  constexpr int CPR = R::W / V;            // chunks per row
  static_assert(R::W % V == 0 && C % V == 0 && (32 % V) == 0, "chunking");
  const bool vec = ((reinterpret_cast<uintptr_t>(f.x0) & 15u) == 0) && (nx % V == 0) && ox - C >= 0 &&
                   ox + TW + C <= nx;
  // Interior tiles: the rows are copied asynchronously (16-byte cp.async),
  // in flight while the mask words load and their bits are spread.
  if (vec) {
    for (int i = threadIdx.x; i < (TH + 2 * H) * CPR; i += NT) {
      const int r = i / CPR, q = i % CPR;
      const int gy = clampi(oy - H + r, 0, ny - 1);
      const XT* src = static_cast<const XT*>(f.x0) + (size_t)gy * nx + (ox - C + q * V);
      const unsigned dst = (unsigned)__cvta_generic_to_shared(X + r * R::W + q * V);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int i = threadIdx.x; i < (TH + 2 * H) * MWORDS; i += NT) {
    const int r = i / MWORDS, w = w0 + i % MWORDS;
    const int gy = clampi(oy - H + r, 0, ny - 1);
    Mw[r][i % MWORDS] = w < f.wpr ? __ldg(M + (size_t)gy * f.wpr + w) : 0u;
  }
  __syncthreads();
  if (vec) {
    for (int i = threadIdx.x; i < (TH + 2 * H) * CPR; i += NT) {
      const int r = i / CPR, q = i % CPR;
      const int gx = ox - C + q * V;
      const uint32_t bits = Mw[r][(gx >> 5) - w0] >> (gx & 31);
      // V mask bits -> V bytes (bit t moves to bit 8t by the multiply; no carries)
      if constexpr (std::is_same<XT, float>::value)
        *reinterpret_cast<uint32_t*>(Mb + r * R::W + q * V) = ((bits & 0xfu) * 0x00204081u) & 0x01010101u;
      else
        *reinterpret_cast<uint2*>(Mb + r * R::W + q * V) = make_uint2(((bits & 0xfu) * 0x00204081u) & 0x01010101u,
                                                                 (((bits >> 4) & 0xfu) * 0x00204081u) & 0x01010101u);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // this thread's copies; the caller's barrier publishes them
    if constexpr (std::is_same<XT, float>::value) {
      // float input: canonicalise -0 and flag non-finite values in the chunks this thread copied
      for (int i = threadIdx.x; i < (TH + 2 * H) * CPR; i += NT) {
        float4* p = reinterpret_cast<float4*>(X + (i / CPR) * R::W + (i % CPR) * V);
        const float4 v = *p;
        float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (!isfinite(e[t])) { bad = true; e[t] = 0.0f; }
          e[t] = e[t] == 0.0f ? 0.0f : e[t];  // -0 -> +0
        }
        *p = make_float4(e[0], e[1], e[2], e[3]);
      }
    }
    return;
  }
#pragma unroll 4
  for (int i = threadIdx.x; i < R::N; i += NT) {
    const int ly = i / R::W - H, lx = i % R::W - C;
    const int gy = clampi(oy + ly, 0, ny - 1), gx = clampi(ox + lx, 0, nx - 1);
    if constexpr (std::is_same<XT, float>::value)
      X[i] = load_x0(f, gy, gx, bad);
    else
      X[i] = __ldg((const unsigned short*)f.x0 + (size_t)gy * nx + gx);
    Mb[i] = (uint8_t)((Mw[ly + H][(gx >> 5) - w0] >> (gx & 31)) & 1u);
  }
}

__device__ __forceinline__ float noise_of_g(float gain, float rn2, float m5) {
  const float gm = __fmul_rn(gain, m5);
  const float e = gm < 1e-4f ? 1e-4f : gm;
  return __fdiv_rn(__fsqrt_rn(__fadd_rn(e, rn2)), gain);
}

__device__ __forceinline__ float noise_of(const FrameDesc& f, float m5) { return noise_of_g(f.gain, f.rn2, m5); }

// {D, y} = {2N, RN(1/D)} for an integer med5 value m (N with the same
// arithmetic as noise_of; doubling is exact).
__device__ __forceinline__ float2 ntab_entry_g(float gain, float rn2, int m) {
  const float N = noise_of_g(gain, rn2, (float)m);
  const float D = __fadd_rn(N, N);
  return make_float2(D, __fdiv_rn(1.0f, D));
}

__device__ __forceinline__ float2 ntab_entry(const FrameDesc& f, int m) { return ntab_entry_g(f.gain, f.rn2, m); }

// The table of a uint16 frame, once per request instead of once per pixel
// (per level, by ntab_level_kernel, when the gain is estimated).
__global__ void ntab_kernel(const FrameDesc* __restrict__ fr, int nframes) {
  const int fi = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (fi >= nframes || m > 65535) return;
  const FrameDesc& f = fr[fi];
  if (f.dtype == 1 && !f.gain_est) f.ntab[m] = ntab_entry(f, m);
}

// ---- gain estimation (C15), per level, for frames with gain 0 --------------
//
// One pass over the level's image builds a histogram of the pair differences:
// for every pair (columns 2m, 2m+1) whose pixels are both unflagged in
// M_(k-1) and unsaturated -- so both hold input values -- the count of pairs
// and the sum of a + b per value of d = a - b.  Every clipping round then
// runs on the histogram (gain_fold_kernel): the sums n, sum d, sum d^2 and
// sum (a + b) over the pairs with d in the round's interval are the same
// integers as over the pairs themselves, so the estimate is exact.  Each
// block counts the common small differences in shared memory and adds them
// to the frame's histogram once; larger ones go to it directly.
__global__ void __launch_bounds__(kBlock, 4) gain_hist_kernel(const FrameDesc* __restrict__ fr, int nframes, int k) {
  const int fi = blockIdx.y;
  if (fi >= nframes) return;
  const FrameDesc& f = fr[fi];
  FrameState* st = f.st;
  if (!f.gain_est || !iteration_runs(f, k)) return;
  // Shared bins: the count, and the sum of a + b as two 32-bit halves (a
  // carry out of the low half is added to the high half by the thread whose
  // addition wrapped, so the pair of words holds the exact 64-bit sum).
  __shared__ unsigned int hn[2 * kGainSmemHalf], hlo[2 * kGainSmemHalf], hhi[2 * kGainSmemHalf];
  __shared__ unsigned long long red[kBlock / 32][4];
  for (int i = threadIdx.x; i < 2 * kGainSmemHalf; i += kBlock) {
    hn[i] = 0u;
    hlo[i] = 0u;
    hhi[i] = 0u;
  }
  __syncthreads();
  const uint32_t* Mprev = ((k - 1) & 1) ? f.mbuf1 : f.mbuf0;  // M_(k-1)
  const bool satchk = f.p_sat == nullptr && f.satlevel > 0.0f;
  // Rows start on 16-byte boundaries and hold whole 8-pixel chunks: each
  // word's 32 pixels are four 16-byte loads.
  const bool vec = (reinterpret_cast<uintptr_t>(f.x0) & 15u) == 0 && f.nx % 8 == 0;
  const unsigned nwords = (unsigned)f.ny * (unsigned)f.wpr;
  const uint16_t* x0 = static_cast<const uint16_t*>(f.x0);
  unsigned dneg = 0, dpos = 0;  // max(65535 - d), max(d + 65535) over this thread's pairs
  unsigned long long n0 = 0, s20 = 0, a0 = 0;  // the full set's sums (clipping round 0)
  long long s10 = 0;
  for (unsigned w = blockIdx.x * kBlock + threadIdx.x; w < nwords; w += gridDim.x * kBlock) {
    const int y = (int)(w / (unsigned)f.wpr), xw = (int)(w % (unsigned)f.wpr) * 32;
    const int cnt = min(32, f.nx - xw);  // pixels of this word
    uint32_t bad = __ldg(Mprev + w);
    if (f.p_sat) bad |= __ldg(f.p_sat + w);
    const uint16_t* row = x0 + (size_t)y * f.nx + xw;
    uint32_t v[16];  // pair m: column xw+2m in the low half, xw+2m+1 in the high half
    if (vec) {
      const uint4* src = reinterpret_cast<const uint4*>(row);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (c < cnt / 8) {
          const uint4 u = __ldg(src + c);
          v[4 * c] = u.x;
          v[4 * c + 1] = u.y;
          v[4 * c + 2] = u.z;
          v[4 * c + 3] = u.w;
        } else {
          v[4 * c] = v[4 * c + 1] = v[4 * c + 2] = v[4 * c + 3] = 0u;
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < 16; ++m)
        v[m] = 2 * m + 1 < cnt ? (uint32_t)__ldg(row + 2 * m) | ((uint32_t)__ldg(row + 2 * m + 1) << 16) : 0u;
    }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      if (2 * m + 1 >= cnt || ((bad >> (2 * m)) & 3u)) continue;
      const int va = (int)(v[m] & 0xffffu), vb = (int)(v[m] >> 16);
      if (satchk && ((float)va >= f.satlevel || (float)vb >= f.satlevel)) continue;
      const int d = va - vb;
      dneg = max(dneg, (unsigned)(65535 - d));
      dpos = max(dpos, (unsigned)(d + 65535));
      n0 += 1;
      s10 += d;
      s20 += (unsigned long long)((long long)d * d);
      a0 += (unsigned long long)(va + vb);
      if (d >= -kGainSmemHalf && d < kGainSmemHalf) {
        const int i = d + kGainSmemHalf;
        const unsigned ab = (unsigned)(va + vb);
        atomicAdd(&hn[i], 1u);
        if (atomicAdd(&hlo[i], ab) > 0xffffffffu - ab) atomicAdd(&hhi[i], 1u);
      } else {
        atomicAdd(&f.ghist_n[d + 65535], 1u);
        atomicAdd(&f.ghist_a[d + 65535], (unsigned long long)(va + vb));
      }
    }
  }
  dneg = __reduce_max_sync(0xffffffffu, dneg);
  dpos = __reduce_max_sync(0xffffffffu, dpos);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n0 += __shfl_down_sync(0xffffffffu, n0, o);
    s10 += __shfl_down_sync(0xffffffffu, s10, o);
    s20 += __shfl_down_sync(0xffffffffu, s20, o);
    a0 += __shfl_down_sync(0xffffffffu, a0, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (dneg) atomicMax(&st->g_dneg, dneg);
    if (dpos) atomicMax(&st->g_dpos, dpos);
    red[threadIdx.x >> 5][0] = n0;
    red[threadIdx.x >> 5][1] = (unsigned long long)s10;
    red[threadIdx.x >> 5][2] = s20;
    red[threadIdx.x >> 5][3] = a0;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    unsigned long long t = 0;
    for (int q = 0; q < kBlock / 32; ++q) t += red[q][threadIdx.x];
    if (t) atomicAdd(&st->g0[threadIdx.x], t);
  }
  for (int i = threadIdx.x; i < 2 * kGainSmemHalf; i += kBlock) {
    if (!hn[i]) continue;
    atomicAdd(&f.ghist_n[i - kGainSmemHalf + 65535], hn[i]);
    atomicAdd(&f.ghist_a[i - kGainSmemHalf + 65535], ((unsigned long long)hhi[i] << 32) | hlo[i]);
  }
}

// The clipping rounds of level k on the frame's histogram, one block per
// frame: round r sums the bins with d in the clip interval (every d at
// r = 0); when the clipping has converged (the round kept as many pairs as
// the one before, or this is the fifth clipping round) the round's sums give
// the level's gain, otherwise the next interval is the current one
// intersected with 3 population standard deviations of the round's set.
// The block then clears the bins it read for the next level.
constexpr int kFoldThreads = 1024;
__global__ void __launch_bounds__(kFoldThreads) gain_fold_kernel(const FrameDesc* __restrict__ fr, int nframes, int k) {
  const int fi = blockIdx.x;
  if (fi >= nframes) return;
  const FrameDesc& f = fr[fi];
  FrameState* st = f.st;
  if (!f.gain_est || !iteration_runs(f, k)) return;
  const int dlo = 65535 - (int)__ldcg(&st->g_dneg), dhi = (int)__ldcg(&st->g_dpos) - 65535;  // d range present
  __shared__ unsigned long long red[kFoldThreads / 32][4];
  __shared__ long long s_lo, s_hi;
  __shared__ int s_done;
  __shared__ unsigned long long s_prev_n;
  if (threadIdx.x == 0) {
    s_lo = -65536;
    s_hi = 65536;
    s_done = 0;
    s_prev_n = 0;
  }
  __syncthreads();
  for (int r = 0; r < kGainRounds; ++r) {
    // Round 0 takes every pair: its sums came with the histogram.
    const long long lo = r == 0 ? 1 : max(s_lo, (long long)dlo), hi = r == 0 ? 0 : min(s_hi, (long long)dhi);
    unsigned long long n = 0, s2 = 0, a = 0;
    long long s1 = 0;
    if (r == 0 && threadIdx.x < 4) {
      const unsigned long long t = __ldcg(&st->g0[threadIdx.x]);
      if (threadIdx.x == 0) n = t;
      if (threadIdx.x == 1) s1 = (long long)t;
      if (threadIdx.x == 2) s2 = t;
      if (threadIdx.x == 3) a = t;
    }
    for (long long d = lo + threadIdx.x; d <= hi; d += kFoldThreads) {
      const unsigned long long c = __ldcg(&f.ghist_n[d + 65535]);
      if (!c) continue;
      n += c;
      s1 += d * (long long)c;
      s2 += (unsigned long long)(d * d) * c;
      a += __ldcg(&f.ghist_a[d + 65535]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n += __shfl_down_sync(0xffffffffu, n, o);
      s1 += __shfl_down_sync(0xffffffffu, s1, o);
      s2 += __shfl_down_sync(0xffffffffu, s2, o);
      a += __shfl_down_sync(0xffffffffu, a, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5][0] = n;
      red[threadIdx.x >> 5][1] = (unsigned long long)s1;
      red[threadIdx.x >> 5][2] = s2;
      red[threadIdx.x >> 5][3] = a;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t[4] = {0ull, 0ull, 0ull, 0ull};
      for (int q = 0; q < kFoldThreads / 32; ++q)
        for (int i = 0; i < 4; ++i) t[i] += red[q][i];
      const unsigned long long n_r = t[0], s2_r = t[2], a_r = t[3];
      const long long s1_r = (long long)t[1];
      const bool done = n_r == 0 || r == kGainRounds - 1 || (r > 0 && n_r == s_prev_n);
      if (done) {
        double g = 0.0;
        float gf = 1.0f;
        if (lacos_gain::gm_gain(n_r, s1_r, s2_r, a_r, f.rn, &g))
          gf = __double2float_rn(g);
        else
          atomicOr(&st->err, ERR_NOGAIN);
        if (k == 1 || __float_as_uint(gf) != __float_as_uint(st->gain)) st->g_all_level = k;
        st->gain = gf;
        s_done = 1;
      } else {
        long long l, h;
        lacos_gain::gm_clip_interval(n_r, s1_r, s2_r, &l, &h);
        s_lo = l > s_lo ? l : s_lo;
        s_hi = h < s_hi ? h : s_hi;
        s_prev_n = n_r;
      }
    }
    __syncthreads();
    if (s_done) break;
  }
  // The next level starts from an empty histogram.
  for (int d = dlo + (int)threadIdx.x; d <= dhi; d += kFoldThreads) {
    f.ghist_n[d + 65535] = 0u;
    f.ghist_a[d + 65535] = 0ull;
  }
  if (threadIdx.x < 4) st->g0[threadIdx.x] = 0ull;
  if (threadIdx.x == 0) {
    st->g_dneg = 0u;
    st->g_dpos = 0u;
  }
}

// At each level where a frame's estimated gain differs from the previous
// level's (and at the first): its N table for the new gain, and every core
// tile marked for recomputation at this level (N changes everywhere).
// Grid: 256 x frames blocks of 256 threads, one table entry per thread,
// tiles in a grid-stride loop.
__global__ void ntab_level_kernel(const FrameDesc* __restrict__ fr, int nframes, int k) {
  const int fi = blockIdx.y;
  if (fi >= nframes) return;
  const FrameDesc& f = fr[fi];
  if (!f.gain_est || !iteration_runs(f, k) || __ldcg(&f.st->g_all_level) != k) return;
  const unsigned m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m <= 65535u) f.ntab[m] = ntab_entry_g(__ldcg(&f.st->gain), f.rn2, (int)m);
  if (k == 1) return;  // level 1 computes every tile anyway
  uint8_t* marks = f.tflags + (size_t)(k & 1) * tiles_of(f);
  for (unsigned t = m; t < tiles_of(f); t += gridDim.x * blockDim.x) marks[t] = 1;
}

// Saturated-star protection (C16), once per request: the seeds (input >=
// satlevel; a saturated pixel is never flagged, so the set does not depend
// on the mask) as 32-pixel words, staged in the level-1 mask buffer, which
// nothing reads before the first growth pass writes it ...
__global__ void satseed_kernel(const FrameDesc* __restrict__ fr, int fi, unsigned nwords) {
  const FrameDesc& f = fr[fi];
  const unsigned q0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool on = f.satlevel > 0.0f;
  const int V = f.dtype == 1 ? 8 : 4;  // pixels per 16-byte load
  if ((reinterpret_cast<uintptr_t>(f.x0) & 15u) == 0 && f.nx % V == 0) {
    // Every row starts on a 16-byte boundary and holds whole 16-byte chunks:
    // one thread per word, 16-byte loads of its chunks (a row's last word may
    // hold fewer than 32 pixels).
    if (q0 >= nwords) return;
    const int y = (int)(q0 / (unsigned)f.wpr), x0 = (int)(q0 % (unsigned)f.wpr) * 32;
    const int nch = min(32, f.nx - x0) / V;
    const size_t p0 = (size_t)y * f.nx + x0;
    uint32_t bits = 0;
    if (on) {
      if (f.dtype == 1) {
        const uint4* src = reinterpret_cast<const uint4*>(static_cast<const uint16_t*>(f.x0) + p0);
        for (int c = 0; c < nch; ++c) {
          const uint4 u = __ldg(src + c);
          const uint32_t h[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
          for (int e = 0; e < 8; ++e)
            bits |= ((float)((h[e >> 1] >> (16 * (e & 1))) & 0xffffu) >= f.satlevel ? 1u : 0u) << (8 * c + e);
        }
      } else {
        const float4* src = reinterpret_cast<const float4*>(static_cast<const float*>(f.x0) + p0);
        for (int c = 0; c < nch; ++c) {
          const float4 u = __ldg(src + c);
          const float e4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) bits |= (e4[e] >= f.satlevel ? 1u : 0u) << (4 * c + e);
        }
      }
    }
    f.mbuf1[q0] = bits;
    return;
  }
  // General layout: a warp forms 32 consecutive words, one per step (lane l
  // tests pixel l of the word; the ballot is the word; lane j keeps word j).
  const unsigned base = q0 & ~31u;
  const int lane = threadIdx.x & 31;
  uint32_t mine = 0;
  float v[32];  // all 32 loads in flight before the ballots
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const unsigned q = base + j;
    v[j] = -1.0f;
    if (q < nwords) {
      const int y = (int)(q / (unsigned)f.wpr), x = (int)(q % (unsigned)f.wpr) * 32 + lane;
      if (x < f.nx) {
        const size_t p = (size_t)y * f.nx + x;
        v[j] = f.dtype == 1 ? (float)__ldg((const unsigned short*)f.x0 + p) : __ldg((const float*)f.x0 + p);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < 32; ++j) {
    const uint32_t word = __ballot_sync(0xffffffffu, on && v[j] >= f.satlevel);
    if (lane == j) mine = word;
  }
  if (base + lane < nwords) f.mbuf1[base + lane] = mine;
}

// ... then grown by the square of radius satgrow: per word, the OR over rows
// -r..r of each row's OR over columns -r..r (funnel shifts with the
// neighbouring words; bits beyond the frame are never set).
__global__ void satgrow_kernel(const FrameDesc* __restrict__ fr, int fi, unsigned nwords) {
  const FrameDesc& f = fr[fi];
  const unsigned q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nwords) return;
  const int y = (int)(q / (unsigned)f.wpr), w = (int)(q % (unsigned)f.wpr), r = f.satgrow;
  uint32_t g = 0;
#pragma unroll
  for (int a = -4; a <= 4; ++a) {  // rows -r..r (r <= 4), all loads in flight
    const int yy = y + a;
    if (a < -r || a > r || yy < 0 || yy >= f.ny) continue;
    const uint32_t* row = f.mbuf1 + (size_t)yy * f.wpr;
    const uint32_t c = row[w], lft = w > 0 ? row[w - 1] : 0u, rgt = w + 1 < f.wpr ? row[w + 1] : 0u;
    uint32_t h = c;
    for (int d = 1; d <= r; ++d) h |= __funnelshift_r(c, rgt, d) | __funnelshift_l(lft, c, d);
    g |= h;
  }
  f.p_sat[q] = g;
}

// L / D rounded to nearest, for D > 0, L >= 0 and y = RN(1/D), without a
// divide: Markstein's correction (P. Markstein, "Computation of elementary
// functions on the IBM RISC System/6000 processor", IBM J. Res. Dev. 34(1),
// 1990).  q0 = RN(L y) can be off by more than an ulp; one correction
// q1 = RN(q0 + r0 y), with r0 = L - D q0 from one fused multiply-add, makes
// it faithful; then the remainder r1 = L - D q1 is exact and, y being
// within half an ulp of 1/D, q1 + r1 y rounds to the correctly rounded
// quotient.  The identity with IEEE division is checked exhaustively over
// every L a uint16 frame's L+ can take (multiples of 1/4 up to 131070) and
// every table entry by lacos_selftest_division.
__device__ __forceinline__ float div_recip(float L, float D, float y) {
  const float q0 = __fmul_rn(L, y);
  const float r0 = __fmaf_rn(-q0, D, L);
  const float q1 = __fmaf_rn(r0, y, q0);
  const float r1 = __fmaf_rn(-q1, D, L);
  return __fmaf_rn(r1, y, q1);
}

// Exhaustive check of div_recip against IEEE division: table entry m per
// block, every L = k/4 with k = 0..524280 (the range of a uint16 frame's L+:
// each of its four clipped terms is at most 2 * 65535) per thread stride.
__global__ void selftest_division_kernel(FrameDesc f, unsigned long long* mismatches) {
  const float2 t = ntab_entry(f, (int)blockIdx.x);
  unsigned cnt = 0;
  for (int k = threadIdx.x; k <= 4 * 131070; k += blockDim.x) {
    const float L = __fmul_rn((float)k, 0.25f);
    cnt += __float_as_uint(div_recip(L, t.x, t.y)) != __float_as_uint(__fdiv_rn(L, t.x)) ? 1u : 0u;
  }
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(mismatches, (unsigned long long)cnt);
}

__device__ __forceinline__ float lplus(float vc, float up, float dn, float lf, float rt) {
  const float vv = __fadd_rn(vc, vc);
  float c1 = __fsub_rn(__fsub_rn(vv, up), lf);
  float c2 = __fsub_rn(__fsub_rn(vv, up), rt);
  float c3 = __fsub_rn(__fsub_rn(vv, dn), lf);
  float c4 = __fsub_rn(__fsub_rn(vv, dn), rt);
  c1 = c1 > 0.0f ? c1 : 0.0f;
  c2 = c2 > 0.0f ? c2 : 0.0f;
  c3 = c3 > 0.0f ? c3 : 0.0f;
  c4 = c4 > 0.0f ? c4 : 0.0f;
  return __fmul_rn(__fadd_rn(__fadd_rn(c1, c2), __fadd_rn(c3, c4)), 0.25f);
}

// Shared memory of one core tile, by working-image type.
template <class G, class XT> struct CoreSmemT;
template <class G> struct CoreSmemT<G, float> {
  using XR6 = typename G::XR6;
  float X[XR6::N];                       // X0 on R6, then the working image I_{k-1} on R4
  uint8_t Mb[XR6::N];                    // M_{k-1} on R6
  uint32_t Mw[G::TH + 12][G::MWORDS];    // M_{k-1} words of the R6 rows (clamped rows)
  float S[G::template Reg<2>::N];        // S on R2
  float N[G::TH * G::TW];                // N on the tile
  float M3[G::template Reg<3>::N];       // med3(I) on R3
  uint16_t list[G::template Reg<4>::N];  // work lists: replacement on R4; then fine-structure
                                         // items from the front and S'-only items from the back
  uint8_t flags[G::TH * G::TW];          // bit3: saturated
  uint32_t pw[3][G::TH][G::TWW];         // the tile's sig, lo and candidate bit-plane words
  uint32_t Sw[G::TH][G::TWW];            // satgrow > 0: the tile's words of the grown saturated set
  unsigned nlist, nlist2;                // list lengths (S'-only, fine-structure)
  unsigned nfine, nfine_net;             // F evaluations of the tile; of them by the med7 network
};
template <class G> struct CoreSmemT<G, uint16_t> {
  using XR6 = typename G::XR6;
  uint16_t X[XR6::N];                    // X0 on R6, then I_{k-1} on R4 (uint16 frames stay integral)
  uint8_t Mb[XR6::N];
  uint32_t Mw[G::TH + 12][G::MWORDS];
  float S[G::template Reg<2>::N];
  float2 DY[G::template Reg<2>::N];      // {2N, 1/(2N)} on R2 (the table at med5(I))
  uint16_t M3[G::template Reg<3>::N];
  uint16_t list[G::template Reg<4>::N];
  uint8_t flags[G::TH * G::TW];
  uint32_t pw[3][G::TH][G::TWW];
  uint32_t Sw[G::TH][G::TWW];
  unsigned nlist, nlist2;
  unsigned nfine, nfine_net;
};
// Alignment of the vector accesses: 16-byte staging rows (X; Mb in 8-byte
// groups), 4-pixel block-network loads, 2-pixel pairs of S, N, DY and flags;
// both sparse lists of a tile fit in one list array, and list entries (tile
// and region indices) fit in 16 bits.
template <class G>
constexpr bool core_layout_ok() {
  using F = CoreSmemT<G, float>;
  using U = CoreSmemT<G, uint16_t>;
  return offsetof(F, X) % 16 == 0 && offsetof(F, Mb) % 8 == 0 && offsetof(F, S) % 8 == 0 &&
         offsetof(F, flags) % 8 == 0 && offsetof(U, X) % 16 == 0 && offsetof(U, Mb) % 8 == 0 &&
         offsetof(U, S) % 8 == 0 && offsetof(U, flags) % 8 == 0 && offsetof(F, N) % 8 == 0 &&
         offsetof(U, DY) % 16 == 0 && G::TH * G::TW <= G::template Reg<4>::N && G::XR6::N <= 65536;
}
static_assert(core_layout_ok<G32x64>() && core_layout_ok<G64x64>() && core_layout_ok<G32x128>() &&
                  core_layout_ok<G32x32>(),
              "core layout");
// Dynamic shared memory of a core launch, by geometry and working-image type.
template <class G, class XT>
constexpr size_t kCoreSmemBytes = sizeof(CoreSmemT<G, XT>);

__device__ __forceinline__ U16x2 pack2(uint16_t lo, uint16_t hi) {
  return U16x2{(uint32_t)lo | ((uint32_t)hi << 16)};
}
__device__ __forceinline__ int half_of(U16x2 p, int h) { return h ? (int)(p.v >> 16) : (int)(p.v & 0xffffu); }

// L+ of integer-valued pixels: every intermediate of the float definition is
// an integer below 2^24, so this integer form gives the same float.
__device__ __forceinline__ float lplus_int(int vc, int up, int dn, int lf, int rt) {
  const int vv = vc + vc;
  const int c1 = max(vv - up - lf, 0), c2 = max(vv - up - rt, 0);
  const int c3 = max(vv - dn - lf, 0), c4 = max(vv - dn - rt, 0);
  return __fmul_rn((float)((c1 + c2) + (c3 + c4)), 0.25f);
}

// Block-network inputs from the staged image, 4 aligned pixels per shared
// load (the network asks for each input once; loads of the same group are
// merged).  Window column 0 must sit on a 4-pixel boundary of the row.
template <int P, int W>
struct QuadLoaderF32 {
  const float* base;  // window element (0, 0); rows W apart
  __device__ __forceinline__ float operator()(int i) const {
    const int a = i / P, b = i % P;
    const float4 q = *reinterpret_cast<const float4*>(base + a * W + (b & ~3));
    return (b & 3) == 0 ? q.x : (b & 3) == 1 ? q.y : (b & 3) == 2 ? q.z : q.w;
  }
};
// Packed pairs for uint16 frames: low half from the window row, high half
// from the row DY further down.
template <int P, int DY, int W>
struct QuadLoaderU16 {
  const uint16_t* base;  // rows W apart
  __device__ __forceinline__ U16x2 operator()(int i) const {
    const int a = i / P, b = i % P;
    const uint16_t* p = base + a * W + (b & ~3);
    const uint2 lo = *reinterpret_cast<const uint2*>(p);
    const uint2 hi = *reinterpret_cast<const uint2*>(p + DY * W);
    const uint32_t l = (b & 2) ? lo.y : lo.x, h = (b & 2) ? hi.y : hi.x;
    return U16x2{__byte_perm(l, h, (b & 1) ? 0x7632 : 0x5410)};
  }
};

// Assignment of the dense step's block units to (round, thread): the med5
// units first, the med3 units after them starting at a warp boundary, so
// that no warp runs both kinds (a warp with both would execute the two
// networks one after the other).
template <int NT, int S_UNITS, int M_UNITS>
struct UnitMap {
  static constexpr int RS = (S_UNITS + NT - 1) / NT;     // rounds with med5 units
  static constexpr int REM = S_UNITS - (RS - 1) * NT;    // med5 units in the last of them
  static constexpr int MF = (REM + 31) / 32 * 32;        // its first med3 thread
  static constexpr int M0 = NT - MF;                     // med3 units that round can take
  static constexpr int ROUNDS = RS + (M_UNITS > M0 ? (M_UNITS - M0 + NT - 1) / NT : 0);
  // Unit of thread t in round r (< S_UNITS: med5, else med3), or -1.
  __device__ static __forceinline__ int unit(int r, int t) {
    if (r < RS - 1) return r * NT + t;
    if (r == RS - 1) {
      if (t < REM) return r * NT + t;
      return (t >= MF && t - MF < M_UNITS) ? S_UNITS + (t - MF) : -1;
    }
    const int m = M0 + (r - RS) * NT + t;
    return m < M_UNITS ? S_UNITS + m : -1;
  }
};

// Saturation flags of the tile (the original input at an unflagged pixel),
// four pixels per item, by the threads from FIRST on (for uint16 frames the
// block threads without a med5 block, which would otherwise wait at the next
// barrier).
template <class G, class XT, int FIRST, class SM>
__device__ __forceinline__ void sat_flags(const FrameDesc& f, SM& sm) {
  constexpr int TH = G::TH, TW = G::TW, NT = G::NT;
  using XR6 = typename G::XR6;
  static_assert(FIRST >= 0 && FIRST < NT, "some threads must take the flags");
  constexpr int first = FIRST;
  const int tid = (int)threadIdx.x;
  if (f.satgrow) {  // the grown set (C16), built once per request: expand the tile's words
    for (int q = tid - first; q < TH * TW / 8; q += NT - first) {
      const int ly = q / (TW / 8), g = q % (TW / 8);
      const uint32_t bits = (sm.Sw[ly][g >> 2] >> (8 * (g & 3))) & 0xffu;
      // bit t -> byte t, value 8 (bit t moves to bit 8t by the multiply; no carries)
      uint2 out;
      out.x = (((bits & 0xfu) * 0x00204081u) & 0x01010101u) << 3;
      out.y = ((((bits >> 4) & 0xfu) * 0x00204081u) & 0x01010101u) << 3;
      *reinterpret_cast<uint2*>(sm.flags + ly * TW + 8 * g) = out;
    }
    return;
  }
  if (tid < first) return;
  const bool chk = f.satlevel > 0.0f;
  for (int q = tid - first; q < TH * TW / 4; q += NT - first) {
    const int ly = q / (TW / 4), lx = (q % (TW / 4)) * 4;
    const int c = XR6::idx(ly, lx);
    float v[4];
    if constexpr (std::is_same<XT, float>::value) {
      const float4 x = *reinterpret_cast<const float4*>(sm.X + c);
      v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else {
      const uint2 x = *reinterpret_cast<const uint2*>(sm.X + c);
      v[0] = (float)(x.x & 0xffffu); v[1] = (float)(x.x >> 16);
      v[2] = (float)(x.y & 0xffffu); v[3] = (float)(x.y >> 16);
    }
    const uint32_t mb = *reinterpret_cast<const uint32_t*>(sm.Mb + c);
    uint32_t fl = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if (chk && !((mb >> (8 * e)) & 0xffu) && v[e] >= f.satlevel) fl |= 8u << (8 * e);
    *reinterpret_cast<uint32_t*>(sm.flags + ly * TW + lx) = fl;
  }
}

// Dense networks for float32 frames: med5 on R2 by 4x2 blocks (parked in
// S), med3 on R3 by 8x2 blocks.  Blocks also evaluate out-of-frame
// positions (from clamped inputs); those are overwritten by the edge fill.
template <class G>
__device__ __forceinline__ void dense_f32(const FrameDesc& f, CoreSmemT<G, float>& sm) {
  constexpr int TH = G::TH, TW = G::TW, NT = G::NT;
  using XR6 = typename G::XR6;
  using R2 = typename G::template Reg<2>;
  using R3 = typename G::template Reg<3>;
  constexpr int S_BW = 4, S_BH = 2, S_UX = (TW + 4) / S_BW, S_UY = (TH + 4) / S_BH;
  constexpr int M_BW = 8, M_BH = 2, M_UX = (TW + 6 + M_BW - 1) / M_BW, M_UY = (TH + 6) / M_BH;
  constexpr int S_UNITS = S_UX * S_UY;
  using UM = UnitMap<NT, S_UNITS, M_UX * M_UY>;
  static_assert((TW + 4) % S_BW == 0 && (TH + 4) % S_BH == 0 && (TH + 6) % M_BH == 0, "block tiling");
  // Window columns start at lx0 - 2 = 4u - 4 (med5) and lx0 - 1 = 8m - 4
  // (med3): 4-pixel aligned in the 8-column-halo staging rows; the med3
  // window's last 4-group reads at most 2 pixels past it, still in the row.
  static_assert(XR6::W % 4 == 0 && XR6::idx(0, -4) % 4 == 0 && (-3 + 8 * (M_UX - 1)) - 1 + 12 <= TW + 8,
                "aligned block windows");
  for (int rd = 0; rd < UM::ROUNDS; ++rd) {
    const int u = UM::unit(rd, threadIdx.x);
    if (u < 0) continue;
    if (u < S_UNITS) {
      const int ly0 = -2 + (u / S_UX) * S_BH, lx0 = -2 + (u % S_UX) * S_BW;
      constexpr int P = S_BW + 4;
      const QuadLoaderF32<P, XR6::W> ld{sm.X + XR6::idx(ly0 - 2, lx0 - 2)};
      float m5[S_BH * S_BW];
      if (f.sepmed)
        blk_sep5_4x2_ld<float>(ld, m5);
      else
        blk_med5_4x2_ld<float>(ld, m5);
      // med5 parked in S; dense_pixels turns it into N and S.
#pragma unroll
      for (int r = 0; r < S_BH; ++r)
#pragma unroll
        for (int cc = 0; cc < S_BW; ++cc) sm.S[R2::idx(ly0 + r, lx0 + cc)] = m5[r * S_BW + cc];
    } else {
      const int m = u - S_UNITS;
      const int ly0 = -3 + (m / M_UX) * M_BH, lx0 = -3 + (m % M_UX) * M_BW;
      constexpr int P = M_BW + 2;
      const QuadLoaderF32<P, XR6::W> ld{sm.X + XR6::idx(ly0 - 1, lx0 - 1)};
      float m3[M_BH * M_BW];
      blk_med3_8x2_ld<float>(ld, m3);
#pragma unroll
      for (int r = 0; r < M_BH; ++r)
#pragma unroll
        for (int cc = 0; cc < M_BW; ++cc)
          if (lx0 + cc < TW + 3) sm.M3[R3::idx(ly0 + r, lx0 + cc)] = m3[r * M_BW + cc];
    }
  }
  sat_flags<G, float, 0>(f, sm);  // units outnumber threads here: all threads share the flags
}

// Dense part for uint16 frames: the same blocks on packed uint16 pairs, two
// blocks per register -- a block in the upper half of the region with the
// block the same distance further down -- so each min/max instruction
// serves two outputs.  Each med5 indexes the N table right away (the
// block's 16 loads are in flight together); {2N, 1/(2N)} goes to DY.
template <class G>
__device__ __forceinline__ void dense_u16(const FrameDesc& f, CoreSmemT<G, uint16_t>& sm) {
  constexpr int TH = G::TH, TW = G::TW, NT = G::NT;
  using XR6 = typename G::XR6;
  using R2 = typename G::template Reg<2>;
  using R3 = typename G::template Reg<3>;
  constexpr int S_BW = 4, S_BH = 2, S_UX = (TW + 4) / S_BW, S_PAIRS = (TH + 4) / S_BH / 2;
  constexpr int S_DY = S_PAIRS * S_BH;  // row offset of the second block of a pair
  constexpr int M_BW = 8, M_BH = 2, M_UX = (TW + 6 + M_BW - 1) / M_BW;
  constexpr int M_PAIRS = ((TH + 6) / M_BH + 1) / 2, M_DY = M_PAIRS * M_BH;
  constexpr int S_UNITS = S_UX * S_PAIRS;
  using UM = UnitMap<NT, S_UNITS, M_UX * M_PAIRS>;
  static_assert(((TH + 4) / S_BH) % 2 == 0, "S row-pairs pair up");
  static_assert(UM::ROUNDS == 1, "one unit per thread");
  for (int rd = 0; rd < UM::ROUNDS; ++rd) {
    const int u = UM::unit(rd, threadIdx.x);
    if (u < 0) continue;
    if (u < S_UNITS) {
      const int ly0 = -2 + (u / S_UX) * S_BH, lx0 = -2 + (u % S_UX) * S_BW;
      constexpr int P = S_BW + 4;
      const QuadLoaderU16<P, S_DY, XR6::W> ld{sm.X + XR6::idx(ly0 - 2, lx0 - 2)};
      U16x2 m5[S_BH * S_BW];
      if (f.sepmed)
        blk_sep5_4x2_ld<U16x2>(ld, m5);
      else
        blk_med5_4x2_ld<U16x2>(ld, m5);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < S_BH; ++r)
#pragma unroll
          for (int cc = 0; cc < S_BW; ++cc)
            sm.DY[R2::idx(ly0 + h * S_DY + r, lx0 + cc)] = __ldg(f.ntab + half_of(m5[r * S_BW + cc], h));
    } else {
      const int mu = u - S_UNITS;
      const int ly0 = -3 + (mu / M_UX) * M_BH, lx0 = -3 + (mu % M_UX) * M_BW;
      constexpr int P = M_BW + 2;
      const QuadLoaderU16<P, M_DY, XR6::W> ld{sm.X + XR6::idx(ly0 - 1, lx0 - 1)};
      U16x2 m3[M_BH * M_BW];
      blk_med3_8x2_ld<U16x2>(ld, m3);
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int r = 0; r < M_BH; ++r) {
          const int ty = ly0 + h * M_DY + r;
          if (ty >= TH + 3) continue;
#pragma unroll
          for (int cc = 0; cc < M_BW; ++cc)
            if (lx0 + cc < TW + 3) sm.M3[R3::idx(ty, lx0 + cc)] = (uint16_t)half_of(m3[r * M_BW + cc], h);
        }
    }
  }
  sat_flags<G, uint16_t, UM::MF>(f, sm);  // the med3 warps
}

// Appends val(it) for every set bit `it` of each lane's `hits` to a shared
// list with one atomic per warp (an exclusive scan of the lane counts):
// upward from lst[0] when top < 0, else downward from lst[top].
template <class V>
__device__ __forceinline__ void warp_emit(uint32_t hits, unsigned* cnt, uint16_t* lst, int top, V val) {
  const int lane = threadIdx.x & 31;
  const unsigned c = __popc(hits);
  unsigned incl = c;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  unsigned base = 0;
  if (lane == 31 && incl) base = atomicAdd(cnt, incl);
  base = __shfl_sync(0xffffffffu, base, 31) + incl - c;
  while (hits) {
    const int it = __ffs(hits) - 1;
    hits &= hits - 1u;
    lst[top < 0 ? (int)base : top - (int)base] = val(it);
    ++base;
  }
}

// Per-pixel part of the dense step, spread evenly over the block: L+, N and
// S = L+/(2N) at every R2 position from the working image and the parked
// med5 (float frames) or N (uint16 frames); for the tile's in-frame pixels
// also the saturation flag (the original input at an unflagged pixel) and
// the two sparse work lists.  Since S' <= S, a test S' > t can only pass
// where S > t: pixels with S > sigclip (unsaturated) are fine-structure
// items (S', then F where S' > sigclip), the others with S above the lower
// threshold are S'-only items; elsewhere every test fails.
template <class G, class XT>
__device__ __forceinline__ void dense_pixels(const FrameDesc& f, CoreSmemT<G, XT>& sm, int oy, int ox) {
  constexpr int TH = G::TH, TW = G::TW, NT = G::NT;
  using XR6 = typename G::XR6;
  using R2 = typename G::template Reg<2>;
  using R4 = typename G::template Reg<4>;
  constexpr bool kU16 = std::is_same<XT, uint16_t>::value;
  // Horizontal pixel pairs (even columns): 2-pixel aligned shared accesses.
  constexpr int PW = R2::W / 2;           // pairs per R2 row
  constexpr int NP = PW * R2::Hh;         // pairs on R2
  constexpr int IT = (NP + NT - 1) / NT;  // pairs per thread
  static_assert(R2::W % 2 == 0 && XR6::W % 2 == 0 && TW % 2 == 0 && 2 * IT <= 32, "pairs");
  uint32_t hits = 0, hits_f = 0;  // bit 2*it+e: pixel e of pair it is an S'-only / fine item
#pragma unroll 1
  for (int it = 0; it < IT; ++it) {
    const int q = it * NT + (int)threadIdx.x;
    if (q >= NP) break;
    const int ly = q / PW - 2, lx = (q % PW) * 2 - 2;
    const int c = XR6::idx(ly, lx), i2 = R2::idx(ly, lx);
    float S0, S1;
    if constexpr (kU16) {
      const auto ld2 = [&](int o) { return *reinterpret_cast<const uint32_t*>(sm.X + o); };
      const uint32_t mid = ld2(c), lft = ld2(c - 2), rgt = ld2(c + 2);
      const uint32_t up = ld2(c - XR6::W), dn = ld2(c + XR6::W);
      const int v0 = (int)(mid & 0xffffu), v1 = (int)(mid >> 16);
      const float L0 = lplus_int(v0, (int)(up & 0xffffu), (int)(dn & 0xffffu), (int)(lft >> 16), v1);
      const float L1 = lplus_int(v1, (int)(up >> 16), (int)(dn >> 16), v0, (int)(rgt & 0xffffu));
      const float4 dy = *reinterpret_cast<const float4*>(sm.DY + i2);  // {D0, y0, D1, y1}
      S0 = div_recip(L0, dy.x, dy.y);
      S1 = div_recip(L1, dy.z, dy.w);
    } else {
      const auto ld2 = [&](int o) { return *reinterpret_cast<const float2*>(sm.X + o); };
      const float2 mid = ld2(c), lft = ld2(c - 2), rgt = ld2(c + 2);
      const float2 up = ld2(c - XR6::W), dn = ld2(c + XR6::W);
      const float L0 = lplus(mid.x, up.x, dn.x, lft.y, mid.y);
      const float L1 = lplus(mid.y, up.y, dn.y, mid.x, rgt.x);
      const float2 m = *reinterpret_cast<const float2*>(sm.S + i2);
      const float N0 = noise_of(f, m.x), N1 = noise_of(f, m.y);
      S0 = __fdiv_rn(L0, __fadd_rn(N0, N0));
      S1 = __fdiv_rn(L1, __fadd_rn(N1, N1));
      if (ly >= 0 && ly < TH && lx >= 0 && lx < TW)
        *reinterpret_cast<float2*>(sm.N + ly * TW + lx) = make_float2(N0, N1);
    }
    *reinterpret_cast<float2*>(sm.S + i2) = make_float2(S0, S1);
    if (ly >= 0 && ly < TH && lx >= 0 && lx < TW) {
      const int t = ly * TW + lx;
      const uint32_t fl = *reinterpret_cast<const uint16_t*>(sm.flags + t);  // from sat_flags
      const bool sat0 = (fl & 8u) != 0, sat1 = (fl & 0x800u) != 0;
      if ((oy + ly) < f.ny) {
        const uint32_t b0 = 1u << (2 * it), b1 = b0 << 1;
        if ((ox + lx) < f.nx) {
          if (!sat0 && S0 > f.sigclip)
            hits_f |= b0;
          else if (S0 > f.thr_min)
            hits |= b0;
        }
        if ((ox + lx + 1) < f.nx) {
          if (!sat1 && S1 > f.sigclip)
            hits_f |= b1;
          else if (S1 > f.thr_min)
            hits |= b1;
        }
      }
    }
  }
  const auto tix = [&](int bit) {
    const int q = (bit >> 1) * NT + (int)threadIdx.x;
    return (uint16_t)((q / PW - 2) * TW + (q % PW) * 2 - 2 + (bit & 1));
  };
  warp_emit(hits_f, &sm.nlist2, sm.list, -1, tix);
  warp_emit(hits, &sm.nlist, sm.list, R4::N - 1, tix);
}

// The objlim test of step 5 at a pixel with S' = sp, noise N and med3 - med7
// difference diff: F = max(diff / N, 0.01) (diff itself without the
// normalisation), then S' / F > objlim.
// (diff <= 0 gives F = 0.01 whether or not it is divided by N > 0.)
__device__ __forceinline__ bool objlim_test(const FrameDesc& f, float sp, float N, float diff) {
  float F = 0.01f;
  if (diff > 0.0f) {
    F = f.fnorm ? __fdiv_rn(diff, N) : diff;
    F = F < 0.01f ? 0.01f : F;
  }
  return __fdiv_rn(sp, F) > f.objlim;
}

// The lo test of an S'-only item, fl(S - med5(S)) > lo, without the median.
// fl(S - x) can only fall as x grows, so the values x that pass form a lower
// set, and the median (rank 12 of the 25 window values, counted with
// multiplicity) passes iff at least 13 of the 25 values pass.
template <class LD>
__device__ __forceinline__ bool rank_lo_test(float Sc, float lo, const LD& ld5) {
  int pass = 0;
#pragma unroll
  for (int e = 0; e < 25; ++e) pass += __fsub_rn(Sc, ld5(e)) > lo;
  return pass >= 13;
}

// The objlim test of a uint16 frame without the med7 network.  The med3
// values are integers below 2^16, so the float difference m3 - v is exact
// and F depends on d = m3 - v alone; with S' > 0 the test can only turn from
// true to false as d grows (F is non-decreasing in d, S'/F non-increasing in
// F).  So the values v that pass are those v >= m3 - d*, d* the largest d
// that passes, and the median (rank 24 of the 49 window values) passes iff
// at least 25 of them do.  d* is taken from the real-number threshold
// (S'/objlim, times N when F is normalised) and confirmed with the float
// test itself at d* and d* + 1; the search moves at most four steps, and
// returns -1 when it has not settled (the caller then runs the network).
template <int W3>
__device__ __forceinline__ int objlim_rank_u16(const FrameDesc& f, float sp, float N, int m3, const uint16_t* w7) {
  if (!(sp > 0.0f)) return -1;
  const int dlo = m3 - 65535, dhi = m3;  // d over every possible med7 value 65535 .. 0
  const auto pass = [&](int d) { return objlim_test(f, sp, N, (float)d); };
  int ds;
  if (!pass(dlo)) {
    ds = dlo - 1;  // no med7 value passes
  } else if (pass(dhi)) {
    ds = dhi;  // every med7 value passes
  } else {     // pass(dlo) and not pass(dhi): dlo <= d* < dhi
    const float x = f.fnorm ? __fmul_rn(__fdiv_rn(sp, f.objlim), N) : __fdiv_rn(sp, f.objlim);
    int d = !(x > (float)dlo) ? dlo : (x > (float)dhi ? dhi - 1 : (int)ceilf(x) - 1);
    d = clampi(d, dlo, dhi - 1);
    ds = dlo - 2;  // unsettled
#pragma unroll 1
    for (int s = 0; s < 4; ++s) {
      if (!pass(d)) {  // then d > dlo
        --d;
      } else if (pass(d + 1)) {  // then d + 1 < dhi
        ++d;
      } else {
        ds = d;
        break;
      }
    }
    if (ds == dlo - 2) return -1;
  }
  const int t = m3 - ds;  // v passes iff v >= t
  int n = 0;
#pragma unroll
  for (int e = 0; e < 49; ++e) n += (int)w7[(e / 7) * W3 + e % 7] >= t;
  return n >= 25 ? 1 : 0;
}

// Work counters of a tile (valid in thread 0).  A block sums them over its
// tiles and adds them to the frame's state once per frame it leaves, instead
// of one same-address atomic per tile.
struct TileCounts {
  unsigned long long px = 0, sprime = 0, fine = 0, replace = 0, sprime_net = 0, fine_net = 0;
};

__device__ __forceinline__ void flush_counts(FrameState* st, const TileCounts& c) {
  if (!st) return;
  if (c.px) atomicAdd(&st->px_core, c.px);
  if (c.sprime) atomicAdd(&st->n_sprime, c.sprime);
  if (c.fine) atomicAdd(&st->n_fine, c.fine);
  if (c.replace) atomicAdd(&st->n_replace, c.replace);
  if (c.sprime_net) atomicAdd(&st->n_sprime_net, c.sprime_net);
  if (c.fine_net) atomicAdd(&st->n_fine_net, c.fine_net);
}

template <class G, class XT>
__device__ TileCounts core_tile(const FrameDesc& f, int k, int tix, CoreSmemT<G, XT>& sm) {
  constexpr int TH = G::TH, TW = G::TW, TWW = G::TWW, NT = G::NT, MWORDS = G::MWORDS;
  using XR6 = typename G::XR6;
  using R2 = typename G::template Reg<2>;
  using R3 = typename G::template Reg<3>;
  using R4 = typename G::template Reg<4>;
  using KT = KeyOf<XT>;
  using K = typename KT::K;
  constexpr bool kU16 = std::is_same<XT, uint16_t>::value;
  const int tid = threadIdx.x;
  const int oy = (tix / f.tiles_x) * TH;
  const int ox = (tix % f.tiles_x) * TW;
  const int ny = f.ny, nx = f.nx;
  const bool edge = (oy - 6 < 0) || (ox - 6 < 0) || (oy + TH + 6 > ny) || (ox + TW + 6 > nx);
  const uint32_t* Mp = ((k - 1) & 1) ? f.mbuf1 : f.mbuf0;
  TileCounts counts;

  for (int i = tid; i < 3 * TH * TWW; i += NT) (&sm.pw[0][0][0])[i] = 0u;
  if (tid == 0) sm.nfine = sm.nfine_net = 0;

  // The tile's words of the grown saturated set (satgrow > 0): the load is
  // issued before the staging and stored after it, so it waits for nothing.
  const bool sat_words = f.satgrow && tid < TH * TWW;
  uint32_t sw = 0;
  if (sat_words) {
    const int ly = tid / TWW, w = (ox >> 5) + tid % TWW;
    if (w < f.wpr) sw = __ldg(f.p_sat + (size_t)min(oy + ly, ny - 1) * f.wpr + w);
  }

  // Stage X0 and M_{k-1} on R6 at clamped coordinates.
  bool bad = false;
  stage_x0_mask<G, 6>(f, Mp, oy, ox, sm.X, sm.Mb, sm.Mw, bad);
  if (sat_words) sm.Sw[tid / TWW][tid % TWW] = sw;
  if (tid == 0) sm.nlist = 0;
  if (bad) atomicOr(&f.st->err, ERR_NONFINITE);
  __syncthreads();

  // Step 7 of the previous iteration: I_{k-1} = R(X0, M_{k-1}) on R4, at the
  // flagged pixels (a compacted list; reads touch unflagged pixels only, so
  // it is done in place).
  if (k > 1) {
    // The flagged pixels of R4 straight from the staged mask words: one
    // (row, word) pair per thread.
    const int cx0 = max(0, ox - 4), cx1 = min(nx, ox + TW + 4);
    const int w0 = clampi(ox - 8, 0, nx - 1) >> 5;  // as staged
    for (int i = tid; i < (TH + 8) * MWORDS; i += NT) {
      const int ly = i / MWORDS - 4, j = i % MWORDS;
      const int gy = oy + ly;
      if (gy < 0 || gy >= ny) continue;
      const int wbase = (w0 + j) * 32;
      uint32_t bits = sm.Mw[ly + 6][j];
      const int lo = cx0 - wbase, hi = cx1 - wbase;  // keep bits b with lo <= b < hi
      if (hi <= 0 || lo >= 32) continue;
      if (lo > 0) bits &= 0xffffffffu << lo;
      if (hi < 32) bits &= (1u << hi) - 1u;
      if (!bits) continue;
      unsigned pos = atomicAdd(&sm.nlist, (unsigned)__popc(bits));
      while (bits) {
        const int b = __ffs(bits) - 1;
        bits &= bits - 1u;
        sm.list[pos++] = (uint16_t)XR6::idx(ly, wbase + b - ox);
      }
    }
    __syncthreads();
    const unsigned n = sm.nlist;
    for (unsigned j = tid; j < n; j += NT) {
      const int c = sm.list[j];
      XT v;
      if (!maskmed5(sm.X, sm.Mb, XR6::W, c, v)) {
        const int ly = c / XR6::W - 6, lx = c % XR6::W - 8;
        v = (XT)maskmed_wide(f, Mp, oy + ly, ox + lx, 3);
        atomicAdd(&f.st->n_replace_wide, 1ull);
        f.tflags[2 * tiles_of(f) + tix] = 1;  // this tile now depends on more than tile + 6
      }
      sm.X[c] = v;
    }
    if (tid == 0) {
      sm.nlist = 0;
      counts.replace = n;
    }
    __syncthreads();
    if (edge) {
      for (int i = tid; i < R4::N; i += NT) {
        const int ly = i / R4::W - 4, lx = i % R4::W - 4;
        const int gy = oy + ly, gx = ox + lx;
        if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) continue;
        sm.X[XR6::idx(ly, lx)] = sm.X[XR6::idx(clampi(gy, 0, ny - 1) - oy, clampi(gx, 0, nx - 1) - ox)];
      }
      __syncthreads();
    }
  }

  // Dense part: med5 on R2 and med3 on R3 (register blocks of shared min/max
  // networks), then L+, N, S, the saturation flags and the S' list per pixel.
  if constexpr (kU16)
    dense_u16<G>(f, sm);
  else
    dense_f32<G>(f, sm);
  if (tid == 0) sm.nlist2 = 0;
  __syncthreads();
  dense_pixels<G, XT>(f, sm, oy, ox);
  __syncthreads();
  if (edge) {
    for (int i = tid; i < R2::N; i += NT) {
      const int ly = i / R2::W - 2, lx = i % R2::W - 2;
      const int gy = oy + ly, gx = ox + lx;
      if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) continue;
      sm.S[i] = sm.S[R2::idx(clampi(gy, 0, ny - 1) - oy, clampi(gx, 0, nx - 1) - ox)];
    }
    for (int i = tid; i < R3::N; i += NT) {
      const int ly = i / R3::W - 3, lx = i % R3::W - 3;
      const int gy = oy + ly, gx = ox + lx;
      if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) continue;
      sm.M3[i] = sm.M3[R3::idx(clampi(gy, 0, ny - 1) - oy, clampi(gx, 0, nx - 1) - ox)];
    }
  }
  // Steps 4-5 on the sparse items, one block-wide phase: S' = S - med5(S),
  // the sig and lo bits, and at fine items with S' > sigclip F = max((med3 -
  // med7(med3))/N, 0.01) and the objlim test S'/F > objlim.  Fine items (the
  // costly ones) come first and rounds alternate direction, so the cheap
  // S'-only items of a second round land on the threads without a fine item.
  // An S'-only item needs nothing but the lo test, which is decided by rank
  // (rank_lo_test); the objlim test of a uint16 frame is decided by rank too
  // (objlim_rank_u16).  Both give the bit the median would give.
  if (edge) __syncthreads();
  const unsigned n = sm.nlist, n2 = sm.nlist2, total = n + n2;
  unsigned n_eval = 0, n_net7 = 0;
  for (unsigned r = 0; r * NT < total; ++r) {
    const unsigned q = r * NT + ((r & 1) ? (NT - 1 - tid) : tid);
    if (q >= total) continue;
    const bool fine = q < n2;
    const int i = fine ? sm.list[q] : sm.list[R4::N - 1 - (int)(q - n2)];
    const int ly = i / TW, lx = i % TW;
    const int c = R2::idx(ly, lx);
    const float* wb = sm.S + c - 2 * R2::W - 2;
    const auto ld5 = [&](int e) { return wb[(e / 5) * R2::W + e % 5]; };
    const bool sat = (sm.flags[i] & 8) != 0;  // never set for fine items
    const uint32_t bit = 1u << (lx & 31);
    if (!fine && !f.sepmed) {  // S'-only item: S' <= S <= sigclip, or saturated
      if (!sat && rank_lo_test(sm.S[c], f.lo, ld5)) atomicOr(&sm.pw[1][ly][lx >> 5], bit);
      continue;
    }
    float m;
    if (f.sepmed)
      sep5x5_ld<float>(ld5, &m);
    else
      med5x5_ld<float>(ld5, &m);
    const float sp = __fsub_rn(sm.S[c], m);
    if (!sat && sp > f.lo) atomicOr(&sm.pw[1][ly][lx >> 5], bit);
    if (!fine || !(sp > f.sigclip)) continue;  // S'-only items have S' <= S <= sigclip
    atomicOr(&sm.pw[0][ly][lx >> 5], bit);
    ++n_eval;
    const int c3 = R3::idx(ly, lx);
    const XT* w7 = sm.M3 + c3 - 3 * R3::W - 3;
    float N;
    if constexpr (kU16)
      N = __fmul_rn(sm.DY[c].x, 0.5f);  // the table holds 2N; halving is exact
    else
      N = sm.N[i];
    int cand = -1;
    if constexpr (kU16) cand = objlim_rank_u16<R3::W>(f, sp, N, (int)sm.M3[c3], w7);
    if (cand < 0) {  // float frames, and searches that did not settle: the med7 network
      const auto ld7 = [&](int e) { return KT::key(w7[(e / 7) * R3::W + e % 7]); };
      K m7;
      med7x7_ld<K>(ld7, &m7);
      ++n_net7;
      const float diff = __fsub_rn((float)sm.M3[c3], (float)KT::back(m7));
      cand = objlim_test(f, sp, N, diff);
    }
    if (cand) atomicOr(&sm.pw[2][ly][lx >> 5], bit);
  }
  n_eval = __reduce_add_sync(0xffffffffu, n_eval);
  if ((tid & 31) == 0 && n_eval) atomicAdd(&sm.nfine, n_eval);
  if constexpr (!kU16) {
    n_net7 = __reduce_add_sync(0xffffffffu, n_net7);
    if ((tid & 31) == 0 && n_net7) atomicAdd(&sm.nfine_net, n_net7);
  } else {
    if (__any_sync(0xffffffffu, n_net7 != 0)) {  // rare: only searches that did not settle
      n_net7 = __reduce_add_sync(0xffffffffu, n_net7);
      if ((tid & 31) == 0) atomicAdd(&sm.nfine_net, n_net7);
    }
  }
  __syncthreads();

  // Bit-planes of the tile out (only in-frame pixels ever set a bit).
  for (int t = tid; t < 3 * TH * TWW; t += NT) {
    const int pl = t / (TH * TWW), r = (t / TWW) % TH, wd = t % TWW;
    const int gy = oy + r, w = (ox >> 5) + wd;
    if (gy < ny && w < f.wpr) {
      uint32_t* P = pl == 0 ? f.p_sig : (pl == 1 ? f.p_lo : f.p_cand);
      P[(size_t)gy * f.wpr + w] = sm.pw[pl][r][wd];
    }
  }
  if (tid == 0) {
    counts.px = (unsigned long long)(min(TH, ny - oy) * min(TW, nx - ox));
    counts.sprime = total;
    counts.fine = sm.nfine;
    counts.sprime_net = f.sepmed ? total : n2;
    counts.fine_net = sm.nfine_net;
  }
  return counts;
}

// G: the tile geometry (shape and threads); MINB: resident CTAs per SM the
// register allocation is bounded for (the variants trade registers, and so
// spills, against occupancy).  One kernel
// per working-image type: a request orders its frames so that each type's
// tiles form one contiguous item range [item_begin, item_end), and a launch
// walks only its own range (its own queue head).
template <class G, int MINB, class XT>
__global__ void __launch_bounds__(G::NT, MINB) core_kernel(const FrameDesc* __restrict__ fr, int nframes,
                                                           unsigned item_begin, unsigned item_end, int k,
                                                           unsigned* head) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ unsigned s_item;
  __shared__ int s_run, s_fi;
  constexpr int kDtype = std::is_same<XT, uint16_t>::value ? 1 : 0;
  __shared__ TileCounts acc;       // sums of the tiles of frame acc_st so far (thread 0)
  __shared__ FrameState* acc_st;
  if (threadIdx.x == 0) {
    acc = TileCounts{};
    acc_st = nullptr;
  }
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned item = item_begin + atomicAdd(head, 1u);
      int run = 0, fi = 0;
      if (item < item_end) {
        fi = frame_of(fr, nframes, item);
        const FrameDesc& f = fr[fi];
        run = f.dtype == kDtype && iteration_runs(f, k);
        if (run && k > 1) {  // levels after the first: only the tiles whose inputs changed
          const unsigned t = item - f.tile_begin;
          uint8_t* mk = f.tflags + (size_t)(k & 1) * tiles_of(f) + t;
          run = *mk || f.tflags[2 * tiles_of(f) + t];
          *mk = 0;
        }
      }
      s_item = item;
      s_run = run;
      s_fi = fi;
    }
    __syncthreads();
    const unsigned item = s_item;
    const int run = s_run;
    __syncthreads();
    if (item >= item_end) break;
    if (!run) continue;
    const FrameDesc& f = fr[s_fi];
    const TileCounts c = core_tile<G, XT>(f, k, (int)(item - f.tile_begin),
                                         *reinterpret_cast<CoreSmemT<G, XT>*>(smem_raw));
    if (threadIdx.x == 0) {
      if (f.st != acc_st) {
        flush_counts(acc_st, acc);
        acc = TileCounts{};
        acc_st = f.st;
      }
      acc.px += c.px;
      acc.sprime += c.sprime;
      acc.fine += c.fine;
      acc.replace += c.replace;
      acc.sprime_net += c.sprime_net;
      acc.fine_net += c.fine_net;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) flush_counts(acc_st, acc);
}

// ---- which core tiles a level must recompute -------------------------------
//
// A core tile's bit-planes at level k+1 depend on the mask M_k only within
// its tile + 6 (the replacement windows of tile + 4 and the saturation flags),
// unless a replacement there needed a window wider than 5x5.  So a tile with
// no pixel newly flagged by level k within 6 pixels, and no wide window so
// far, would recompute exactly the planes it already holds: level k+1 skips
// it.  grow_kernel(k) marks the tiles near its new flags; core_kernel(k+1)
// reads and clears the mark; a tile that needs a wide window is marked for
// good.


// Marks for level kn every tile whose rows/columns +-6 hold a set bit of
// `bits`, the new flags of word w of row y: tile rows floor((y-6)/th) ..
// floor((y+6)/th), likewise for the columns of the set bits.  The core tile
// sides are powers of two (sh_h, sh_w: their log2), so an arithmetic shift
// is that floor, also for negative numerators.
__device__ __forceinline__ void mark_tiles(const FrameDesc& f, int kn, int y, int w, uint32_t bits, int sh_h,
                                           int sh_w, int tiles_y) {
  const int x_lo = w * 32 + __ffs(bits) - 1, x_hi = w * 32 + 31 - __clz(bits);
  const int ty0 = max(0, (y - 6) >> sh_h), ty1 = min(tiles_y - 1, (y + 6) >> sh_h);
  const int tx0 = max(0, (x_lo - 6) >> sh_w), tx1 = min(f.tiles_x - 1, (x_hi + 6) >> sh_w);
  uint8_t* d = f.tflags + (size_t)(kn & 1) * tiles_of(f);
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx) d[ty * f.tiles_x + tx] = 1;
}

// ---- step 6: growth on 32-pixel words --------------------------------------

__device__ __forceinline__ uint32_t plane_word(const uint32_t* P, int ny, int wpr, int y, int w) {
  if (y < 0 || y >= ny || w < 0 || w >= wpr) return 0u;
  return __ldg(P + (size_t)y * wpr + w);
}

// Horizontal 3-dilation of word c with the edge bits of its neighbours.
__device__ __forceinline__ uint32_t hdil(uint32_t l, uint32_t c, uint32_t r) {
  return c | (c << 1) | (c >> 1) | (l >> 31) | (r << 31);
}

// Growth blocks of H rows x W words, WPT words per thread: 64 x 16 for
// requests of many blocks (12% less time per level on a 61-Mpx frame than
// 32 x 8: the halo words are a smaller share), 32 x 8 for small requests.
template <int H_, int W_>
struct GrowGeo {
  static constexpr int H = H_, W = W_, WPT = H * W / kBlock;
  static_assert(H * W == WPT * kBlock, "whole words per thread");
};
using GrowBig = GrowGeo<64, 16>;
using GrowSmall = GrowGeo<32, 8>;

__device__ __forceinline__ int frame_of_gblk(const FrameDesc* fr, int nframes, unsigned b) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (fr[mid].gblk_begin <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Step 6 for a block of GG::H rows x GG::W words: the candidate words (with a
// 2-row, 2-word halo) and the first growth g1 = dil3(cand) & sig (1-row,
// 1-word halo) are staged in shared memory; each thread then forms
// g2 = dil3(g1) & lo for its words, M_k = M_{k-1} | g2, and counts new flags.
// Every global load of the block (candidate, sig, lo and mask words) is
// issued up front, so the block waits for one memory round trip.  Bounded
// for six resident blocks per SM (40 registers, no spills).
template <class GG>
__global__ void __launch_bounds__(kBlock, 6) grow_kernel(const FrameDesc* __restrict__ fr, int nframes,
                                                      unsigned total_blocks, int k) {
  constexpr int NT = kBlock, GB_H = GG::H, GB_W = GG::W, GB_WPT = GG::WPT;
  constexpr int CW = GB_W + 4;  // candidate region: GB_H + 4 rows of CW words
  constexpr int GW = GB_W + 2;  // g1 region: GB_H + 2 rows of GW words
  // The halo regions in two dimensions: a thread keeps one column of a region
  // and steps its rows, so each load costs a row test and an address, not a
  // division by the region's width.
  constexpr int CR = NT / CW, CPASS = (GB_H + 4 + CR - 1) / CR;  // candidate rows per pass, passes
  constexpr int GR = NT / GW, GPASS = (GB_H + 2 + GR - 1) / GR;  // g1 rows per pass, passes
  __shared__ uint32_t C[GB_H + 4][CW];
  __shared__ uint32_t G1[GB_H + 2][GW];
  const int tid = threadIdx.x;
  const unsigned blk = blockIdx.x;
  if (blk >= total_blocks) return;
  const FrameDesc& f = fr[frame_of_gblk(fr, nframes, blk)];
  if (!iteration_runs(f, k)) return;
  const unsigned b = blk - f.gblk_begin;
  const int y0 = (int)(b / (unsigned)f.gblk_x) * GB_H, w0 = (int)(b % (unsigned)f.gblk_x) * GB_W;
  const int ny = f.ny, wpr = f.wpr;
  const uint32_t* Mp = ((k - 1) & 1) ? f.mbuf1 : f.mbuf0;
  const int cc = tid % CW, cr0 = tid / CW, gc = tid % GW, gr0 = tid / GW;
  const int cwc = w0 - 2 + cc, gwc = w0 - 1 + gc;  // frame word columns of this thread
  const bool ccol = cr0 < CR && cwc >= 0 && cwc < wpr, gcol = gr0 < GR && gwc >= 0 && gwc < wpr;
  uint32_t cw[CPASS], sw[GPASS];
#pragma unroll
  for (int p = 0; p < CPASS; ++p) {
    const int r = cr0 + p * CR, y = y0 - 2 + r;
    cw[p] = (ccol && r < GB_H + 4 && y >= 0 && y < ny) ? __ldg(f.p_cand + (size_t)y * wpr + cwc) : 0u;
  }
#pragma unroll
  for (int p = 0; p < GPASS; ++p) {
    const int r = gr0 + p * GR, y = y0 - 1 + r;
    sw[p] = (gcol && r < GB_H + 2 && y >= 0 && y < ny) ? __ldg(f.p_sig + (size_t)y * wpr + gwc) : 0u;
  }
  uint32_t lo[GB_WPT], mp[GB_WPT];
#pragma unroll
  for (int p = 0; p < GB_WPT; ++p) {
    const int i = p * NT + tid, y = y0 + i / GB_W, w = w0 + i % GB_W;
    const bool own = y < ny && w < wpr;
    lo[p] = own ? __ldg(f.p_lo + (size_t)y * wpr + w) : 0u;
    mp[p] = own ? __ldg(Mp + (size_t)y * wpr + w) : 0u;
  }
  if (cr0 < CR) {
#pragma unroll
    for (int p = 0; p < CPASS; ++p) {
      const int r = cr0 + p * CR;
      if (r < GB_H + 4) C[r][cc] = cw[p];
    }
  }
  __syncthreads();
  if (gr0 < GR) {
#pragma unroll
    for (int p = 0; p < GPASS; ++p) {
      const int r = gr0 + p * GR;
      if (r < GB_H + 2) {
        uint32_t d = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) d |= hdil(C[r + a][gc], C[r + a][gc + 1], C[r + a][gc + 2]);
        G1[r][gc] = d & sw[p];
      }
    }
  }
  __syncthreads();
  bool any = false;
  uint32_t* Mn = (k & 1) ? f.mbuf1 : f.mbuf0;
  const int sh_h = __ffs(f.th) - 1, sh_w = __ffs(f.tw) - 1;  // the request's core tiles
  const int tiles_y = (ny + f.th - 1) >> sh_h;
#pragma unroll
  for (int p = 0; p < GB_WPT; ++p) {
    const int i = p * NT + tid, ty = i / GB_W, tx = i % GB_W;
    const int y = y0 + ty, w = w0 + tx;
    if (y < ny && w < wpr) {
      uint32_t d2 = 0;
#pragma unroll
      for (int a = 0; a < 3; ++a) d2 |= hdil(G1[ty + a][tx], G1[ty + a][tx + 1], G1[ty + a][tx + 2]);
      const uint32_t g2 = d2 & lo[p];
      Mn[(size_t)y * wpr + w] = mp[p] | g2;
      const uint32_t fresh = g2 & ~mp[p];
      any = any || fresh != 0;
      if (fresh && k < f.niter) mark_tiles(f, k + 1, y, w, fresh, sh_h, sh_w, tiles_y);
    }
  }
  // Only "did level k flag anything" is used (early stop): one flag store
  // per block that found new pixels, skipped once some block has set it.
  if (__syncthreads_or(any) && tid == 0 && !*(volatile unsigned long long*)&f.st->fresh[k])
    f.st->fresh[k] = 1;
}

// ---- output: cleaned frame and uint8 mask of the last mask ----------------

template <class FG, class XT>
struct FinalSmemT {
  XT X[FG::XR3::N];
  uint8_t Mb[FG::XR3::N];
  uint32_t Mw[FG::TH + 6][FG::MWORDS];
  uint16_t list[FG::TH * FG::TW];
  unsigned nlist;
};

// The rare replacements whose 5x5 window is fully flagged: the 7x7 window
// from shared memory, else wider windows from global memory.  Kept out of
// line so that the common path's register allocation does not carry the
// 49-key network.
template <class FG, class XT>
__device__ __noinline__ XT replace_wide(const FrameDesc& f, const uint32_t* M, const FinalSmemT<FG, XT>& sm, int c,
                                        int gy, int gx) {
  XT v;
  if (!maskmed7(sm.X, sm.Mb, FG::XR3::W, c, v)) v = (XT)maskmed_wide(f, M, gy, gx, 4);
  return v;
}

// cleaned = R(X0, M_run) (the masked median at flagged pixels, X0 elsewhere),
// mask = M_run as uint8, the flagged count and the iterations run.  The
// flagged pixels of a tile are compacted into a list, replaced in shared
// memory, and the tile is then written out coalesced, four pixels per
// thread where the row pitch allows 16-byte stores.
template <class FG, class XT>
__device__ unsigned finalize_tile(const FrameDesc& f, int tix, FinalSmemT<FG, XT>& sm) {
  constexpr int TH = FG::TH, TW = FG::TW, TWW = FG::TWW, NT = kBlock;
  using XR3 = typename FG::XR3;
  static_assert(FG::NT == kBlock, "finalize geometry");
  const int tid = threadIdx.x;
  const int oy = (tix / f.ftiles_x) * TH, ox = (tix % f.ftiles_x) * TW;
  const int run = run_of(f);
  const uint32_t* M = (run & 1) ? f.mbuf1 : f.mbuf0;
  bool bad = false;
  stage_x0_mask<FG, 3>(f, M, oy, ox, sm.X, sm.Mb, sm.Mw, bad);
  if (bad) atomicOr(&f.st->err, ERR_NONFINITE);
  __syncthreads();
  // The tile's flagged pixels straight from the staged mask words (the
  // tile's columns are whole words; bits beyond the frame are never set):
  // the first two warps, one word each, one shared atomic per warp.
  static_assert(TH * TWW % 32 == 0 && TH * TWW <= NT, "whole warps of mask words");
  if (tid < TH * TWW) {
    const int ly = tid / TWW, wd = tid % TWW;
    const int w0 = clampi(ox - 8, 0, f.nx - 1) >> 5;  // as staged
    const uint32_t bits = (oy + ly) < f.ny ? sm.Mw[ly + 3][((ox >> 5) + wd) - w0] : 0u;
    warp_emit(bits, &sm.nlist, sm.list, -1, [&](int b) { return (uint16_t)(ly * TW + wd * 32 + b); });
  }
  __syncthreads();
  const unsigned n = sm.nlist;
  // In place: reads touch unflagged pixels only, writes flagged ones.
  for (unsigned j = tid; j < n; j += NT) {
    const int i = sm.list[j];
    const int ly = i / TW, lx = i % TW;
    const int c = XR3::idx(ly, lx);
    XT v;
    if (!maskmed5(sm.X, sm.Mb, XR3::W, c, v)) v = replace_wide<FG, XT>(f, M, sm, c, oy + ly, ox + lx);
    sm.X[c] = v;
  }
  __syncthreads();
  // 16-byte stores of the cleaned frame and 4-byte stores of the mask where
  // the row pitch and the caller's output pointers allow them.
  const bool vec = (f.nx & 3) == 0 && (reinterpret_cast<uintptr_t>(f.clean_out) & 15u) == 0 &&
                   (reinterpret_cast<uintptr_t>(f.mask_out) & 3u) == 0;
  for (int qd = tid; qd < TH * TW / 4; qd += NT) {
    const int ly = qd / (TW / 4), lx = (qd % (TW / 4)) * 4;
    const int gy = oy + ly, gx = ox + lx;
    if (gy >= f.ny || gx >= f.nx) continue;
    const int c = XR3::idx(ly, lx);
    const size_t q = (size_t)gy * f.nx + gx;
    if (vec && gx + 3 < f.nx) {  // c is a multiple of 4: aligned shared-memory reads
      float4 o;
      if constexpr (std::is_same<XT, float>::value) {
        o = *reinterpret_cast<const float4*>(sm.X + c);
      } else {
        const uint2 u = *reinterpret_cast<const uint2*>(sm.X + c);
        o = make_float4((float)(u.x & 0xffffu), (float)(u.x >> 16), (float)(u.y & 0xffffu), (float)(u.y >> 16));
      }
      *reinterpret_cast<float4*>(f.clean_out + q) = o;
      *reinterpret_cast<uint32_t*>(f.mask_out + q) = *reinterpret_cast<const uint32_t*>(sm.Mb + c);
    } else {
      for (int e = 0; e < 4 && gx + e < f.nx; ++e) {
        f.clean_out[q + e] = (float)sm.X[c + e];
        f.mask_out[q + e] = sm.Mb[c + e];
      }
    }
  }
  if (tid == 0 && tix == 0) f.st->iters_run = run;
  return n;
}

template <class FG>
__global__ void __launch_bounds__(kBlock, 6) finalize_kernel(const FrameDesc* __restrict__ fr, int nframes,
                                                         unsigned total, unsigned* head) {
  __shared__ __align__(16) unsigned char smem[sizeof(FinalSmemT<FG, float>)];
  __shared__ unsigned s_item;
  const int tid = threadIdx.x;
  __shared__ unsigned long long flagged;  // flagged pixels of frame acc_st so far (thread 0)
  __shared__ FrameState* acc_st;
  if (tid == 0) {
    flagged = 0;
    acc_st = nullptr;
  }
  for (;;) {
    if (tid == 0) s_item = atomicAdd(head, 1u);
    __syncthreads();
    const unsigned item = s_item;
    if (item >= total) break;
    const FrameDesc& f = fr[frame_of_fin(fr, nframes, item)];
    const int tix = (int)(item - f.fin_begin);
    unsigned n;
    if (f.dtype == 1) {
      auto& sm = *reinterpret_cast<FinalSmemT<FG, uint16_t>*>(smem);
      if (tid == 0) sm.nlist = 0;
      __syncthreads();
      n = finalize_tile<FG, uint16_t>(f, tix, sm);
    } else {
      auto& sm = *reinterpret_cast<FinalSmemT<FG, float>*>(smem);
      if (tid == 0) sm.nlist = 0;
      __syncthreads();
      n = finalize_tile<FG, float>(f, tix, sm);
    }
    if (tid == 0) {
      if (f.st != acc_st) {
        if (acc_st && flagged) atomicAdd(&acc_st->flagged, flagged);
        flagged = 0;
        acc_st = f.st;
      }
      flagged += n;
    }
    __syncthreads();
  }
  if (tid == 0 && acc_st && flagged) atomicAdd(&acc_st->flagged, flagged);
}

}  // namespace lacos
