// Device code of the L.A.Cosmic detect-and-clean iteration (sm_103a).
//
// Iteration k is two kernels over the frame's tiles:
//   core_kernel: a CTA takes a TH x TW output tile, stages the original
//     frame X0 and the cumulative mask M_{k-1} with a 6-pixel halo in shared
//     memory and rebuilds the working image I_{k-1} on the fly (unflagged
//     pixels keep X0, flagged pixels take the masked median of unflagged X0:
//     step 7 of the previous iteration depends only on X0 and M_{k-1}).  It
//     then computes L+, N and S densely on the tile + 2, med3(I) on the
//     tile + 3, and -- only where a threshold can still pass, from compacted
//     lists -- S' = S - med5(S) and the fine-structure test, and writes three
//     bit-planes for the tile: S' > sigclip, S' > sigfrac*sigclip (both
//     excluding saturated pixels) and the candidates (steps 1-5).
//   grow_kernel: word-parallel 3x3 dilations of the bit-planes (step 6),
//     M_k = M_{k-1} | g2 and the count of newly flagged pixels.
// finalize_kernel writes the uint8 mask and the float32 cleaned frame.
//
// Every stage evaluates its own array at in-frame positions only and reads
// out-of-frame neighbours at clamped coordinates (clamp-to-edge per stage).
//
// Exactness: all float arithmetic uses the explicit round-to-nearest
// intrinsics in the same operation order as the float32 CPU definition, the
// translation unit is compiled with -fmad=false, and medians are selections
// (min/max networks), so results are bit-identical to it.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lacos.h"

namespace lacos_net {
template <class K> __device__ __forceinline__ K neg_inf();
template <class K> __device__ __forceinline__ K pos_inf();
template <> __device__ __forceinline__ float neg_inf<float>() { return -__int_as_float(0x7f800000); }
template <> __device__ __forceinline__ float pos_inf<float>() { return __int_as_float(0x7f800000); }
}  // namespace lacos_net

__device__ __forceinline__ float MN(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float MX(float a, float b) { return fmaxf(a, b); }

#include "networks.cuh"

namespace lacos {

constexpr int TH = 32;   // output tile rows
constexpr int TW = 64;   // output tile columns (two 32-bit mask words per row)
constexpr int TWW = TW / 32;
constexpr int NT = 256;  // threads per CTA
constexpr int HX = 6;    // staging halo of the core kernel

constexpr unsigned ERR_NONFINITE = 1u;
constexpr unsigned ERR_TIMEOUT = 2u;

struct FrameState {
  unsigned long long fresh[LACOS_MAX_NITER + 1];  // new pixels found by iteration k
  unsigned long long flagged;                      // pixels in the final mask
  unsigned long long n_sprime, n_fine, n_replace;  // sparse-work counters (profiling)
  unsigned int err;
  int iters_run;
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
  uint8_t* mask_out;
  float* clean_out;
  FrameState* st;
  float gain, rn2, satlevel, sigclip, lo, thr_min, objlim;
  int niter, fnorm;
  int tiles_x;
  unsigned int tile_begin, tile_end;    // this frame's range in the flattened tile list
  unsigned long long word_begin;        // this frame's range in the flattened word list
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

// Masked median with the window widened beyond 5x5 (rare: every pixel of
// the 5x5 window is flagged).  Reads X0 and the mask from global memory and
// selects the lower median by a 32-pass radix select on order keys.
__device__ float maskmed_wide(const FrameDesc& f, const uint32_t* M, int gy, int gx) {
  const int rmax = max(f.ny, f.nx) + 2;
  bool bad = false;
  for (int r = 3; r <= rmax; ++r) {
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

// Masked 5x5 median at shared-memory index c of X (pitch P) with flags Mb:
// the lower median of the unflagged members.  Flagged members are replaced
// by sentinels, the first (12 - (n-1)/2) by -inf and the rest by +inf, so
// that the rank-12 element of the 25 is the rank-(n-1)/2 unflagged value.
// Returns false when no member is unflagged.
__device__ __forceinline__ bool maskmed5(const float* X, const uint8_t* Mb, int P, int c, float& out) {
  int n = 0;
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) n += Mb[c + dy * P + dx] ? 0 : 1;
  if (n == 0) return false;
  const int plo = 12 - (n - 1) / 2;
  float v[25];
  int seen = 0;
#pragma unroll
  for (int dy = -2; dy <= 2; ++dy)
#pragma unroll
    for (int dx = -2; dx <= 2; ++dx) {
      const int q = c + dy * P + dx;
      const bool fl = Mb[q] != 0;
      const float s = (seen < plo) ? lacos_net::neg_inf<float>() : lacos_net::pos_inf<float>();
      seen += fl ? 1 : 0;
      v[(dy + 2) * 5 + dx + 2] = fl ? s : X[q];
    }
  med5x5<float>(v, &out);
  return true;
}

template <int H>
struct Reg {
  static constexpr int W = TW + 2 * H;
  static constexpr int Hh = TH + 2 * H;
  static constexpr int N = W * Hh;
  __device__ static __forceinline__ int idx(int ly, int lx) { return (ly + H) * W + (lx + H); }
};

__device__ __forceinline__ int frame_of(const FrameDesc* fr, int nframes, unsigned item) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (fr[mid].tile_begin <= item) lo = mid; else hi = mid - 1;
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

// Warp-aggregated append of `val` to a shared list when `pred` holds.  All
// 32 lanes of the warp must call it.
__device__ __forceinline__ void list_append(bool pred, uint16_t val, uint16_t* lst, unsigned* cnt) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (!m) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(cnt, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) lst[base + __popc(m & ((1u << lane) - 1u))] = val;
}

// Copies every out-of-frame position of region H of an array indexed with
// Reg<ARH> from its clamped in-frame position (clamp-to-edge of that stage).
template <int H, int ARH, class T>
__device__ __forceinline__ void edge_fill(T* A, int oy, int ox, int ny, int nx) {
  for (int i = threadIdx.x; i < Reg<H>::N; i += NT) {
    const int ly = i / Reg<H>::W - H, lx = i % Reg<H>::W - H;
    const int gy = oy + ly, gx = ox + lx;
    if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) continue;
    const int cy = clampi(gy, 0, ny - 1) - oy, cx = clampi(gx, 0, nx - 1) - ox;
    A[Reg<ARH>::idx(ly, lx)] = A[Reg<ARH>::idx(cy, cx)];
  }
}

struct CoreSmem {
  float X[Reg<6>::N];        // X0, then I_{k-1} on R4
  uint8_t Mb[Reg<6>::N];     // M_{k-1}
  float S[Reg<2>::N];        // S on R2
  float M3[Reg<3>::N];       // med3(I) on R3
  float SpL[TH * TW];        // S' of the entries of the S' list
  uint16_t list[Reg<4>::N];  // compacted work list (R4 indices for replacement, R0 otherwise)
  uint16_t list2[TH * TW];   // F list: indices into the S' list
  uint8_t flags[TH * TW];    // bit0: S' > sigclip, bit1: S' > lo, bit2: candidate
  unsigned nlist, nlist2;
  unsigned n_sp, n_f, n_rep;
};

__device__ __forceinline__ float med5_at(const float* A, int P, int c) {
  float w[25];
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = 0; b < 5; ++b) w[a * 5 + b] = A[c + (a - 2) * P + (b - 2)];
  float m;
  med5x5<float>(w, &m);
  return m;
}

__device__ __forceinline__ float noise_of(const FrameDesc& f, float m5) {
  const float gm = __fmul_rn(f.gain, m5);
  const float e = gm < 1e-4f ? 1e-4f : gm;
  return __fdiv_rn(__fsqrt_rn(__fadd_rn(e, f.rn2)), f.gain);
}

__device__ void core_tile(const FrameDesc& f, int k, int tix, CoreSmem& sm) {
  const int tid = threadIdx.x;
  const int oy = (tix / f.tiles_x) * TH;
  const int ox = (tix % f.tiles_x) * TW;
  const int ny = f.ny, nx = f.nx;
  const uint32_t* Mp = ((k - 1) & 1) ? f.mbuf1 : f.mbuf0;
  const bool edge = (oy - HX < 0) || (ox - HX < 0) || (oy + TH + HX > ny) || (ox + TW + HX > nx);
  bool bad = false;

  // Stage X0 and M_{k-1} on R6 at clamped coordinates.
  for (int i = tid; i < Reg<6>::N; i += NT) {
    const int ly = i / Reg<6>::W - 6, lx = i % Reg<6>::W - 6;
    const int gy = clampi(oy + ly, 0, ny - 1), gx = clampi(ox + lx, 0, nx - 1);
    sm.X[i] = load_x0(f, gy, gx, bad);
    sm.Mb[i] = (uint8_t)mask_bit(Mp, f.wpr, gy, gx);
  }
  for (int i = tid; i < TH * TW; i += NT) sm.flags[i] = 0;
  if (tid == 0) { sm.n_sp = 0; sm.n_f = 0; sm.n_rep = 0; sm.nlist = 0; sm.nlist2 = 0; }
  if (bad) atomicOr(&f.st->err, ERR_NONFINITE);
  __syncthreads();

  // Step 7 of the previous iteration: I_{k-1} on R4 at flagged pixels (a
  // compacted list; reads touch unflagged pixels only, so it is in place).
  if (k > 1) {
    for (int b = 0; b < Reg<4>::N; b += NT) {
      const int i = b + tid;
      bool p = false;
      int c = 0;
      if (i < Reg<4>::N) {
        const int ly = i / Reg<4>::W - 4, lx = i % Reg<4>::W - 4;
        const int gy = oy + ly, gx = ox + lx;
        c = Reg<6>::idx(ly, lx);
        p = gy >= 0 && gy < ny && gx >= 0 && gx < nx && sm.Mb[c];
      }
      list_append(p, (uint16_t)c, sm.list, &sm.nlist);
    }
    __syncthreads();
    const unsigned n = sm.nlist;
    for (unsigned j = tid; j < n; j += NT) {
      const int c = sm.list[j];
      float v;
      if (!maskmed5(sm.X, sm.Mb, Reg<6>::W, c, v)) {
        const int ly = c / Reg<6>::W - 6, lx = c % Reg<6>::W - 6;
        v = maskmed_wide(f, Mp, oy + ly, ox + lx);
      }
      sm.X[c] = v;
    }
    if (tid == 0) { sm.n_rep = n; sm.nlist = 0; }
    __syncthreads();
    if (edge) {
      edge_fill<4, 6>(sm.X, oy, ox, ny, nx);
      __syncthreads();
    }
  }

  // Steps 1-3 (L+, noise, significance) on R2, and med3(I) on R3.
  for (int i = tid; i < Reg<2>::N; i += NT) {
    const int ly = i / Reg<2>::W - 2, lx = i % Reg<2>::W - 2;
    const int gy = oy + ly, gx = ox + lx;
    if (gy < 0 || gy >= ny || gx < 0 || gx >= nx) continue;
    const int c = Reg<6>::idx(ly, lx);
    constexpr int P = Reg<6>::W;
    const float v = sm.X[c], u = sm.X[c - P], d = sm.X[c + P], l = sm.X[c - 1], r = sm.X[c + 1];
    const float vv = __fadd_rn(v, v);
    float c1 = __fsub_rn(__fsub_rn(vv, u), l);
    float c2 = __fsub_rn(__fsub_rn(vv, u), r);
    float c3 = __fsub_rn(__fsub_rn(vv, d), l);
    float c4 = __fsub_rn(__fsub_rn(vv, d), r);
    c1 = c1 > 0.0f ? c1 : 0.0f;
    c2 = c2 > 0.0f ? c2 : 0.0f;
    c3 = c3 > 0.0f ? c3 : 0.0f;
    c4 = c4 > 0.0f ? c4 : 0.0f;
    const float L = __fmul_rn(__fadd_rn(__fadd_rn(c1, c2), __fadd_rn(c3, c4)), 0.25f);
    const float N = noise_of(f, med5_at(sm.X, P, c));
    sm.S[i] = __fdiv_rn(L, __fadd_rn(N, N));
  }
  for (int i = tid; i < Reg<3>::N; i += NT) {
    const int ly = i / Reg<3>::W - 3, lx = i % Reg<3>::W - 3;
    const int gy = oy + ly, gx = ox + lx;
    if (gy < 0 || gy >= ny || gx < 0 || gx >= nx) continue;
    const int c = Reg<6>::idx(ly, lx);
    float w[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) w[a * 3 + b] = sm.X[c + (a - 1) * Reg<6>::W + (b - 1)];
    float m;
    med3x3<float>(w, &m);
    sm.M3[i] = m;
  }
  __syncthreads();
  if (edge) {
    edge_fill<2, 2>(sm.S, oy, ox, ny, nx);
    edge_fill<3, 3>(sm.M3, oy, ox, ny, nx);
    __syncthreads();
  }

  // S' = S - med5(S), only where S exceeds the lower threshold (elsewhere
  // S' <= S fails every test): compacted list over the tile.
  for (int b = 0; b < TH * TW; b += NT) {
    const int i = b + tid;
    const int ly = i / TW, lx = i % TW;
    const bool p = (oy + ly) < ny && (ox + lx) < nx && sm.S[Reg<2>::idx(ly, lx)] > f.thr_min;
    list_append(p, (uint16_t)i, sm.list, &sm.nlist);
  }
  __syncthreads();
  {
    const unsigned n = sm.nlist;
    for (unsigned j = tid; j < n; j += NT) {
      const int i = sm.list[j];
      const int ly = i / TW, lx = i % TW;
      const int c = Reg<2>::idx(ly, lx);
      const float sp = __fsub_rn(sm.S[c], med5_at(sm.S, Reg<2>::W, c));
      sm.SpL[j] = sp;
      const int c6 = Reg<6>::idx(ly, lx);
      const bool sat = f.satlevel > 0.0f && !sm.Mb[c6] && sm.X[c6] >= f.satlevel;
      const bool sig = !sat && sp > f.sigclip;
      sm.flags[i] = (uint8_t)((sig ? 1 : 0) | ((!sat && sp > f.lo) ? 2 : 0));
    }
    if (tid == 0) sm.n_sp = n;
  }
  __syncthreads();

  // Steps 4-5: the fine-structure test where S' > sigclip (not saturated).
  {
    const unsigned n = sm.nlist;
    for (unsigned b = 0; b < n; b += NT) {
      const unsigned j = b + tid;
      const bool p = j < n && (sm.flags[sm.list[j]] & 1);
      list_append(p, (uint16_t)j, sm.list2, &sm.nlist2);
    }
  }
  __syncthreads();
  {
    const unsigned n = sm.nlist2;
    for (unsigned t = tid; t < n; t += NT) {
      const int j = sm.list2[t];
      const int i = sm.list[j];
      const int ly = i / TW, lx = i % TW;
      const int c3 = Reg<3>::idx(ly, lx);
      float w[49];
#pragma unroll
      for (int a = 0; a < 7; ++a)
#pragma unroll
        for (int b = 0; b < 7; ++b) w[a * 7 + b] = sm.M3[c3 + (a - 3) * Reg<3>::W + (b - 3)];
      float m7;
      med7x7<float>(w, &m7);
      const float diff = __fsub_rn(sm.M3[c3], m7);
      float F = diff;
      if (f.fnorm) F = __fdiv_rn(diff, noise_of(f, med5_at(sm.X, Reg<6>::W, Reg<6>::idx(ly, lx))));
      F = F < 0.01f ? 0.01f : F;
      if (__fdiv_rn(sm.SpL[j], F) > f.objlim) sm.flags[i] |= 4;
    }
    if (tid == 0) sm.n_f = n;
  }
  __syncthreads();

  // Bit-planes of the tile (bits beyond the frame stay 0).
  const int lane = tid & 31, warp = tid >> 5;
  for (int r = warp; r < TH * TWW; r += NT / 32) {
    const int ly = r / TWW, wd = r % TWW;
    const int lx = wd * 32 + lane;
    const int gy = oy + ly;
    const uint8_t fl = ((ox + lx) < nx && gy < ny) ? sm.flags[ly * TW + lx] : 0;
    const unsigned sig = __ballot_sync(0xffffffffu, fl & 1);
    const unsigned lo = __ballot_sync(0xffffffffu, fl & 2);
    const unsigned cand = __ballot_sync(0xffffffffu, fl & 4);
    const int w = (ox >> 5) + wd;
    if (lane == 0 && gy < ny && w < f.wpr) {
      const size_t q = (size_t)gy * f.wpr + w;
      f.p_sig[q] = sig;
      f.p_lo[q] = lo;
      f.p_cand[q] = cand;
    }
  }
  if (tid == 0) {
    if (sm.n_sp) atomicAdd(&f.st->n_sprime, (unsigned long long)sm.n_sp);
    if (sm.n_f) atomicAdd(&f.st->n_fine, (unsigned long long)sm.n_f);
    if (sm.n_rep) atomicAdd(&f.st->n_replace, (unsigned long long)sm.n_rep);
  }
}

__device__ __forceinline__ bool iteration_runs(const FrameDesc& f, int k) {
  if (k > f.niter) return false;
  return k == 1 || *(volatile unsigned long long*)&f.st->fresh[k - 1] != 0;
}

__global__ void __launch_bounds__(NT) core_kernel(const FrameDesc* __restrict__ fr, int nframes,
                                                  unsigned total, int k, unsigned* head) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CoreSmem& sm = *reinterpret_cast<CoreSmem*>(smem_raw);
  __shared__ unsigned s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(head, 1u);
    __syncthreads();
    const unsigned item = s_item;
    __syncthreads();
    if (item >= total) break;
    const FrameDesc& f = fr[frame_of(fr, nframes, item)];
    if (!iteration_runs(f, k)) continue;
    core_tile(f, k, (int)(item - f.tile_begin), sm);
    __syncthreads();
  }
}

// Step 6 on 32-pixel words: one thread per word of M_k.  The horizontal
// 3-dilation of a word takes the edge bits of its neighbours.
__device__ __forceinline__ uint32_t plane_word(const uint32_t* P, int ny, int wpr, int y, int w) {
  if (y < 0 || y >= ny || w < 0 || w >= wpr) return 0u;
  return __ldg(P + (size_t)y * wpr + w);
}

__device__ __forceinline__ uint32_t hdil(uint32_t l, uint32_t c, uint32_t r) {
  return c | (c << 1) | (c >> 1) | (l >> 31) | (r << 31);
}

__global__ void __launch_bounds__(NT) grow_kernel(const FrameDesc* __restrict__ fr, int nframes,
                                                  unsigned long long total_words, int k) {
  const unsigned long long gw = (unsigned long long)blockIdx.x * NT + threadIdx.x;
  unsigned cnt = 0;
  int fi = -1;
  if (gw < total_words) {
    fi = frame_of_word(fr, nframes, gw);
    const FrameDesc& f = fr[fi];
    if (iteration_runs(f, k)) {
      const unsigned long long q = gw - f.word_begin;
      const int y = (int)(q / (unsigned)f.wpr), w = (int)(q % (unsigned)f.wpr);
      const int ny = f.ny, wpr = f.wpr;
      // Dilated candidates on rows y-1..y+1 for words w-1..w+1.
      uint32_t dc[3][3];
      uint32_t cand[5][5];
#pragma unroll
      for (int a = 0; a < 5; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) cand[a][b] = plane_word(f.p_cand, ny, wpr, y - 2 + a, w - 2 + b);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          uint32_t v = 0;
#pragma unroll
          for (int a = 0; a < 3; ++a) v |= hdil(cand[r + a][b], cand[r + a][b + 1], cand[r + a][b + 2]);
          dc[r][b] = v;
        }
      // g1 = dil3(cand) & sig on rows y-1..y+1, words w-1..w+1; the edge words
      // are exact where g2 of word w reads them (their inner edge bit).
      uint32_t g1[3][3];
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int b = 0; b < 3; ++b) g1[r][b] = dc[r][b] & plane_word(f.p_sig, ny, wpr, y - 1 + r, w - 1 + b);
      uint32_t d2 = 0;
#pragma unroll
      for (int r = 0; r < 3; ++r) d2 |= hdil(g1[r][0], g1[r][1], g1[r][2]);
      const uint32_t g2 = d2 & plane_word(f.p_lo, ny, wpr, y, w);
      const uint32_t* Mp = ((k - 1) & 1) ? f.mbuf1 : f.mbuf0;
      uint32_t* Mn = (k & 1) ? f.mbuf1 : f.mbuf0;
      const uint32_t mp = __ldg(Mp + (size_t)y * wpr + w);
      Mn[(size_t)y * wpr + w] = mp | g2;
      cnt = __popc(g2 & ~mp);
    }
  }
  // Per-warp reduction; lanes may belong to different frames at a frame
  // boundary, so each lane with a count adds it (rare) unless the warp agrees.
  const int lane = threadIdx.x & 31;
  const int f0 = __shfl_sync(0xffffffffu, fi, 0);
  const bool same = __all_sync(0xffffffffu, fi == f0);
  if (same) {
    unsigned s = cnt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && s && f0 >= 0) atomicAdd(&fr[f0].st->fresh[k], (unsigned long long)s);
  } else if (cnt) {
    atomicAdd(&fr[fi].st->fresh[k], (unsigned long long)cnt);
  }
}

// Finalize: cleaned = I_{run} (masked median at flagged pixels), mask = M_{run}.
__global__ void __launch_bounds__(NT) finalize_kernel(const FrameDesc* __restrict__ fr, int nframes,
                                                      unsigned total, unsigned* head) {
  __shared__ float X[Reg<2>::N];
  __shared__ uint8_t Mb[Reg<2>::N];
  __shared__ unsigned s_item;
  __shared__ unsigned long long s_cnt;
  const int tid = threadIdx.x;
  for (;;) {
    if (tid == 0) { s_item = atomicAdd(head, 1u); s_cnt = 0; }
    __syncthreads();
    const unsigned item = s_item;
    __syncthreads();
    if (item >= total) break;
    const FrameDesc& f = fr[frame_of(fr, nframes, item)];
    const int tix = (int)(item - f.tile_begin);
    const int oy = (tix / f.tiles_x) * TH, ox = (tix % f.tiles_x) * TW;
    int run = f.niter;
    for (int k = 1; k <= f.niter; ++k)
      if (f.st->fresh[k] == 0) { run = k; break; }
    const uint32_t* M = (run & 1) ? f.mbuf1 : f.mbuf0;
    bool bad = false;
    for (int i = tid; i < Reg<2>::N; i += NT) {
      const int ly = i / Reg<2>::W - 2, lx = i % Reg<2>::W - 2;
      const int gy = clampi(oy + ly, 0, f.ny - 1), gx = clampi(ox + lx, 0, f.nx - 1);
      X[i] = load_x0(f, gy, gx, bad);
      Mb[i] = (uint8_t)mask_bit(M, f.wpr, gy, gx);
    }
    if (bad) atomicOr(&f.st->err, ERR_NONFINITE);
    __syncthreads();
    unsigned long long cnt = 0;
    for (int i = tid; i < TH * TW; i += NT) {
      const int ly = i / TW, lx = i % TW;
      const int gy = oy + ly, gx = ox + lx;
      const bool in = gy < f.ny && gx < f.nx;
      const int c = Reg<2>::idx(ly, lx);
      const bool m = in && Mb[c];
      if (in) {
        float v = X[c];
        if (m && !maskmed5(X, Mb, Reg<2>::W, c, v)) v = maskmed_wide(f, M, gy, gx);
        const size_t q = (size_t)gy * f.nx + gx;
        f.clean_out[q] = v;
        f.mask_out[q] = m ? 1 : 0;
      }
      cnt += __popc(__ballot_sync(0xffffffffu, m));
    }
    if ((tid & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (tid == 0) {
      if (s_cnt) atomicAdd(&f.st->flagged, s_cnt);
      if (tix == 0) f.st->iters_run = run;
    }
    __syncthreads();
  }
}

}  // namespace lacos
