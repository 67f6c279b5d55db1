// Device code of the L.A.Cosmic detect-and-clean iteration (sm_103a).
//
// One iteration k is ONE kernel over a tile work queue.  A CTA takes an
// output tile, stages the original frame X0 and the previous cumulative mask
// M_{k-1} with an 8-pixel halo in shared memory, rebuilds the working image
// I_{k-1} on the fly (unflagged pixels keep X0, flagged pixels take the
// masked median of unflagged X0 -- step 7 of the previous iteration, which
// depends only on X0 and M_{k-1}), then runs steps 1-6 on the tile and
// writes M_k = M_{k-1} | g2 as packed bits.  A finalize kernel writes the
// uint8 mask and the float32 cleaned frame from the last mask.
//
// Regions (relative to the tile): R8 staged X0/M, R6 working image,
// R4 significance S, R2 S'/F/candidates, R1 first growth, R0 output.  Every
// stage evaluates its own array only at in-frame positions and reads out-of-
// frame neighbours at clamped coordinates (clamp-to-edge per stage).
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
constexpr int TW = 32;   // output tile columns (one 32-bit mask word per row)
constexpr int NT = 256;  // threads per CTA
constexpr int HX = 8;    // staging halo

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
  uint8_t* mask_out;
  float* clean_out;
  FrameState* st;
  float gain, rn2, satlevel, sigclip, lo, thr_min, objlim;
  int niter, fnorm;
  int tiles_x;
  unsigned int tile_begin, tile_end;  // this frame's range in the flattened tile list
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

struct TileSmem {
  float X[Reg<8>::N];        // X0, then I_{k-1} on R6
  uint8_t Mb[Reg<8>::N];     // M_{k-1}
  float S[Reg<4>::N];        // S on R4
  float N[Reg<2>::N];        // N on R2
  float Sp[Reg<2>::N];       // S' on R2 (-inf where S <= min threshold)
  uint8_t C[Reg<2>::N];      // candidates on R2
  uint8_t G1[Reg<1>::N];     // first growth on R1
  unsigned long long cnt;
  unsigned n_sp, n_f, n_rep;
};

__device__ __forceinline__ int frame_of(const FrameDesc* fr, int nframes, unsigned item) {
  int lo = 0, hi = nframes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (fr[mid].tile_begin <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ void detect_tile(const FrameDesc& f, int k, int tix, TileSmem& sm) {
  const int tid = threadIdx.x;
  const int oy = (tix / f.tiles_x) * TH;
  const int ox = (tix % f.tiles_x) * TW;
  const int ny = f.ny, nx = f.nx;
  const uint32_t* Mp = ((k - 1) & 1) ? f.mbuf1 : f.mbuf0;
  uint32_t* Mn = (k & 1) ? f.mbuf1 : f.mbuf0;
  const bool edge = (oy - HX < 0) || (ox - HX < 0) || (oy + TH + HX > ny) || (ox + TW + HX > nx);
  bool bad = false;

  // Stage X0 and M_{k-1} on R8 at clamped coordinates.
  for (int i = tid; i < Reg<8>::N; i += NT) {
    const int ly = i / Reg<8>::W - 8, lx = i % Reg<8>::W - 8;
    const int gy = clampi(oy + ly, 0, ny - 1), gx = clampi(ox + lx, 0, nx - 1);
    sm.X[i] = load_x0(f, gy, gx, bad);
    sm.Mb[i] = (uint8_t)mask_bit(Mp, f.wpr, gy, gx);
  }
  if (tid == 0) { sm.cnt = 0; sm.n_sp = 0; sm.n_f = 0; sm.n_rep = 0; }
  if (bad) atomicOr(&f.st->err, ERR_NONFINITE);
  __syncthreads();

  // Step 7 of the previous iteration: I_{k-1} on R6 (flagged pixels only;
  // reads touch unflagged pixels only, writes flagged ones, so in place).
  if (k > 1) {
    for (int i = tid; i < Reg<6>::N; i += NT) {
      const int ly = i / Reg<6>::W - 6, lx = i % Reg<6>::W - 6;
      const int gy = oy + ly, gx = ox + lx;
      if (gy < 0 || gy >= ny || gx < 0 || gx >= nx) continue;
      const int c = Reg<8>::idx(ly, lx);
      if (!sm.Mb[c]) continue;
      float v;
      if (!maskmed5(sm.X, sm.Mb, Reg<8>::W, c, v)) v = maskmed_wide(f, Mp, gy, gx);
      sm.X[c] = v;
      atomicAdd(&sm.n_rep, 1u);
    }
    __syncthreads();
    if (edge) {
      for (int i = tid; i < Reg<6>::N; i += NT) {
        const int ly = i / Reg<6>::W - 6, lx = i % Reg<6>::W - 6;
        const int gy = oy + ly, gx = ox + lx;
        if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) continue;
        sm.X[Reg<8>::idx(ly, lx)] =
            sm.X[Reg<8>::idx(clampi(gy, 0, ny - 1) - oy, clampi(gx, 0, nx - 1) - ox)];
      }
      __syncthreads();
    }
  }

  // Steps 1-3: L+, noise, significance on R4.
  for (int i = tid; i < Reg<4>::N; i += NT) {
    const int ly = i / Reg<4>::W - 4, lx = i % Reg<4>::W - 4;
    const int gy = oy + ly, gx = ox + lx;
    if (gy < 0 || gy >= ny || gx < 0 || gx >= nx) continue;
    const int c = Reg<8>::idx(ly, lx);
    constexpr int P = Reg<8>::W;
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
    float w[25];
#pragma unroll
    for (int a = 0; a < 5; ++a)
#pragma unroll
      for (int b = 0; b < 5; ++b) w[a * 5 + b] = sm.X[c + (a - 2) * P + (b - 2)];
    float m5;
    med5x5<float>(w, &m5);
    const float gm = __fmul_rn(f.gain, m5);
    const float e = gm < 1e-4f ? 1e-4f : gm;
    const float N = __fdiv_rn(__fsqrt_rn(__fadd_rn(e, f.rn2)), f.gain);
    sm.S[i] = __fdiv_rn(L, __fadd_rn(N, N));
    if (ly >= -2 && ly < TH + 2 && lx >= -2 && lx < TW + 2) sm.N[Reg<2>::idx(ly, lx)] = N;
  }
  __syncthreads();
  if (edge) {
    for (int i = tid; i < Reg<4>::N; i += NT) {
      const int ly = i / Reg<4>::W - 4, lx = i % Reg<4>::W - 4;
      const int gy = oy + ly, gx = ox + lx;
      if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) continue;
      sm.S[i] = sm.S[Reg<4>::idx(clampi(gy, 0, ny - 1) - oy, clampi(gx, 0, nx - 1) - ox)];
    }
    __syncthreads();
  }

  // Large-structure removal S' = S - med5(S), only where S exceeds the lower
  // threshold (S' <= S there otherwise, so every test on S' fails anyway).
  for (int i = tid; i < Reg<2>::N; i += NT) {
    const int ly = i / Reg<2>::W - 2, lx = i % Reg<2>::W - 2;
    const int gy = oy + ly, gx = ox + lx;
    float sp = lacos_net::neg_inf<float>();
    if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) {
      const int c = Reg<4>::idx(ly, lx);
      const float s = sm.S[c];
      if (s > f.thr_min) {
        float w[25];
#pragma unroll
        for (int a = 0; a < 5; ++a)
#pragma unroll
          for (int b = 0; b < 5; ++b) w[a * 5 + b] = sm.S[c + (a - 2) * Reg<4>::W + (b - 2)];
        float m;
        med5x5<float>(w, &m);
        sp = __fsub_rn(s, m);
        atomicAdd(&sm.n_sp, 1u);
      }
    }
    sm.Sp[i] = sp;
  }
  __syncthreads();

  // Steps 4-5: candidates (sigclip on S', objlim on S'/F), F only where needed.
  for (int i = tid; i < Reg<2>::N; i += NT) {
    const int ly = i / Reg<2>::W - 2, lx = i % Reg<2>::W - 2;
    const int gy = oy + ly, gx = ox + lx;
    uint8_t cand = 0;
    if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) {
      const int c8 = Reg<8>::idx(ly, lx);
      const bool sat = f.satlevel > 0.0f && !sm.Mb[c8] && sm.X[c8] >= f.satlevel;
      const float sp = sm.Sp[i];
      if (!sat && sp > f.sigclip) {
        // med3 at the 7x7 clamped neighbourhood, then med7 of those.
        float m3w[49];
        float m3p = 0.0f;
        for (int a = 0; a < 7; ++a) {
          const int qy = clampi(gy + a - 3, 0, ny - 1) - oy;
          for (int b = 0; b < 7; ++b) {
            const int qx = clampi(gx + b - 3, 0, nx - 1) - ox;
            const int q = Reg<8>::idx(qy, qx);
            float w[9];
#pragma unroll
            for (int e = 0; e < 3; ++e)
#pragma unroll
              for (int g = 0; g < 3; ++g) w[e * 3 + g] = sm.X[q + (e - 1) * Reg<8>::W + (g - 1)];
            float m;
            med3x3<float>(w, &m);
            m3w[a * 7 + b] = m;
            if (a == 3 && b == 3) m3p = m;
          }
        }
        float m7;
        med7x7<float>(m3w, &m7);
        const float diff = __fsub_rn(m3p, m7);
        float F = f.fnorm ? __fdiv_rn(diff, sm.N[i]) : diff;
        F = F < 0.01f ? 0.01f : F;
        cand = __fdiv_rn(sp, F) > f.objlim ? 1 : 0;
        atomicAdd(&sm.n_f, 1u);
      }
    }
    sm.C[i] = cand;
  }
  __syncthreads();

  // Step 6a: g1 = dil3(cand) & S' > sigclip & !sat on R1.
  for (int i = tid; i < Reg<1>::N; i += NT) {
    const int ly = i / Reg<1>::W - 1, lx = i % Reg<1>::W - 1;
    const int gy = oy + ly, gx = ox + lx;
    uint8_t g = 0;
    if (gy >= 0 && gy < ny && gx >= 0 && gx < nx) {
      const int c2 = Reg<2>::idx(ly, lx);
      const int c8 = Reg<8>::idx(ly, lx);
      const bool sat = f.satlevel > 0.0f && !sm.Mb[c8] && sm.X[c8] >= f.satlevel;
      uint8_t d = 0;
#pragma unroll
      for (int a = -1; a <= 1; ++a)
#pragma unroll
        for (int b = -1; b <= 1; ++b) d |= sm.C[c2 + a * Reg<2>::W + b];  // C = 0 off-frame
      g = (d && sm.Sp[c2] > f.sigclip && !sat) ? 1 : 0;
    }
    sm.G1[i] = g;
  }
  __syncthreads();

  // Step 6b: g2 = dil3(g1) & S' > sigfrac*sigclip & !sat; M_k = M_{k-1} | g2.
  const int lane = tid & 31, warp = tid >> 5;
  unsigned long long fresh = 0;
  for (int ly = warp; ly < TH; ly += NT / 32) {
    const int lx = lane;
    const int gy = oy + ly, gx = ox + lx;
    const bool in = gy < ny && gx < nx;
    const int c8 = Reg<8>::idx(ly, lx);
    bool g2 = false, mprev = false;
    if (in) {
      const int c1 = Reg<1>::idx(ly, lx);
      const int c2 = Reg<2>::idx(ly, lx);
      const bool sat = f.satlevel > 0.0f && !sm.Mb[c8] && sm.X[c8] >= f.satlevel;
      uint8_t d = 0;
#pragma unroll
      for (int a = -1; a <= 1; ++a)
#pragma unroll
        for (int b = -1; b <= 1; ++b) d |= sm.G1[c1 + a * Reg<1>::W + b];
      g2 = d && sm.Sp[c2] > f.lo && !sat;
      mprev = sm.Mb[c8] != 0;
    }
    const unsigned word = __ballot_sync(0xffffffffu, g2 || mprev);
    const unsigned nw = __ballot_sync(0xffffffffu, g2 && !mprev);
    if (lane == 0 && gy < ny) Mn[(size_t)gy * f.wpr + (ox >> 5)] = word;
    fresh += __popc(nw);
  }
  if (lane == 0 && fresh) atomicAdd(&sm.cnt, fresh);
  __syncthreads();
  if (tid == 0) {
    if (sm.cnt) atomicAdd(&f.st->fresh[k], sm.cnt);
    if (sm.n_sp) atomicAdd(&f.st->n_sprime, (unsigned long long)sm.n_sp);
    if (sm.n_f) atomicAdd(&f.st->n_fine, (unsigned long long)sm.n_f);
    if (sm.n_rep) atomicAdd(&f.st->n_replace, (unsigned long long)sm.n_rep);
  }
}

__global__ void __launch_bounds__(NT) detect_kernel(const FrameDesc* __restrict__ fr, int nframes,
                                                    unsigned total, int k, unsigned* head) {
  __shared__ TileSmem sm;
  __shared__ unsigned s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(head, 1u);
    __syncthreads();
    const unsigned item = s_item;
    __syncthreads();
    if (item >= total) break;
    const int fi = frame_of(fr, nframes, item);
    const FrameDesc& f = fr[fi];
    if (k > f.niter) continue;
    if (k > 1 && *(volatile unsigned long long*)&f.st->fresh[k - 1] == 0) continue;
    detect_tile(f, k, (int)(item - f.tile_begin), sm);
    __syncthreads();
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
