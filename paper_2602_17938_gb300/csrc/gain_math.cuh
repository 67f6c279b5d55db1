// Integer and double arithmetic of the per-iteration gain estimate (reading
// C15: photon transfer on adjacent pixel pairs with 3-sigma clipping of their
// differences), shared by the device kernels and a host-compiled unit test.
//
// The pair statistics are exact integers: n pairs, S1 = sum d, S2 = sum d^2
// and A = sum (a + b) for uint16 pairs (a, b), d = a - b.
//  - gm_clip_interval: the integer d with (n d - S1)^2 <= 9 (n S2 - S1^2),
//    i.e. within 3 population standard deviations of the mean, as the
//    interval [lo, hi]: |n d - S1| <= isqrt(9 (n S2 - S1^2)).
//  - gm_gain: the positive root of V g^2 - A g - 2 n rn^2 = 0 with
//    V = (n S2 - S1^2) / n, in double, in the fixed order
//    g = (A + sqrt(A*A + ((8 n) rn^2) V)) / (2 V), every operation rounded to
//    nearest; false when n < 2 or V = 0 (the estimate is undefined).
// Plain C++ when compiled without nvcc (the host test defines nothing else).
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define GM_FN __host__ __device__ __forceinline__
#else
#define GM_FN inline
#endif

#ifdef __CUDA_ARCH__
#define GM_MUL(a, b) __dmul_rn(a, b)
#define GM_ADD(a, b) __dadd_rn(a, b)
#define GM_DIV(a, b) __ddiv_rn(a, b)
#define GM_SQRT(a) __dsqrt_rn(a)
#else
#define GM_MUL(a, b) ((a) * (b))
#define GM_ADD(a, b) ((a) + (b))
#define GM_DIV(a, b) ((a) / (b))
#define GM_SQRT(a) __builtin_sqrt(a)
#endif

namespace lacos_gain {

typedef __int128 i128;
typedef unsigned __int128 u128;

// Bits needed to write v (v > 0).
GM_FN int gm_bitlen(u128 v) {
  int b = 0;
  while (v) {
    v >>= 1;
    ++b;
  }
  return b;
}

// Round-to-nearest-even conversion of 0 <= v < 2^126 to double: values below
// 2^62 convert directly; larger ones are shifted down to 62 significant bits
// with the dropped bits folded into the lowest bit (sticky), which keeps the
// rounding decision of the 53-bit result, and scaled back exactly.
GM_FN double gm_u128_to_double(u128 v) {
  const int b = gm_bitlen(v);
  if (b <= 62) return (double)(long long)v;
  const int s = b - 62;
  const u128 dropped = v & ((((u128)1) << s) - 1);
  const long long top = (long long)(v >> s) | (dropped ? 1 : 0);
  double r = (double)top;
  for (int i = 0; i < s; ++i) r *= 2.0;  // exact: powers of two, far from overflow
  return r;
}

// floor(sqrt(q)) for 0 <= q < 2^100.
GM_FN u128 gm_isqrt(u128 q) {
  if (q == 0) return 0;
  u128 x = (u128)(unsigned long long)GM_SQRT(gm_u128_to_double(q));
  // The double estimate is within 1 of the root for q < 2^100; settle it.
  for (int i = 0; i < 4 && x * x > q; ++i) --x;
  for (int i = 0; i < 4 && (x + 1) * (x + 1) <= q; ++i) ++x;
  return x;
}

GM_FN i128 gm_floordiv(i128 a, i128 b) {  // b > 0
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}

// The clip interval of one round from the statistics of the kept pairs (n >= 1).
GM_FN void gm_clip_interval(unsigned long long n, long long s1, unsigned long long s2, long long* lo,
                            long long* hi) {
  const i128 N = (i128)n, S1 = (i128)s1;
  const i128 q = 9 * (N * (i128)s2 - S1 * S1);
  const i128 R = (i128)gm_isqrt((u128)q);
  i128 l = -gm_floordiv(-(S1 - R), N);  // ceil((S1 - R) / n)
  i128 h = gm_floordiv(S1 + R, N);      // floor((S1 + R) / n)
  // d of uint16 pairs lies in [-65535, 65535]
  if (l < -65536) l = -65536;
  if (h > 65536) h = 65536;
  *lo = (long long)l;
  *hi = (long long)h;
}

// The gain of the final pair set (see the header comment); false when undefined.
GM_FN bool gm_gain(unsigned long long n, long long s1, unsigned long long s2, unsigned long long a,
                   float rn, double* g_out) {
  if (n < 2) return false;
  const i128 vnum = (i128)n * (i128)s2 - (i128)s1 * (i128)s1;
  if (vnum <= 0) return false;
  const double nd = (double)n;  // exact: n < 2^53
  const double V = GM_DIV(gm_u128_to_double((u128)vnum), nd);
  const double A = (double)a;  // exact: a < 2^53
  const double rn2 = GM_MUL((double)rn, (double)rn);
  const double disc = GM_ADD(GM_MUL(A, A), GM_MUL(GM_MUL(GM_MUL(8.0, nd), rn2), V));
  const double g = GM_DIV(GM_ADD(A, GM_SQRT(disc)), GM_MUL(2.0, V));
  if (!(g > 0.0) || !(g < 1.0e300)) return false;
  *g_out = g;
  return true;
}

#undef GM_MUL
#undef GM_ADD
#undef GM_DIV
#undef GM_SQRT

}  // namespace lacos_gain
