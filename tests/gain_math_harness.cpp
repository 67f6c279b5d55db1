// Host build of the library's gain arithmetic for the CPU unit test.
#include "../paper_2602_17938_gb300/csrc/gain_math.cuh"

using namespace lacos_gain;

extern "C" {
double h_u128_to_double(unsigned long long hi, unsigned long long lo) {
  return gm_u128_to_double(((u128)hi << 64) | (u128)lo);
}
void h_isqrt(unsigned long long hi, unsigned long long lo, unsigned long long* out_hi,
             unsigned long long* out_lo) {
  const u128 r = gm_isqrt(((u128)hi << 64) | (u128)lo);
  *out_hi = (unsigned long long)(r >> 64);
  *out_lo = (unsigned long long)r;
}
void h_clip_interval(unsigned long long n, long long s1, unsigned long long s2, long long* lo,
                     long long* hi) {
  gm_clip_interval(n, s1, s2, lo, hi);
}
int h_gain(unsigned long long n, long long s1, unsigned long long s2, unsigned long long a, float rn,
           double* g) {
  return gm_gain(n, s1, s2, a, rn, g) ? 1 : 0;
}
}
