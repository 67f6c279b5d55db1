// L.A.Cosmic detect-and-clean oracle: plain, slow, single-threaded C++.
//
// TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
// benchmark's CPU-baseline / reference leg may load this library.  The
// product path (the CUDA library and its Python binding) never calls it and
// shares no code, header, table or helper with it.
//
// What it computes: the L.A.Cosmic iteration of van Dokkum (2001), whose
// seven steps dfcosmic lists in its Methods section ("Algorithm": Laplacian
// detection, noise model, significance map, initial candidates, rejection of
// compact objects, neighbour inclusion, median replacement), with the three
// user parameters of "Main parameters" (objlim, sigfrac, sigclip) plus gain
// and read noise.  The paper does not restate the equations; the readings
// taken here (numbered C1..C17) are listed in the design notes and repeated
// next to each step below.
//
// Every function is templated on the working type T (float or double).  For
// T = float every binary operation rounds to float, the file is compiled
// with -ffp-contract=off and without fast-math, so sqrt and '/' are IEEE
// round-to-nearest.  Step order follows the paper's step list.
//
// Parity status: every function is pinned by tests against brute force,
// closed forms, library routines or invariants (see the tests' oracle-pin
// module).  Gain estimation (C15) follows a reading of this library's own
// (the paper prints no formula); it is pinned against scipy's sigma clipping,
// the exact 3-sigma boundary and the gain it recovers from synthetic Poisson
// frames, not against the paper.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

// Clamp-to-edge coordinate (C2: every windowed stage reads its own input
// with coordinates clamped into the frame).
inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Step 1 (Laplacian detection), reading C1: the image is block-replicated
// 2x, convolved with the 3x3 kernel [[0,-1,0],[-1,4,-1],[0,-1,0]], clipped
// at zero and block-averaged 2x2 back to the original grid.  On the
// original grid this is, per pixel with value v and clamped neighbours
// u (up), d (down), l (left), r (right):
//   L = ( (c(u,l) + c(u,r)) + (c(d,l) + c(d,r)) ) * 1/4,
//   c(a,b) = max(0, ((v+v) - a) - b)
// (each sub-pixel of the replicated 2x2 block sees itself twice, one
// vertical and one horizontal neighbour from the adjacent blocks).
template <class T>
void lplus(const T* I, int ny, int nx, T* L) {
  for (int i = 0; i < ny; ++i) {
    for (int j = 0; j < nx; ++j) {
      const T v = I[(size_t)i * nx + j];
      const T u = I[(size_t)clampi(i - 1, 0, ny - 1) * nx + j];
      const T d = I[(size_t)clampi(i + 1, 0, ny - 1) * nx + j];
      const T l = I[(size_t)i * nx + clampi(j - 1, 0, nx - 1)];
      const T r = I[(size_t)i * nx + clampi(j + 1, 0, nx - 1)];
      const T vv = v + v;
      const T c1 = std::max(T(0), (vv - u) - l);
      const T c2 = std::max(T(0), (vv - u) - r);
      const T c3 = std::max(T(0), (vv - d) - l);
      const T c4 = std::max(T(0), (vv - d) - r);
      L[(size_t)i * nx + j] = ((c1 + c2) + (c3 + c4)) * T(0.25);
    }
  }
}

// The literal form of step 1 (C1), kept as a second route: replicate 2x,
// convolve (clamped edges on the replicated grid), clip, block-average.
template <class T>
void lplus_literal(const T* I, int ny, int nx, T* L) {
  const int Y = 2 * ny, X = 2 * nx;
  std::vector<T> R((size_t)Y * X), C((size_t)Y * X);
  for (int i = 0; i < Y; ++i)
    for (int j = 0; j < X; ++j) R[(size_t)i * X + j] = I[(size_t)(i / 2) * nx + (j / 2)];
  for (int i = 0; i < Y; ++i) {
    for (int j = 0; j < X; ++j) {
      const T v = R[(size_t)i * X + j];
      const T u = R[(size_t)clampi(i - 1, 0, Y - 1) * X + j];
      const T d = R[(size_t)clampi(i + 1, 0, Y - 1) * X + j];
      const T l = R[(size_t)i * X + clampi(j - 1, 0, X - 1)];
      const T r = R[(size_t)i * X + clampi(j + 1, 0, X - 1)];
      const T c = (v + v + v + v) - u - d - l - r;
      C[(size_t)i * X + j] = std::max(T(0), c);
    }
  }
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      const T s = (C[(size_t)(2 * i) * X + 2 * j] + C[(size_t)(2 * i) * X + 2 * j + 1]) +
                  (C[(size_t)(2 * i + 1) * X + 2 * j] + C[(size_t)(2 * i + 1) * X + 2 * j + 1]);
      L[(size_t)i * nx + j] = s * T(0.25);
    }
}

// True (non-separable) K x K median (C3): the element of rank (K*K-1)/2 in
// ascending order of the clamped window.  Used for med3, med5 and med7.
template <class T>
void median_filter(const T* A, int ny, int nx, int K, T* out) {
  const int r = K / 2;
  std::vector<T> w((size_t)K * K);
  for (int i = 0; i < ny; ++i) {
    for (int j = 0; j < nx; ++j) {
      size_t n = 0;
      for (int di = -r; di <= r; ++di)
        for (int dj = -r; dj <= r; ++dj)
          w[n++] = A[(size_t)clampi(i + di, 0, ny - 1) * nx + clampi(j + dj, 0, nx - 1)];
      std::nth_element(w.begin(), w.begin() + (n - 1) / 2, w.begin() + n);
      out[(size_t)i * nx + j] = w[(n - 1) / 2];
    }
  }
}

// Reading C17 (the comparison mode): the separable K x K median -- the
// median over the K rows of the window of each row's K-tap median, with the
// same clamped coordinates as median_filter.  The paper notes that
// implementations using it for speed misclassify the centres of bright or
// saturated stars as cosmic rays; this mode exists to show that, and is not
// the method itself.
template <class T>
void median_filter_sep(const T* A, int ny, int nx, int K, T* out) {
  const int r = K / 2;
  std::vector<T> row((size_t)K), meds((size_t)K);
  for (int i = 0; i < ny; ++i) {
    for (int j = 0; j < nx; ++j) {
      for (int di = -r; di <= r; ++di) {
        for (int dj = -r; dj <= r; ++dj)
          row[dj + r] = A[(size_t)clampi(i + di, 0, ny - 1) * nx + clampi(j + dj, 0, nx - 1)];
        std::nth_element(row.begin(), row.begin() + r, row.end());
        meds[di + r] = row[r];
      }
      std::nth_element(meds.begin(), meds.begin() + r, meds.end());
      out[(size_t)i * nx + j] = meds[r];
    }
  }
}

// 3x3 binary dilation; out-of-frame positions count as false.
void dilate3(const uint8_t* in, int ny, int nx, uint8_t* out) {
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      uint8_t v = 0;
      for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
          const int y = i + di, x = j + dj;
          if (y >= 0 && y < ny && x >= 0 && x < nx && in[(size_t)y * nx + x]) v = 1;
        }
      out[(size_t)i * nx + j] = v;
    }
}

// Step 7 (replacement), reading C11: the lower median (rank (n-1)/2) of the
// ORIGINAL values X0 at the unflagged positions of the clamped 5x5 window,
// positions counted with multiplicity.  If none is unflagged, widen to 7x7,
// 9x9, ... .  Returns false only if no unflagged pixel exists in the frame.
template <class T>
bool maskmed(const T* X0, const uint8_t* M, int ny, int nx, int i, int j, T* out) {
  std::vector<T> pool;
  const int rmax = std::max(ny, nx) + 2;
  for (int r = 2; r <= rmax; ++r) {
    pool.clear();
    for (int di = -r; di <= r; ++di)
      for (int dj = -r; dj <= r; ++dj) {
        const size_t q = (size_t)clampi(i + di, 0, ny - 1) * nx + clampi(j + dj, 0, nx - 1);
        if (!M[q]) pool.push_back(X0[q]);
      }
    if (!pool.empty()) {
      std::sort(pool.begin(), pool.end());
      *out = pool[(pool.size() - 1) / 2];
      return true;
    }
  }
  return false;
}

template <class T>
struct Params {
  T gain, readnoise, satlevel, sigclip, sigfrac, objlim;
  int niter;
  int fnorm;    // 1: F = max((m3-m7)/N, 0.01) (reading C6); 0: F = max(m3-m7, 0.01)
  int satgrow;  // reading C16: radius of the protected region around saturated pixels (0..4)
  int sepmed;   // reading C17: 1 takes both 5x5 detection medians separably (comparison mode)
};

// Reading C16 (saturated-star protection, the paper's concern that centres
// of (near-)saturated stars get taken for cosmic rays): the saturated set is
// grown by the square of radius r (all pixels within Chebyshev distance r,
// inside the frame), and every use of "saturated" -- never a candidate,
// never grown into, so never replaced -- uses the grown set.  r = 0 leaves
// reading C9 unchanged.
void dilate_square(const uint8_t* in, int ny, int nx, int r, uint8_t* out) {
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      uint8_t v = 0;
      for (int a = std::max(0, i - r); a <= std::min(ny - 1, i + r) && !v; ++a)
        for (int b = std::max(0, j - r); b <= std::min(nx - 1, j + r); ++b)
          if (in[(size_t)a * nx + b]) { v = 1; break; }
      out[(size_t)i * nx + j] = v;
    }
}

// Ingest (a0): convert to T, canonicalise -0 to +0, reject non-finite input,
// and mark saturated pixels (C9: original input >= satlevel, satlevel > 0).
template <class T>
int ingest(const void* frame, int dtype, size_t n, T satlevel, std::vector<T>& X0,
           std::vector<uint8_t>& sat) {
  X0.resize(n);
  sat.assign(n, 0);
  for (size_t p = 0; p < n; ++p) {
    T v;
    if (dtype == 1) {
      v = (T)((const uint16_t*)frame)[p];
    } else {
      const float f = ((const float*)frame)[p];
      if (!std::isfinite(f)) return -5;
      v = (T)f;
    }
    if (v == T(0)) v = T(0);  // -0 -> +0
    X0[p] = v;
    if (satlevel > T(0) && v >= satlevel) sat[p] = 1;
  }
  return 0;
}

// Intermediates of one iteration (any pointer may be null).
template <class T>
struct Dumps {
  T *L, *m5, *N, *S, *mS, *Sp, *m3, *m7, *F;
  uint8_t *cand, *g1, *g2;
};

// One iteration k: steps 1-7 on the working image I (in/out) and the
// cumulative mask M (in/out).  Returns the number of newly flagged pixels.
template <class T>
long long iterate(const T* X0, const uint8_t* sat, int ny, int nx, const Params<T>& p,
                  T* I, uint8_t* M, const Dumps<T>* dump) {
  const size_t n = (size_t)ny * nx;
  std::vector<T> L(n), m5(n), N(n), S(n), mS(n), Sp(n), m3(n), m7(n), F(n);
  std::vector<uint8_t> cand(n), d1(n), g1(n), d2(n), g2(n);
  const T g = p.gain;
  const T rn2 = p.readnoise * p.readnoise;

  // Step 1: Laplacian detection (C1).
  lplus(I, ny, nx, L.data());
  // Step 2: noise model N = sqrt(max(g*med5(I), 1e-4) + rn^2) / g (C4), in ADU.
  (p.sepmed ? median_filter_sep<T> : median_filter<T>)(I, ny, nx, 5, m5.data());
  for (size_t q = 0; q < n; ++q) {
    const T e = std::max(g * m5[q], T(1e-4));
    N[q] = std::sqrt(e + rn2) / g;
  }
  // Step 3: significance map S = L / (2N) (C5), then large-structure removal
  // S' = S - med5(S).
  for (size_t q = 0; q < n; ++q) S[q] = L[q] / (N[q] + N[q]);
  (p.sepmed ? median_filter_sep<T> : median_filter<T>)(S.data(), ny, nx, 5, mS.data());
  for (size_t q = 0; q < n; ++q) Sp[q] = S[q] - mS[q];
  // Step 5 input: fine-structure image F = max((med3(I) - med7(med3(I))) / N, 0.01) (C6).
  median_filter(I, ny, nx, 3, m3.data());
  median_filter(m3.data(), ny, nx, 7, m7.data());
  for (size_t q = 0; q < n; ++q) {
    const T diff = m3[q] - m7[q];
    F[q] = p.fnorm ? std::max(diff / N[q], T(0.01)) : std::max(diff, T(0.01));
  }
  // Steps 4-5: candidates pass sigclip on S' and objlim on S'/F (C7, C8, C9).
  for (size_t q = 0; q < n; ++q)
    cand[q] = (!sat[q] && Sp[q] > p.sigclip && (Sp[q] / F[q]) > p.objlim) ? 1 : 0;
  // Step 6: neighbour growth with the sigclip and sigfrac*sigclip re-tests (C10).
  const T lo = p.sigfrac * p.sigclip;
  dilate3(cand.data(), ny, nx, d1.data());
  for (size_t q = 0; q < n; ++q) g1[q] = (d1[q] && Sp[q] > p.sigclip && !sat[q]) ? 1 : 0;
  dilate3(g1.data(), ny, nx, d2.data());
  for (size_t q = 0; q < n; ++q) g2[q] = (d2[q] && Sp[q] > lo && !sat[q]) ? 1 : 0;
  long long fresh = 0;
  for (size_t q = 0; q < n; ++q) {
    if (g2[q] && !M[q]) ++fresh;
    if (g2[q]) M[q] = 1;
  }
  // Step 7: replace every flagged pixel by the masked median of unflagged
  // original values (C11).  Unflagged pixels keep X0.
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j < nx; ++j) {
      const size_t q = (size_t)i * nx + j;
      if (M[q]) {
        T v;
        if (maskmed(X0, M, ny, nx, i, j, &v)) I[q] = v;
      }
    }
  if (dump) {
    auto cp = [n](T* dst, const std::vector<T>& src) {
      if (dst) std::memcpy(dst, src.data(), n * sizeof(T));
    };
    auto cpb = [n](uint8_t* dst, const std::vector<uint8_t>& src) {
      if (dst) std::memcpy(dst, src.data(), n);
    };
    cp(dump->L, L); cp(dump->m5, m5); cp(dump->N, N); cp(dump->S, S); cp(dump->mS, mS);
    cp(dump->Sp, Sp); cp(dump->m3, m3); cp(dump->m7, m7); cp(dump->F, F);
    cpb(dump->cand, cand); cpb(dump->g1, g1); cpb(dump->g2, g2);
  }
  return fresh;
}

// Reading C15 (gain estimation; "Main parameters": a gain that is not
// supplied is estimated at each iteration, with sigma-clipped statistics --
// the paper names its sigma-clipping helper but prints no formula).  Photon
// transfer on adjacent pixel pairs of the iteration's image I:
//  - pairs: columns (2m, 2m+1) of every row, both pixels unflagged in M and
//    not saturated, so both hold input values; d = a - b;
//  - clipping: the pair set K_0 holds every such pair; K_(r+1) keeps the pairs
//    of K_r whose d lies within 3 population standard deviations of K_r's
//    mean, (n d - S1)^2 <= 9 (n S2 - S1^2) with n = |K_r|, S1 = sum d,
//    S2 = sum d^2, evaluated exactly in integers; at most 5 such rounds,
//    stopping once a round keeps every pair (astropy's sigma_clip defaults,
//    with the mean as centre);
//  - gain: for a pair of means mu_a, mu_b (ADU), var(d) = (mu_a + mu_b)/g +
//    2 rn^2/g^2 (Poisson electrons plus read noise, in ADU), so over the
//    final set V g^2 - A g - 2 n rn^2 = 0 with V = sum (d - mean d)^2 =
//    (n S2 - S1^2)/n and A = sum (a + b); g is the positive root
//    (A + sqrt(A^2 + 8 n rn^2 V)) / (2 V), in double in exactly this order.
// The sums are exact only for integer values, so the estimate is defined
// for uint16 frames (whose image stays integer: replacements copy input
// values).  With no pair, or V = 0, the estimate is undefined; the
// iteration then uses g = 1 and the run reports it.
struct GainStats {
  long long n = 0, s1 = 0;
  unsigned long long s2 = 0, a = 0;
};

template <class T>
int estimate_gain(const T* I, const uint8_t* M, const uint8_t* sat, int ny, int nx, double rn,
                  double* g_out, int* rounds_out, GainStats* final_out) {
  struct Pair { long long a, b; };
  std::vector<Pair> pairs;
  for (int i = 0; i < ny; ++i)
    for (int j = 0; j + 1 < nx; j += 2) {
      const size_t q = (size_t)i * nx + j;
      if (M[q] || M[q + 1] || sat[q] || sat[q + 1]) continue;
      const T va = I[q], vb = I[q + 1];
      if (!(va >= T(0) && va <= T(65535) && va == std::floor(va))) return -1;
      if (!(vb >= T(0) && vb <= T(65535) && vb == std::floor(vb))) return -1;
      pairs.push_back({(long long)va, (long long)vb});
    }
  std::vector<uint8_t> kept(pairs.size(), 1);
  GainStats st, prev;
  int r = 0;
  for (r = 0;; ++r) {
    st = GainStats{};
    for (size_t t = 0; t < pairs.size(); ++t) {
      if (!kept[t]) continue;
      const long long d = pairs[t].a - pairs[t].b;
      st.n += 1;
      st.s1 += d;
      st.s2 += (unsigned long long)(d * d);
      st.a += (unsigned long long)(pairs[t].a + pairs[t].b);
    }
    if (st.n == 0 || r == 5 || (r > 0 && st.n == prev.n)) break;
    const __int128 n = st.n, s1 = st.s1, s2 = (__int128)st.s2;
    const __int128 bound = 9 * (n * s2 - s1 * s1);
    for (size_t t = 0; t < pairs.size(); ++t) {
      if (!kept[t]) continue;
      const __int128 e = n * (__int128)(pairs[t].a - pairs[t].b) - s1;
      if (e * e > bound) kept[t] = 0;
    }
    prev = st;
  }
  if (rounds_out) *rounds_out = r;
  if (final_out) *final_out = st;
  if (st.n < 2) return 0;
  const __int128 vnum = (__int128)st.n * (__int128)st.s2 - (__int128)st.s1 * (__int128)st.s1;
  if (vnum <= 0) return 0;
  const double nd = (double)st.n;
  const double V = (double)vnum / nd;
  const double A = (double)st.a;
  const double rn2 = rn * rn;
  const double disc = A * A + 8.0 * nd * rn2 * V;
  const double g = (A + std::sqrt(disc)) / (2.0 * V);
  if (!(g > 0) || !std::isfinite(g)) return 0;
  *g_out = g;
  return 1;
}

bool params_ok(double gain, double rn, double sigclip, double sigfrac, double objlim, int niter) {
  if (!(gain >= 0) || !(rn >= 0) || !(sigclip > 0) || !(sigfrac > 0) || !(objlim > 0)) return false;
  if (niter < 0) return false;
  return std::isfinite(gain) && std::isfinite(rn) && std::isfinite(sigclip) &&
         std::isfinite(sigfrac) && std::isfinite(objlim);
}

// The whole detect-and-clean loop (step a9): repeat until niter iterations
// or no new pixel (C13).  Output mask is cumulative; cleaned = I.
// gain = 0 estimates the gain at every iteration (C15, uint16 frames only);
// *gain_last receives the gain of the last iteration run (the supplied one
// when gain > 0) and *gain_ok 0 when some iteration's estimate was undefined.
template <class T>
int run(const void* frame, int dtype, int ny, int nx, const Params<T>& p, uint8_t* mask_out,
        T* clean_out, int* iters_run, long long* n_flagged, double* gain_last, int* gain_ok) {
  if (!frame || ny < 1 || nx < 1 || (dtype != 0 && dtype != 1)) return -1;
  if (!params_ok(p.gain, p.readnoise, p.sigclip, p.sigfrac, p.objlim, p.niter)) return -1;
  const bool estimate = p.gain == T(0);
  if (estimate && dtype != 1) return -1;
  if (p.satgrow < 0 || p.satgrow > 4 || (p.sepmed != 0 && p.sepmed != 1)) return -1;
  const size_t n = (size_t)ny * nx;
  std::vector<T> X0;
  std::vector<uint8_t> sat;
  const int rc = ingest(frame, dtype, n, p.satlevel, X0, sat);
  if (rc) return rc;
  if (p.satgrow > 0) {
    std::vector<uint8_t> grown(n);
    dilate_square(sat.data(), ny, nx, p.satgrow, grown.data());
    sat.swap(grown);
  }
  std::vector<T> I(X0);
  std::vector<uint8_t> M(n, 0);
  Params<T> pk = p;
  int ok = 1;
  int k = 0;
  for (k = 1; k <= p.niter; ++k) {
    if (estimate) {  // C15: the gain of iteration k from I_k and M_(k-1)
      double g = 0.0;
      const int e = estimate_gain(I.data(), M.data(), sat.data(), ny, nx, (double)p.readnoise, &g,
                                  nullptr, nullptr);
      if (e < 0) return -1;
      if (e == 0) ok = 0;
      pk.gain = e == 1 ? (T)g : T(1);
    }
    const long long fresh = iterate(X0.data(), sat.data(), ny, nx, pk, I.data(), M.data(),
                                    (const Dumps<T>*)nullptr);
    if (fresh == 0) break;
  }
  if (gain_last) *gain_last = (double)pk.gain;
  if (gain_ok) *gain_ok = ok;
  if (k > p.niter) k = p.niter;
  long long cnt = 0;
  for (size_t q = 0; q < n; ++q) {
    mask_out[q] = M[q];
    cnt += M[q];
    clean_out[q] = I[q];
  }
  if (iters_run) *iters_run = k;
  if (n_flagged) *n_flagged = cnt;
  return 0;
}

template <class T>
Params<T> make_params(double gain, double rn, double satlevel, double sigclip, double sigfrac,
                      double objlim, int niter, int fnorm, int satgrow, int sepmed) {
  Params<T> p;
  p.gain = (T)gain; p.readnoise = (T)rn; p.satlevel = (T)satlevel;
  p.sigclip = (T)sigclip; p.sigfrac = (T)sigfrac; p.objlim = (T)objlim;
  p.niter = niter; p.fnorm = fnorm; p.satgrow = satgrow; p.sepmed = sepmed;
  return p;
}

}  // namespace

// ---------------------------------------------------------------------------
// C entry points (loaded by the tests through ctypes).  Parameters arrive as
// float (the library's own parameter type) and are widened exactly to T.
// dtype: 0 = float32 frame, 1 = uint16 frame.  Return 0 on success, -1 for
// invalid arguments, -5 for non-finite input.
extern "C" {

int oracle_run_f32(const void* frame, int dtype, int ny, int nx, float gain, float rn,
                   float satlevel, float sigclip, float sigfrac, float objlim, int niter,
                   int fnorm, int satgrow, int sepmed, uint8_t* mask, float* clean, int* iters_run,
                   long long* n_flagged, double* gain_last, int* gain_ok) {
  return run<float>(frame, dtype, ny, nx,
                    make_params<float>(gain, rn, satlevel, sigclip, sigfrac, objlim, niter, fnorm, satgrow,
                                       sepmed),
                    mask, clean, iters_run, n_flagged, gain_last, gain_ok);
}

int oracle_run_f64(const void* frame, int dtype, int ny, int nx, float gain, float rn,
                   float satlevel, float sigclip, float sigfrac, float objlim, int niter,
                   int fnorm, int satgrow, int sepmed, uint8_t* mask, double* clean, int* iters_run,
                   long long* n_flagged, double* gain_last, int* gain_ok) {
  return run<double>(frame, dtype, ny, nx,
                     make_params<double>(gain, rn, satlevel, sigclip, sigfrac, objlim, niter, fnorm, satgrow,
                                         sepmed),
                     mask, clean, iters_run, n_flagged, gain_last, gain_ok);
}

// C15 on one image: I (float or double values), M and sat 0/1 per pixel.
// Returns 1 with *g set, 0 when undefined, -1 for a non-integer value in a
// pair.  stats receives n, sum d, sum d^2 and sum (a + b) of the final set.
#define ORACLE_GAIN(SUF, T)                                                                    \
  int oracle_estimate_gain_##SUF(const T* I, const uint8_t* M, const uint8_t* sat, int ny,     \
                                 int nx, float rn, double* g, int* rounds, long long* stats) { \
    GainStats st;                                                                             \
    const int e = estimate_gain<T>(I, M, sat, ny, nx, (double)rn, g, rounds, &st);             \
    if (stats) {                                                                              \
      stats[0] = st.n;                                                                        \
      stats[1] = st.s1;                                                                       \
      stats[2] = (long long)st.s2;                                                            \
      stats[3] = (long long)st.a;                                                             \
    }                                                                                         \
    return e;                                                                                 \
  }
ORACLE_GAIN(f32, float)
ORACLE_GAIN(f64, double)

// One iteration with every intermediate exposed.  X0 and I are in T; sat is
// 0/1 per pixel.  I and M are updated in place.  Returns the new-pixel count.
#define ORACLE_ITER(SUF, T)                                                                       \
  long long oracle_iterate_##SUF(const T* X0, const uint8_t* sat, int ny, int nx, float gain,    \
                                 float rn, float sigclip, float sigfrac, float objlim, int fnorm, \
                                 T* I, uint8_t* M, T* L, T* m5, T* N, T* S, T* mS, T* Sp, T* m3,  \
                                 T* m7, T* F, uint8_t* cand, uint8_t* g1, uint8_t* g2) {         \
    Params<T> p = make_params<T>(gain, rn, 0.0, sigclip, sigfrac, objlim, 1, fnorm, 0, 0);       \
    Dumps<T> d{L, m5, N, S, mS, Sp, m3, m7, F, cand, g1, g2};                                     \
    return iterate<T>(X0, sat, ny, nx, p, I, M, &d);                                              \
  }
ORACLE_ITER(f32, float)
ORACLE_ITER(f64, double)

void oracle_lplus_f32(const float* I, int ny, int nx, float* L) { lplus(I, ny, nx, L); }
void oracle_lplus_f64(const double* I, int ny, int nx, double* L) { lplus(I, ny, nx, L); }
void oracle_lplus_literal_f32(const float* I, int ny, int nx, float* L) {
  lplus_literal(I, ny, nx, L);
}
void oracle_lplus_literal_f64(const double* I, int ny, int nx, double* L) {
  lplus_literal(I, ny, nx, L);
}
void oracle_median_f32(const float* A, int ny, int nx, int K, float* out) {
  median_filter(A, ny, nx, K, out);
}
void oracle_median_f64(const double* A, int ny, int nx, int K, double* out) {
  median_filter(A, ny, nx, K, out);
}
void oracle_median_sep_f32(const float* A, int ny, int nx, int K, float* out) {
  median_filter_sep(A, ny, nx, K, out);
}
void oracle_median_sep_f64(const double* A, int ny, int nx, int K, double* out) {
  median_filter_sep(A, ny, nx, K, out);
}
void oracle_dilate3(const uint8_t* in, int ny, int nx, uint8_t* out) { dilate3(in, ny, nx, out); }
void oracle_dilate_square(const uint8_t* in, int ny, int nx, int r, uint8_t* out) {
  dilate_square(in, ny, nx, r, out);
}
int oracle_maskmed_f32(const float* X0, const uint8_t* M, int ny, int nx, int i, int j,
                       float* out) {
  return maskmed(X0, M, ny, nx, i, j, out) ? 0 : 1;
}
int oracle_maskmed_f64(const double* X0, const uint8_t* M, int ny, int nx, int i, int j,
                       double* out) {
  return maskmed(X0, M, ny, nx, i, j, out) ? 0 : 1;
}

}  // extern "C"
