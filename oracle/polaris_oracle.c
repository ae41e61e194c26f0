/*
 * FP64 CPU oracle for the PolariS spectrometer hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call
 * this file: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference leg use it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes, in the paper's order (Section 2, Fig. 2 caption; Section 2.1):
 *   1. data translation: b-bit integer codes -> levels           (Fig. 2 caption)
 *   2. segmentation into n_fft-sample segments, hop apart        (Fig. 2 caption; Sec. 3.1)
 *   3. window (rectangular in the paper; Hann / custom taps)     (Sec. 3.1; Sec. 5)
 *   4. FFT of each segment: X_k = sum_n y[n] exp(-2 pi i n k / N), k = 0..N/2
 *   5. power spectra <XX*>, <YY*> and cross spectrum <XY*>,
 *      accumulated over the integration                          (Fig. 1 caption; Table 1)
 *   6. full-Stokes I, Q, U, V by Eq. (2) (linear feeds) and the
 *      circular-feed analogue (our reading, the paper is silent) (Sec. 2.1, Eq. 2)
 *
 * Readings where the paper is silent:
 *   - code -> level: b < 8: level = 2c - (2^b - 1) (odd levels, e.g. 2-bit {-3,-1,1,3});
 *     b = 8: two's-complement int8.  Sample j of a little-endian 32-bit word sits in
 *     bits [j*b, (j+1)*b).
 *   - FFT unnormalised, forward sign e^{-i}; accumulations are sums, not means.
 *   - Hann is the periodic Hann 0.5 - 0.5 cos(2 pi n / N).
 *   - circular feeds: with R_k = (X_k + i Y_k)/sqrt2, L_k = (X_k - i Y_k)/sqrt2,
 *     I = (RR + LL)/2, V = (RR - LL)/2, Q + iU = e^{2 i psi} RL*  — the same
 *     rotation sense as Eq. (2), so a given sky signal gives the same Stokes
 *     through either feed type.
 *
 * Pins for every function live in tests/test_oracle_*.py (brute-force DFT,
 * numpy FFT, Parseval, tone closed forms, polarisation closed forms, radiometer
 * statistics, exhaustive code tables).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

static const double OR_PI = 3.14159265358979323846264338327950288;

/* Step 1: decode one code (Fig. 2 caption: "4 or 8-bit integer to 4-byte float"). */
static double decode_one(int bits, uint32_t code) {
  if (bits == 8) {
    int v = (int)(code & 0xFFu);
    if (v >= 128) v -= 256; /* two's complement */
    return (double)v;
  }
  return 2.0 * (double)code - (double)((1u << bits) - 1u);
}

int oracle_decode(int bits, const uint32_t* words, int64_t n, double* out) {
  if (!(bits == 1 || bits == 2 || bits == 4 || bits == 8) || n < 0 || (n > 0 && (!words || !out))) return OR_EINVAL;
  const int64_t per_word = 32 / bits;
  const uint32_t mask = (1u << bits) - 1u;
  for (int64_t j = 0; j < n; ++j) {
    uint32_t w = words[j / per_word];
    uint32_t c = (w >> ((j % per_word) * bits)) & mask;
    out[j] = decode_one(bits, c);
  }
  return OR_OK;
}

/* Step 3: window taps.  0 = rectangular (the paper's online choice, Sec. 3.1),
 * 1 = periodic Hann, 2 = caller's taps widened from f32. */
int oracle_window(int kind, int64_t n, const float* taps, double* w) {
  if (n <= 0 || !w) return OR_EINVAL;
  for (int64_t i = 0; i < n; ++i) {
    if (kind == 0) w[i] = 1.0;
    else if (kind == 1) w[i] = 0.5 - 0.5 * cos(2.0 * OR_PI * (double)i / (double)n);
    else if (kind == 2) {
      if (!taps) return OR_EINVAL;
      w[i] = (double)taps[i];
    } else return OR_EINVAL;
  }
  return OR_OK;
}

/* Step 4, textbook form: X_k = sum_n x[n] e^{-2 pi i n k / N}, O(N^2). */
int oracle_dft(int64_t n, const double* xr, const double* xi, double* yr, double* yi) {
  if (n <= 0 || !xr || !xi || !yr || !yi) return OR_EINVAL;
  for (int64_t k = 0; k < n; ++k) {
    double sr = 0.0, si = 0.0;
    for (int64_t t = 0; t < n; ++t) {
      /* reduce n*k mod N exactly before forming the angle */
      int64_t m = (t * k) % n;
      double a = -2.0 * OR_PI * (double)m / (double)n;
      double c = cos(a), s = sin(a);
      sr += xr[t] * c - xi[t] * s;
      si += xr[t] * s + xi[t] * c;
    }
    yr[k] = sr;
    yi[k] = si;
  }
  return OR_OK;
}

/* Step 4, fast form: iterative radix-2 decimation-in-time, in place, N a power of two.
 * Twiddles are FP64 cos/sin of -2 pi j / span. */
int oracle_fft(int64_t n, double* re, double* im) {
  if (n <= 0 || (n & (n - 1)) || !re || !im) return OR_EINVAL;
  /* bit-reversal permutation */
  for (int64_t i = 1, j = 0; i < n; ++i) {
    int64_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) {
      double t = re[i]; re[i] = re[j]; re[j] = t;
      t = im[i]; im[i] = im[j]; im[j] = t;
    }
  }
  for (int64_t span = 2; span <= n; span <<= 1) {
    const int64_t half = span >> 1;
    for (int64_t j = 0; j < half; ++j) {
      double a = -2.0 * OR_PI * (double)j / (double)span;
      double wr = cos(a), wi = sin(a);
      for (int64_t s = j; s < n; s += span) {
        int64_t t = s + half;
        double br = re[t] * wr - im[t] * wi;
        double bi = re[t] * wi + im[t] * wr;
        re[t] = re[s] - br;
        im[t] = im[s] - bi;
        re[s] += br;
        im[s] += bi;
      }
    }
  }
  return OR_OK;
}

/* Step 6: Stokes from accumulated spectra.
 *   feed 0 (linear): Eq. (2) written out as the complex 4x4 matrix M times the
 *     gain-corrected correlation vector v = (XX/|Gx|^2, XY/(Gx conj Gy), YX/(Gy conj Gx), YY/|Gy|^2),
 *     where XY = sum X conj(Y) and YX = conj(XY); (I,Q,U,V) = Re(M v)/2.
 *   feed 1 (circular): the reading in the file header, with x = RR, y = LL, c = RL.
 * aa, bb: power spectra of the pair's two IFs; ab: complex cross, re/im interleaved,
 * = sum A conj(B); ga, gb: complex voltage gains (re, im); out: 4 x nbin (I, Q, U, V). */
int oracle_stokes(int feed, double psi, const double* ga, const double* gb, int64_t nbin, const double* aa,
                  const double* bb, const double* ab, double* out) {
  if (nbin <= 0 || !ga || !gb || !aa || !bb || !ab || !out || (feed != 0 && feed != 1)) return OR_EINVAL;
  const double gar = ga[0], gai = ga[1], gbr = gb[0], gbi = gb[1];
  const double gaa = gar * gar + gai * gai, gbb = gbr * gbr + gbi * gbi;
  if (gaa == 0.0 || gbb == 0.0) return OR_EINVAL;
  /* g = Ga conj(Gb) */
  const double g_r = gar * gbr + gai * gbi, g_i = gai * gbr - gar * gbi;
  const double g2 = g_r * g_r + g_i * g_i;
  const double c2 = cos(2.0 * psi), s2 = sin(2.0 * psi);
  /* Eq. (2) matrix, real and imaginary parts */
  const double Mr[4][4] = {{1, 0, 0, 1}, {c2, -s2, -s2, -c2}, {s2, c2, c2, -s2}, {0, 0, 0, 0}};
  const double Mi[4][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}, {0, 0, 0, 0}, {0, -1, 1, 0}};
  for (int64_t k = 0; k < nbin; ++k) {
    const double x = aa[k] / gaa, y = bb[k] / gbb;
    /* c = ab / g */
    const double abr = ab[2 * k], abi = ab[2 * k + 1];
    const double cr = (abr * g_r + abi * g_i) / g2;
    const double ci = (abi * g_r - abr * g_i) / g2;
    double st[4];
    if (feed == 0) {
      const double vr[4] = {x, cr, cr, y};
      const double vi[4] = {0, ci, -ci, 0};
      for (int r = 0; r < 4; ++r) {
        double acc = 0.0; /* real part of row r of M v */
        for (int j = 0; j < 4; ++j) acc += Mr[r][j] * vr[j] - Mi[r][j] * vi[j];
        st[r] = 0.5 * acc;
      }
    } else {
      st[0] = 0.5 * (x + y);
      st[3] = 0.5 * (x - y);
      /* Q + iU = e^{2 i psi} (cr + i ci) */
      st[1] = c2 * cr - s2 * ci;
      st[2] = s2 * cr + c2 * ci;
    }
    out[k] = st[0];
    out[nbin + k] = st[1];
    out[2 * nbin + k] = st[2];
    out[3 * nbin + k] = st[3];
  }
  return OR_OK;
}

/* Steps 2-5 on already-decoded levels (one double array per IF, n_samples each).
 *   segments s = 0,1,.. with s*hop + n_fft <= n_samples (only whole segments).
 *   autos: n_if x (N/2+1); cross: n_pair x (N/2+1) x 2 (re, im), pair p = (pairs[2p], pairs[2p+1]),
 *   cross = sum_s X_a conj(X_b).  n_seg_out: segments per IF. */
int oracle_spectra_levels(int n_if, int64_t n_fft, int64_t hop, int window, const float* taps, int n_pair,
                          const int* pairs, const double* const* levels, int64_t n_samples, double* autos,
                          double* cross, int64_t* n_seg_out) {
  if (n_if < 1 || n_fft < 2 || (n_fft & (n_fft - 1)) || hop < 1 || hop > n_fft || n_samples < 0 || !levels || !autos)
    return OR_EINVAL;
  if (n_pair > 0 && (!pairs || !cross)) return OR_EINVAL;
  for (int p = 0; p < 2 * n_pair; ++p)
    if (pairs[p] < 0 || pairs[p] >= n_if) return OR_EINVAL;
  const int64_t nbin = n_fft / 2 + 1;
  const int64_t n_seg = (n_samples >= n_fft) ? (n_samples - n_fft) / hop + 1 : 0;
  double* w = (double*)malloc(sizeof(double) * n_fft);
  double* re = (double*)malloc(sizeof(double) * n_fft * n_if);
  double* im = (double*)malloc(sizeof(double) * n_fft * n_if);
  if (!w || !re || !im) { free(w); free(re); free(im); return OR_ENOMEM; }
  int rc = oracle_window(window, n_fft, taps, w);
  if (rc != OR_OK) { free(w); free(re); free(im); return rc; }
  memset(autos, 0, sizeof(double) * n_if * nbin);
  if (n_pair > 0) memset(cross, 0, sizeof(double) * 2 * n_pair * nbin);
  for (int64_t s = 0; s < n_seg; ++s) {
    for (int i = 0; i < n_if; ++i) {
      /* steps 2-3: the segment's samples, windowed */
      for (int64_t t = 0; t < n_fft; ++t) {
        re[i * n_fft + t] = w[t] * levels[i][s * hop + t];
        im[i * n_fft + t] = 0.0;
      }
      /* step 4 */
      oracle_fft(n_fft, re + i * n_fft, im + i * n_fft);
      /* step 5: autos */
      for (int64_t k = 0; k < nbin; ++k) {
        double xr = re[i * n_fft + k], xi = im[i * n_fft + k];
        autos[i * nbin + k] += xr * xr + xi * xi;
      }
    }
    /* step 5: crosses X_a conj(X_b) */
    for (int p = 0; p < n_pair; ++p) {
      const int a = pairs[2 * p], b = pairs[2 * p + 1];
      for (int64_t k = 0; k < nbin; ++k) {
        double ar = re[a * n_fft + k], ai = im[a * n_fft + k];
        double br = re[b * n_fft + k], bi = im[b * n_fft + k];
        cross[(p * nbin + k) * 2 + 0] += ar * br + ai * bi;
        cross[(p * nbin + k) * 2 + 1] += ai * br - ar * bi;
      }
    }
  }
  if (n_seg_out) *n_seg_out = n_seg;
  free(w); free(re); free(im);
  return OR_OK;
}

/* Steps 1-5 from packed streams: decode every IF (step 1), then steps 2-5. */
int oracle_accumulate(int n_if, int bits, int64_t n_fft, int64_t hop, int window, const float* taps, int n_pair,
                      const int* pairs, const uint32_t* const* packed, int64_t n_samples, double* autos,
                      double* cross, int64_t* n_seg_out) {
  if (n_if < 1 || !packed || n_samples < 0) return OR_EINVAL;
  double** lev = (double**)calloc((size_t)n_if, sizeof(double*));
  if (!lev) return OR_ENOMEM;
  int rc = OR_OK;
  for (int i = 0; i < n_if && rc == OR_OK; ++i) {
    lev[i] = (double*)malloc(sizeof(double) * (size_t)(n_samples > 0 ? n_samples : 1));
    if (!lev[i]) rc = OR_ENOMEM;
    else rc = oracle_decode(bits, packed[i], n_samples, lev[i]);
  }
  if (rc == OR_OK)
    rc = oracle_spectra_levels(n_if, n_fft, hop, window, taps, n_pair, pairs, (const double* const*)lev, n_samples,
                               autos, cross, n_seg_out);
  for (int i = 0; i < n_if; ++i) free(lev[i]);
  free(lev);
  return rc;
}

/* Bit distribution (Sec. 2: each IF's total power comes from the histogram of its
 * digitised samples; Sec. 3.2.2 tests that measurement's linearity).  counts[i * 2^bits
 * + c] = number of samples with code c among the samples of every whole segment of IF i
 * (segment s = samples [s*hop, s*hop + n_fft)), so a sample in two overlapping segments
 * counts twice.  Plain loop over segments and samples. */
int oracle_code_histogram(int n_if, int bits, int64_t n_fft, int64_t hop, const uint32_t* const* packed,
                          int64_t n_samples, uint64_t* counts) {
  if (n_if < 1 || !(bits == 1 || bits == 2 || bits == 4 || bits == 8) || n_fft < 1 || hop < 1 || !packed ||
      !counts || n_samples < 0)
    return OR_EINVAL;
  const int nc = 1 << bits;
  const int64_t per_word = 32 / bits;
  const uint32_t mask = (uint32_t)nc - 1u;
  memset(counts, 0, sizeof(uint64_t) * (size_t)n_if * (size_t)nc);
  const int64_t n_seg = n_samples >= n_fft ? (n_samples - n_fft) / hop + 1 : 0;
  for (int i = 0; i < n_if; ++i)
    for (int64_t s = 0; s < n_seg; ++s)
      for (int64_t n = s * hop; n < s * hop + n_fft; ++n) {
        const uint32_t code = (packed[i][n / per_word] >> (uint32_t)((n % per_word) * bits)) & mask;
        counts[(size_t)i * nc + code] += 1;
      }
  return OR_OK;
}

/* erfc(x) = p for p in (0, 1]: bisection on [0, 40] (erfc decreasing), to the last bit. */
static double erfc_inverse_bisect(double p) {
  double lo = 0.0, hi = 40.0;
  for (int it = 0; it < 2000 && hi > lo; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (erfc(mid) > p) lo = mid;
    else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Total power from one IF's histogram (our reading of the bit-distribution method):
 *   moment2 = mean of level^2 over the samples (levels as decoded, step 1);
 *   sigma_over_threshold (2-bit): a zero-mean Gaussian of rms sigma falls beyond the
 *   sampler thresholds +-v0 with probability p = erfc(v0 / (sigma sqrt 2)); with p the
 *   fraction of the outer codes (levels -3 and +3), sigma / v0 = 1 / (sqrt2 erfc^-1(p)).
 *   NaN for other widths or p in {0, 1}. */
int oracle_power(int bits, const uint64_t* counts, double* moment2, double* sigma_over_threshold) {
  if (!(bits == 1 || bits == 2 || bits == 4 || bits == 8) || !counts) return OR_EINVAL;
  const int nc = 1 << bits;
  double n = 0.0, sum2 = 0.0;
  for (int c = 0; c < nc; ++c) {
    const double lev = decode_one(bits, (uint32_t)c);
    n += (double)counts[c];
    sum2 += lev * lev * (double)counts[c];
  }
  if (!(n > 0.0)) return OR_EINVAL;
  if (moment2) *moment2 = sum2 / n;
  if (sigma_over_threshold) {
    double sg = NAN;
    if (bits == 2) {
      const double p = ((double)counts[0] + (double)counts[3]) / n;
      if (p > 0.0 && p < 1.0) sg = 1.0 / (sqrt(2.0) * erfc_inverse_bisect(p));
    }
    *sigma_over_threshold = sg;
  }
  return OR_OK;
}

/* ---- Differentiable leakage calibration (our model: the paper treats gains as offline
 * calibration, Sec. 2.1, and is silent on polarisation leakage) ----
 * Two IFs R and L (circular feeds), segments s of n_fft samples at hop n_fft, window w:
 *   X_s[k] = sum_n w[n] x_s[n] e^{-2 pi i n k / N},  Y_s[k] likewise, k = 0..N/2
 *   leakage:  Xt = gR (X + DR[k] Y),   Yt = gL (Y + DL[k] X)
 *   RR = sum_s |Xt|^2,  LL = sum_s |Yt|^2,  RL = sum_s Xt conj(Yt)
 *   I = (RR + LL)/2,  V = (RR - LL)/2,  Q = Re RL,  U = Im RL      (circular feeds, psi = 0)
 *   loss = sum_k sum_{S = I, Q, U, V} (S[k] - T_S[k])^2
 * Layouts: gains = (gR re, gR im, gL re, gL im); leak = DR then DL, each nbin (re, im);
 * target and stokes = I, Q, U, V, each nbin.  Plain loops over segments and bins; each
 * segment's spectra come from oracle_fft of the windowed levels (one IF at a time). */
typedef struct { double re, im; } ocplx;
static ocplx oc(double re, double im) { ocplx z = {re, im}; return z; }
static ocplx oc_add(ocplx a, ocplx b) { return oc(a.re + b.re, a.im + b.im); }
static ocplx oc_mul(ocplx a, ocplx b) { return oc(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re); }
static ocplx oc_conj(ocplx a) { return oc(a.re, -a.im); }
static ocplx oc_scale(ocplx a, double s) { return oc(a.re * s, a.im * s); }

/* spectra X, Y (nbin each) of segment s */
static int leak_segment_spectra(int bits, int64_t N, const uint32_t* const* packed, int64_t s, const double* w,
                                double* lev, double* re, double* im, ocplx* X, ocplx* Y) {
  const int64_t nbin = N / 2 + 1;
  for (int ab = 0; ab < 2; ++ab) {
    /* levels of samples [s N, s N + N): decode from the segment's first word */
    const int64_t per_word = 32 / bits;
    int rc = oracle_decode(bits, packed[ab] + (s * N) / per_word, N, lev);
    if (rc) return rc;
    for (int64_t n = 0; n < N; ++n) { re[n] = w[n] * lev[n]; im[n] = 0.0; }
    rc = oracle_fft(N, re, im);
    if (rc) return rc;
    ocplx* out = ab == 0 ? X : Y;
    for (int64_t k = 0; k < nbin; ++k) out[k] = oc(re[k], im[k]);
  }
  return OR_OK;
}

int oracle_leak_forward(int bits, int64_t N, const uint32_t* const* packed, int64_t n_samples, const double* w,
                        const double* gains, const double* leak, const double* target, double* stokes, double* loss) {
  if (!(bits == 1 || bits == 2 || bits == 4 || bits == 8) || N < 2 || (N & (N - 1)) || N % (32 / bits) || !packed ||
      !w || !gains || !leak || n_samples < N || n_samples % N)
    return OR_EINVAL;
  const int64_t nbin = N / 2 + 1, nseg = n_samples / N;
  double* lev = (double*)malloc(sizeof(double) * (size_t)N);
  double* re = (double*)malloc(sizeof(double) * (size_t)N);
  double* im = (double*)malloc(sizeof(double) * (size_t)N);
  ocplx* X = (ocplx*)malloc(sizeof(ocplx) * (size_t)nbin);
  ocplx* Y = (ocplx*)malloc(sizeof(ocplx) * (size_t)nbin);
  double* acc = (double*)calloc((size_t)(4 * nbin), sizeof(double)); /* RR, LL, RL re, RL im */
  int rc = (lev && re && im && X && Y && acc) ? OR_OK : OR_ENOMEM;
  const ocplx gR = oc(gains[0], gains[1]), gL = oc(gains[2], gains[3]);
  for (int64_t s = 0; s < nseg && rc == OR_OK; ++s) {
    rc = leak_segment_spectra(bits, N, packed, s, w, lev, re, im, X, Y);
    for (int64_t k = 0; k < nbin && rc == OR_OK; ++k) {
      const ocplx DR = oc(leak[2 * k], leak[2 * k + 1]), DL = oc(leak[2 * (nbin + k)], leak[2 * (nbin + k) + 1]);
      const ocplx Xt = oc_mul(gR, oc_add(X[k], oc_mul(DR, Y[k])));
      const ocplx Yt = oc_mul(gL, oc_add(Y[k], oc_mul(DL, X[k])));
      const ocplx rl = oc_mul(Xt, oc_conj(Yt));
      acc[k] += Xt.re * Xt.re + Xt.im * Xt.im;
      acc[nbin + k] += Yt.re * Yt.re + Yt.im * Yt.im;
      acc[2 * nbin + k] += rl.re;
      acc[3 * nbin + k] += rl.im;
    }
  }
  double L = 0.0;
  for (int64_t k = 0; k < nbin && rc == OR_OK; ++k) {
    const double S[4] = {0.5 * (acc[k] + acc[nbin + k]), acc[2 * nbin + k], acc[3 * nbin + k],
                         0.5 * (acc[k] - acc[nbin + k])};
    for (int q = 0; q < 4; ++q) {
      if (stokes) stokes[q * nbin + k] = S[q];
      if (target) {
        const double d = S[q] - target[q * nbin + k];
        L += d * d;
      }
    }
  }
  if (loss && rc == OR_OK) *loss = L;
  free(lev); free(re); free(im); free(X); free(Y); free(acc);
  return rc;
}

/* Gradient of that loss.  With r_S = 2 (S - T_S) per bin, a = (r_I + r_V)/2, b = (r_I - r_V)/2
 * and c = r_Q + i r_U, each segment contributes, per bin,
 *   G_Xt = 2a Xt + c Yt,  G_Yt = 2b Yt + conj(c) Xt          (G = 2 dL/d conj(z): dL = Re sum conj(G) dz)
 *   G_X = conj(gR) G_Xt + conj(gL DL) G_Yt,   G_Y = conj(gR DR) G_Xt + conj(gL) G_Yt
 *   grad gR += conj(X + DR Y) G_Xt,   grad gL += conj(Y + DL X) G_Yt
 *   grad DR[k] += conj(gR Y) G_Xt,    grad DL[k] += conj(gL X) G_Yt
 *   grad w[n] += x[n] Re A_X[n] + y[n] Re A_Y[n],  A = DFT of conj(G) over k = 0..N/2 (zero above)
 * Complex gradients are returned as (d loss / d re, d loss / d im). */
int oracle_leak_grad(int bits, int64_t N, const uint32_t* const* packed, int64_t n_samples, const double* w,
                     const double* gains, const double* leak, const double* target, double* grad_w, double* grad_gains,
                     double* grad_leak) {
  if (!target || !grad_w || !grad_gains || !grad_leak) return OR_EINVAL;
  const int64_t nbin = N / 2 + 1, nseg = n_samples / N;
  double* S = (double*)malloc(sizeof(double) * (size_t)(4 * nbin));
  if (!S) return OR_ENOMEM;
  int rc = oracle_leak_forward(bits, N, packed, n_samples, w, gains, leak, target, S, NULL);
  if (rc) { free(S); return rc; }
  double* lev = (double*)malloc(sizeof(double) * (size_t)N * 2);
  double* re = (double*)malloc(sizeof(double) * (size_t)N);
  double* im = (double*)malloc(sizeof(double) * (size_t)N);
  ocplx* X = (ocplx*)malloc(sizeof(ocplx) * (size_t)nbin);
  ocplx* Y = (ocplx*)malloc(sizeof(ocplx) * (size_t)nbin);
  ocplx* GX = (ocplx*)malloc(sizeof(ocplx) * (size_t)nbin);
  ocplx* GY = (ocplx*)malloc(sizeof(ocplx) * (size_t)nbin);
  rc = (lev && re && im && X && Y && GX && GY) ? OR_OK : OR_ENOMEM;
  for (int64_t n = 0; n < N; ++n) grad_w[n] = 0.0;
  for (int q = 0; q < 4; ++q) grad_gains[q] = 0.0;
  for (int64_t j = 0; j < 4 * nbin; ++j) grad_leak[j] = 0.0;
  const ocplx gR = oc(gains[0], gains[1]), gL = oc(gains[2], gains[3]);
  ocplx ggR = oc(0, 0), ggL = oc(0, 0);
  for (int64_t s = 0; s < nseg && rc == OR_OK; ++s) {
    rc = leak_segment_spectra(bits, N, packed, s, w, lev, re, im, X, Y);
    for (int64_t k = 0; k < nbin && rc == OR_OK; ++k) {
      const double rI = 2.0 * (S[k] - target[k]), rQ = 2.0 * (S[nbin + k] - target[nbin + k]);
      const double rU = 2.0 * (S[2 * nbin + k] - target[2 * nbin + k]), rV = 2.0 * (S[3 * nbin + k] - target[3 * nbin + k]);
      const double a = 0.5 * (rI + rV), b = 0.5 * (rI - rV);
      const ocplx c = oc(rQ, rU);
      const ocplx DR = oc(leak[2 * k], leak[2 * k + 1]), DL = oc(leak[2 * (nbin + k)], leak[2 * (nbin + k) + 1]);
      const ocplx uR = oc_add(X[k], oc_mul(DR, Y[k])), uL = oc_add(Y[k], oc_mul(DL, X[k]));
      const ocplx Xt = oc_mul(gR, uR), Yt = oc_mul(gL, uL);
      const ocplx GXt = oc_add(oc_scale(Xt, 2.0 * a), oc_mul(c, Yt));
      const ocplx GYt = oc_add(oc_scale(Yt, 2.0 * b), oc_mul(oc_conj(c), Xt));
      GX[k] = oc_add(oc_mul(oc_conj(gR), GXt), oc_mul(oc_conj(oc_mul(gL, DL)), GYt));
      GY[k] = oc_add(oc_mul(oc_conj(oc_mul(gR, DR)), GXt), oc_mul(oc_conj(gL), GYt));
      ggR = oc_add(ggR, oc_mul(oc_conj(uR), GXt));
      ggL = oc_add(ggL, oc_mul(oc_conj(uL), GYt));
      const ocplx gDR = oc_mul(oc_conj(oc_mul(gR, Y[k])), GXt), gDL = oc_mul(oc_conj(oc_mul(gL, X[k])), GYt);
      grad_leak[2 * k] += gDR.re;
      grad_leak[2 * k + 1] += gDR.im;
      grad_leak[2 * (nbin + k)] += gDL.re;
      grad_leak[2 * (nbin + k) + 1] += gDL.im;
    }
    /* window: levels of this segment again (x, y), then the DFT of conj(G) */
    const int64_t per_word = 32 / bits;
    if (rc == OR_OK) rc = oracle_decode(bits, packed[0] + (s * N) / per_word, N, lev);
    if (rc == OR_OK) rc = oracle_decode(bits, packed[1] + (s * N) / per_word, N, lev + N);
    for (int ab = 0; ab < 2 && rc == OR_OK; ++ab) {
      const ocplx* G = ab == 0 ? GX : GY;
      for (int64_t k = 0; k < N; ++k) {
        re[k] = k < nbin ? G[k].re : 0.0;
        im[k] = k < nbin ? -G[k].im : 0.0;
      }
      rc = oracle_fft(N, re, im);
      for (int64_t n = 0; n < N && rc == OR_OK; ++n) grad_w[n] += lev[ab * N + n] * re[n];
    }
  }
  grad_gains[0] = ggR.re;
  grad_gains[1] = ggR.im;
  grad_gains[2] = ggL.re;
  grad_gains[3] = ggL.im;
  free(S); free(lev); free(re); free(im); free(X); free(Y); free(GX); free(GY);
  return rc;
}
