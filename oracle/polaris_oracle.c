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
