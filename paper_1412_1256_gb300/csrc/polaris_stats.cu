// Bit-distribution statistics: per-IF histograms of the b-bit codes of every integrated
// segment (the quantity from which PolariS derives each IF's total power, Sec. 2 and
// Sec. 3.2.2), and the host-side power estimates from such a histogram.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "../../include/polaris.h"
#include "polaris_kernels.cuh"

namespace polaris {

struct HistArgs {
  SegSrc in;
  int nseg;                  // segments [0, nseg) of `in`
  int wps_log2;              // log2 of the 32-bit words per segment (N * bits / 32)
  unsigned long long* hist;  // [n_if][2^bits], accumulated with atomics
  int* err;                  // status word (the bounds-checked build records a bad index)
};

// counts of each code value in one 32-bit word (codes are the word's bits / BITS fields)
template <int BITS>
__device__ __forceinline__ void count_word(uint32_t w, uint32_t (&c)[(BITS <= 4) ? (1 << BITS) : 1],
                                           uint32_t* sh) {
  if constexpr (BITS == 1) {
    const uint32_t ones = __popc(w);
    c[1] += ones;
    c[0] += 32u - ones;
  } else if constexpr (BITS == 2) {
    const uint32_t lo = w & 0x55555555u, hi = (w >> 1) & 0x55555555u;  // bit 0 / bit 1 of each code
    const uint32_t n3 = __popc(lo & hi), n2 = __popc(hi & ~lo), n1 = __popc(lo & ~hi);
    c[3] += n3;
    c[2] += n2;
    c[1] += n1;
    c[0] += 16u - n1 - n2 - n3;
  } else if constexpr (BITS == 4) {
    const uint32_t m = 0x11111111u;
    const uint32_t b0 = w & m, b1 = (w >> 1) & m, b2 = (w >> 2) & m, b3 = (w >> 3) & m;
#pragma unroll
    for (int v = 0; v < 16; ++v) {
      const uint32_t x = ((v & 1) ? b0 : ~b0) & ((v & 2) ? b1 : ~b1) & ((v & 4) ? b2 : ~b2) & ((v & 8) ? b3 : ~b3) & m;
      c[v] += __popc(x);
    }
  } else {
#pragma unroll
    for (int j = 0; j < 4; ++j) atomicAdd(sh + ((w >> (8 * j)) & 0xFFu), 1u);
  }
}

// grid (x: word blocks, y: IF); every word of every segment of the IF once.  Counts are
// summed in registers, then over the block in shared memory, so that each block adds
// one value per code to the global histogram (few, wide blocks per IF: the global
// atomics all hit the same 2^b addresses).
constexpr int kHistThreads = 512, kHistWords = 16;  // words per thread per pass, all loads in flight

template <int BITS>
__global__ void __launch_bounds__(kHistThreads, 2) k_code_hist(HistArgs a) {
  constexpr int NC = 1 << BITS, NR = (BITS <= 4) ? NC : 1, NW = kHistThreads / 32;
  __shared__ uint32_t sh[NC * (BITS == 8 ? 1 : NW)];  // 8-bit: the block's bins; else [warp][code]
  const int ifx = blockIdx.y, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t c[NR];
#pragma unroll
  for (int v = 0; v < NR; ++v) c[v] = 0;
  if constexpr (BITS == 8) {
    for (int v = threadIdx.x; v < NC; v += kHistThreads) sh[v] = 0;
    __syncthreads();
  }
  const long long total = (long long)a.nseg << a.wps_log2;
  const long long wmask = (1LL << a.wps_log2) - 1;
  // this IF's two sources (staged segments [0, n0), then the caller's input)
  const uint32_t* src0 = a.in.src0[ifx];
  const uint32_t* src1 = a.in.src1[ifx];
  const long long hop_w = a.in.hop_w;
  const int n0 = a.in.n0;
  const long long chunk = (long long)kHistThreads * kHistWords;
  for (long long base = (long long)blockIdx.x * chunk; base < total; base += (long long)gridDim.x * chunk) {
    uint32_t w[kHistWords];
#pragma unroll
    for (int j = 0; j < kHistWords; ++j) {  // coalesced: consecutive threads, consecutive words
      const long long k = base + (long long)j * kHistThreads + threadIdx.x;
      w[j] = 0;
      if (k < total) {
        const int s = (int)(k >> a.wps_log2);
        const long long o = (s < n0 ? s * hop_w : (s - n0) * hop_w) + (k & wmask);
        if (in_bounds(a.err, o, s < n0 ? a.in.in_words0 : a.in.in_words1))
          w[j] = __ldg((s < n0 ? src0 : src1) + o);
      }
    }
#pragma unroll
    for (int j = 0; j < kHistWords; ++j) {
      if (base + (long long)j * kHistThreads + threadIdx.x < total) count_word<BITS>(w[j], c, sh);
    }
  }
  unsigned long long* h = a.hist + (size_t)ifx * NC;
  if constexpr (BITS <= 4) {
#pragma unroll
    for (int v = 0; v < NC; ++v) {
      uint32_t x = c[v];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) sh[warp * NC + v] = x;
    }
    __syncthreads();
    for (int v = threadIdx.x; v < NC; v += kHistThreads) {
      unsigned long long t = 0;
      for (int q = 0; q < NW; ++q) t += sh[q * NC + v];
      if (t) atomicAdd(h + v, t);
    }
  } else {
    __syncthreads();
    for (int v = threadIdx.x; v < NC; v += kHistThreads)
      if (sh[v]) atomicAdd(h + v, (unsigned long long)sh[v]);
  }
}

cudaError_t launch_code_hist(const SegSrc& in, int n_if, int bits, int nseg, int64_t n_fft,
                             unsigned long long* hist, int* err, int num_sms, cudaStream_t st) {
  if (nseg <= 0) return cudaSuccess;
  int wl = 0;
  while ((1LL << wl) < n_fft * bits / 32) ++wl;
  HistArgs a;
  a.in = in;
  a.nseg = nseg;
  a.wps_log2 = wl;
  a.hist = hist;
  a.err = err;
  const long long total = (long long)nseg << wl;
  const long long chunk = (long long)kHistThreads * kHistWords;
  long long bx = (total + chunk - 1) / chunk;                 // one pass per block where possible
  const long long cap = (2LL * num_sms + n_if - 1) / n_if;  // at most two blocks per SM over all IFs
  if (bx > cap) bx = cap;
  if (bx < 1) bx = 1;
  const dim3 grid((unsigned)bx, (unsigned)n_if);
  switch (bits) {
    case 1: k_code_hist<1><<<grid, kHistThreads, 0, st>>>(a); break;
    case 2: k_code_hist<2><<<grid, kHistThreads, 0, st>>>(a); break;
    case 4: k_code_hist<4><<<grid, kHistThreads, 0, st>>>(a); break;
    case 8: k_code_hist<8><<<grid, kHistThreads, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// x with erfc(x) = p for p in (0, 1]: Newton steps on erfc, kept inside a shrinking
// bracket [lo, hi] (erfc is decreasing), from the start x = 1
static double erfc_inverse(double p) {
  double lo = 0.0, hi = 30.0, x = 1.0;
  for (int it = 0; it < 200; ++it) {
    const double f = std::erfc(x) - p;
    if (f > 0) lo = x;  // erfc(x) too large: root to the right
    else hi = x;
    const double d = -1.1283791670955126 * std::exp(-x * x);  // d erfc / dx = -2 exp(-x^2) / sqrt(pi)
    double xn = (d != 0.0) ? x - f / d : 0.5 * (lo + hi);
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (std::fabs(xn - x) <= 1e-16 * (1.0 + std::fabs(x))) return xn;
    x = xn;
  }
  return x;
}

}  // namespace polaris

extern "C" int polaris_power_from_histogram(int bits, const uint64_t* counts, double* moment2,
                                            double* sigma_over_threshold) {
  if ((bits != 1 && bits != 2 && bits != 4 && bits != 8) || !counts) return POLARIS_EINVAL;
  const int nc = 1 << bits;
  double total = 0.0, m2 = 0.0;
  for (int c = 0; c < nc; ++c) {
    const double level = bits == 8 ? (double)(int8_t)(uint8_t)c : (double)(2 * c - (nc - 1));
    total += (double)counts[c];
    m2 += level * level * (double)counts[c];
  }
  if (total <= 0.0) return POLARIS_EINVAL;
  if (moment2) *moment2 = m2 / total;
  if (sigma_over_threshold) {
    double sig = std::nan("");
    if (bits == 2) {
      const double p = ((double)counts[0] + (double)counts[3]) / total;  // outer levels -3, +3
      if (p > 0.0 && p < 1.0) sig = 1.0 / (std::sqrt(2.0) * polaris::erfc_inverse(p));
    }
    *sigma_over_threshold = sig;
  }
  return POLARIS_OK;
}
