// Device building blocks of the PolariS hot path for sm_103a:
//   * compile-time twiddles (own octant-reduced Taylor series, FP64, rounded once to f32)
//   * in-register radix-2 DIT transforms with the twiddle folded into the butterfly
//     FMAs (cosine-factored form: a +- W b = a +- wr (b + (wi/wr) i b), three packed
//     two-wide FMAs)
//   * the data-translation step (b-bit code -> float level, exact, no I2F)
//   * the per-size two-phase plan N = N1 * N2.
//
// The transform is the segment FFT of the paper (Fig. 2 caption: "FFT"), unnormalised,
// forward sign e^{-i}.  Two real IF streams x, y of a pair are transformed together as
// z = x + i y (one complex FFT of N points per pair-segment).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>

namespace polaris {

// ----------------------------------------------------------------------------------------
// compile-time trigonometry
// ----------------------------------------------------------------------------------------
namespace ct {
constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double sin_small(double x) {  // |x| <= pi/4; Taylor series, error << 1e-17
  double x2 = x * x, t = x, s = x;
  for (int n = 1; n <= 13; ++n) {
    t *= -x2 / (double)((2 * n) * (2 * n + 1));
    s += t;
  }
  return s;
}
constexpr double cos_small(double x) {
  double x2 = x * x, t = 1.0, s = 1.0;
  for (int n = 1; n <= 13; ++n) {
    t *= -x2 / (double)((2 * n - 1) * (2 * n));
    s += t;
  }
  return s;
}
struct CS {
  double c, s;
};
// (cos, sin) of 2 pi k / L with exact integer octant reduction.
constexpr CS cossin2pi(long k, long L) {
  k %= L;
  if (k < 0) k += L;
  const long e = 8 * k;       // angle = (pi/4) * e / L
  const long o = e / L;       // octant 0..7
  const long r = e - o * L;   // remainder in [0, L)
  const long q = o / 2;       // quadrant
  const long num = (o % 2) * L + r;  // angle inside the quadrant = (pi/4) num / L, num in [0, 2L)
  double ca = 0, sa = 0;
  if (num <= L) {
    const double a = (kPi / 4.0) * ((double)num / (double)L);
    ca = cos_small(a);
    sa = sin_small(a);
  } else {
    const double b = (kPi / 4.0) * ((double)(2 * L - num) / (double)L);
    ca = sin_small(b);
    sa = cos_small(b);
  }
  if (q == 0) return CS{ca, sa};
  if (q == 1) return CS{-sa, ca};
  if (q == 2) return CS{-ca, -sa};
  return CS{sa, -ca};
}
constexpr double dabs(double v) { return v < 0 ? -v : v; }
constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }
constexpr int bitrev(int i, int L) {
  int r = 0;
  for (int b = 1; b < L; b <<= 1) {
    r = (r << 1) | (i & 1);
    i >>= 1;
  }
  return r;
}
}  // namespace ct

// static for over [B, E): f(integral_constant<int, i>)
template <int B, int E, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>{});
    sfor<B + 1, E>(static_cast<F&&>(f));
  }
}

// ----------------------------------------------------------------------------------------
// complex helpers
// ----------------------------------------------------------------------------------------
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // conj(a) * b
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}

// Radix-2 DIT butterfly a' = a + W b, b' = a - W b with W = e^{-2 pi i J / SPAN}
// (compile-time).  W = 1 and W = -i cost two packed adds/FMAs; other W use the
// cosine-factored form a +- w (b x-part - t b y-part, ...) with |t| <= 1: three packed FMAs.
// The packed two-wide FP32 operations (__ffma2_rn, __fadd2_rn) round each component once,
// as fmaf and a scalar add do, so the results equal the scalar form bit for bit with half
// the FP32 instructions, which both issue-bound transform kernels need.
template <int J, int SPAN>
__device__ __forceinline__ void dit_bfly(float2& a, float2& b) {
  if constexpr (J == 0) {
    const float2 t = b;
    b = __ffma2_rn(t, make_float2(-1.f, -1.f), a);  // a - t: an exact product, one rounding
    a = __fadd2_rn(a, t);
  } else if constexpr (4 * J == SPAN) {  // W = -i: W b = (b.y, -b.x)
    const float2 s = make_float2(b.y, b.x);
    b = __ffma2_rn(s, make_float2(-1.f, 1.f), a);  // (a.x - b.y, a.y + b.x)
    a = __ffma2_rn(s, make_float2(1.f, -1.f), a);  // (a.x + b.y, a.y - b.x)
  } else {
    constexpr ct::CS cs = ct::cossin2pi(J, SPAN);
    constexpr double wr = cs.c, wi = -cs.s;  // W = wr + i wi
    if constexpr (ct::dabs(wr) >= ct::dabs(wi)) {
      constexpr float r = (float)(wi / wr), sc = (float)wr;
      // W b = wr * u, u = (b.x - r b.y, b.y + r b.x)
      const float2 u = __ffma2_rn(make_float2(b.y, b.x), make_float2(-r, r), b);
      b = __ffma2_rn(make_float2(-sc, -sc), u, a);
      a = __ffma2_rn(make_float2(sc, sc), u, a);
    } else {
      constexpr float r = (float)(wr / wi), sc = (float)wi;
      // W b = wi * u, u = (r b.x - b.y, r b.y + b.x); v = (-u.x, u.y), its first component
      // negated exactly (round-to-nearest is symmetric)
      const float2 v = __ffma2_rn(b, make_float2(-r, r), make_float2(b.y, b.x));
      b = __ffma2_rn(make_float2(sc, -sc), v, a);
      a = __ffma2_rn(make_float2(-sc, sc), v, a);
    }
  }
}

// In-register DFT of L points stored at x[OFF + STRIDE * i], i in [0, L):
// input in bit-reversed order, output in natural order.  X_k = sum_n x_n e^{-2 pi i nk/L}.
template <int L, int OFF = 0, int STRIDE = 1, typename A>
__device__ __forceinline__ void dit(A& x) {
  if constexpr (L > 1) {
    constexpr int LOG = ct::ilog2(L);
    sfor<1, LOG + 1>([&](auto s_) {
      constexpr int span = 1 << decltype(s_)::value;
      constexpr int half = span / 2;
      sfor<0, L / span>([&](auto g_) {
        constexpr int g = decltype(g_)::value * span;
        sfor<0, half>([&](auto j_) {
          constexpr int j = decltype(j_)::value;
          dit_bfly<j, span>(x[OFF + STRIDE * (g + j)], x[OFF + STRIDE * (g + j + half)]);
        });
      });
    });
  }
}

// ----------------------------------------------------------------------------------------
// data translation (Fig. 2 caption): b-bit code -> level, exactly, without I2F
//   b < 8 : level = 2c - (2^b - 1);   b = 8 : two's complement int8
// Built as a float whose mantissa holds the code: 2^23 + v is exact for 0 <= v < 2^23.
// ----------------------------------------------------------------------------------------
template <int BITS>
__device__ __forceinline__ float decode_level(uint32_t word, uint32_t shift) {
  const uint32_t c = (word >> shift) & ((1u << BITS) - 1u);
  if constexpr (BITS == 8) {
    // (c ^ 0x80) - 128 == int8(c)
    return __uint_as_float(0x4B000000u | (c ^ 0x80u)) - 8388736.0f;
  } else {
    // 2c - (2^b - 1) = (2^23 + 2c) - (2^23 + 2^b - 1)
    return __uint_as_float(0x4B000000u | (c << 1)) - (8388608.0f + (float)((1 << BITS) - 1));
  }
}

// (a & b) | c and (a & b) ^ c as one three-input logic operation each (truth tables 0xEA and
// 0x6A over the operand patterns 0xF0, 0xCC, 0xAA).  Written out because with two constant
// operands the compiler spends two logic operations on each.
__device__ __forceinline__ uint32_t and_or(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0xEA;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ uint32_t and_xor(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x6A;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// The same decode from a rotation of the word, for a lane that decodes the same bit
// offset of many words: with rot = decode_rot<BITS>(shift) computed once, a code sits at
// bits [1, BITS] (b < 8) or [0, 8) (b = 8) of rotr(word, rot), so one funnel shift, one
// three-input logic op and one add give the level.
template <int BITS>
__host__ __device__ constexpr uint32_t decode_rot(uint32_t shift) {
  return BITS == 8 ? shift : ((shift + 31u) & 31u);
}
template <int BITS>
__device__ __forceinline__ float decode_level_rot(uint32_t word, uint32_t rot) {
  const uint32_t r = __funnelshift_r(word, word, rot);
  if constexpr (BITS == 8) {
    return __uint_as_float(and_xor(r, 0xFFu, 0x4B000080u)) - 8388736.0f;  // 2^23 + (c ^ 0x80) - 2^23 - 128
  } else {
    return __uint_as_float(and_or(r, ((1u << BITS) - 1u) << 1, 0x4B000000u)) - (8388608.0f + (float)((1 << BITS) - 1));
  }
}

// Both IFs' codes at one rotation into one complex sample, the two final subtractions as
// one packed add (each component rounds as the scalar subtraction; exact here).
template <int BITS>
__device__ __forceinline__ float2 decode_pair_rot(uint32_t wa, uint32_t wb, uint32_t rot) {
  const uint32_t ra = __funnelshift_r(wa, wa, rot), rb = __funnelshift_r(wb, wb, rot);
  if constexpr (BITS == 8) {
    return __fadd2_rn(make_float2(__uint_as_float(and_xor(ra, 0xFFu, 0x4B000080u)),
                                  __uint_as_float(and_xor(rb, 0xFFu, 0x4B000080u))),
                      make_float2(-8388736.0f, -8388736.0f));
  } else {
    constexpr uint32_t m = ((1u << BITS) - 1u) << 1;
    constexpr float c = -(8388608.0f + (float)((1 << BITS) - 1));
    return __fadd2_rn(make_float2(__uint_as_float(and_or(ra, m, 0x4B000000u)), __uint_as_float(and_or(rb, m, 0x4B000000u))),
                      make_float2(c, c));
  }
}

// ----------------------------------------------------------------------------------------
// two-phase plan: N = N1 * N2, n = N2 a + b (a row, b column), k = c + N1 d
//   phase 1: for each column b, DFT-N1 over a (P points per thread, Q1 = N1/P threads)
//   phase 2: for each output column c (pairs c, N1 - c), twiddle W_N^{b c}, DFT-N2 over b
//            (P points per thread, Q2 = N2/P threads), then correlate + accumulate.
// ----------------------------------------------------------------------------------------
// (P, N2) per size; N1 = N / N2.  P = points per thread, 2 <= 2 Q2 <= P, Q1 <= P.
constexpr int plan_p(int logn) { return logn >= 10 ? 32 : (logn >= 8 ? 16 : (logn >= 6 ? 8 : 4)); }
// phase-1 points per lane: 16 at N1 = 128 (half the registers of 32, so three CTAs per SM,
// with the same FFT work per point and warps still four columns = 32 bytes wide).  At
// N1 = 256 sixteen would leave two-column warps whose 16-byte output rows split sectors;
// that measured slower than 32 points per lane at two CTAs per SM.  N1 = 2048 (N = 2^20):
// 64 points per lane, so that one warp still holds a whole column (one CTA per SM).
constexpr int plan_p1(int logn, int n1) { return n1 == 128 ? 16 : (n1 == 2048 ? 64 : plan_p(logn)); }
constexpr int plan_log_n2(int logn) {
  // 4:2 5:3 6:3 7:4 8:4 9:5 10:5 11:6 12:6 13:7 14:7 15:8 16:8 17:9 18:9 19:9 20:9
  return logn >= 17 ? 9 : (logn + 1) / 2;
}
// ----------------------------------------------------------------------------------------
// shared-memory layouts of the warp-local transposes.  The strides below were chosen by an
// offline simulation of the bank conflicts of each transpose's write and read patterns.
// An 8-byte warp access is served as two half-warps; each half costs the largest number of
// distinct elements that fall on one of the 16 bank pairs (this model reproduces the
// measured wavefront counts).  All phase-1 layouts reach the minimum of 2 wavefronts per
// access; phase 2 reaches it at Q2 = 16 and P = 4, Q2 = 2, and costs at most 4 otherwise.
//   phase 1, element (q, p, cw) at q * LDQ1 + p * LDP1 + cw; written by lane (q, cw) for all
//            p, read by lane (q1, cw) for p = r Q1 + q1, then reused as the [c][cw] output tile
//   phase 2, element (unit, e, p, q) at (unit * 2 + e) * LDE2 + p * LDQ2 + q
// ----------------------------------------------------------------------------------------
namespace bank {
struct Ld2 {
  int a, b;
};
constexpr Ld2 p1_layout(int P, int Q1) {
  return (P == 16 && Q1 == 4)    ? Ld2{8, 136}
         : (P == 16 && Q1 == 8)  ? Ld2{4, 68}
         : (P == 16 && Q1 == 16) ? Ld2{2, 34}
         : (P == 32 && Q1 == 2)  ? Ld2{16, 512}
         : (P == 32 && Q1 == 4)  ? Ld2{8, 264}
         : (P == 32 && Q1 == 8)  ? Ld2{4, 132}
         : (P == 32 && Q1 == 16) ? Ld2{2, 66}
         : (P == 32 && Q1 == 32) ? Ld2{1, 33}
         : (P == 64 && Q1 == 32) ? Ld2{1, 65}
                                 : Ld2{32 / Q1, P * (32 / Q1)};  // Q1 = 1: no transpose
}
constexpr Ld2 p2_layout(int P, int Q2) {
  return (P == 32 && Q2 == 16)  ? Ld2{17, 544}
         : (P == 32 && Q2 == 8) ? Ld2{9, 296}
         : (P == 32 && Q2 == 4) ? Ld2{5, 163}
         : (P == 32 && Q2 == 2) ? Ld2{3, 95}
         : (P == 32 && Q2 == 1) ? Ld2{1, 33}
         : (P == 16 && Q2 == 2) ? Ld2{2, 33}
         : (P == 16 && Q2 == 1) ? Ld2{1, 17}
         : (P == 8 && Q2 == 2)  ? Ld2{3, 26}
         : (P == 8 && Q2 == 1)  ? Ld2{1, 9}
         : (P == 4 && Q2 == 2)  ? Ld2{3, 14}
                                : Ld2{1, 5};  // P = 4, Q2 = 1
}
}  // namespace bank

constexpr int pow2_at_least(int v, int lo) {
  int r = lo;
  while (r < v) r *= 2;
  return r;
}

template <int LOGN>
struct Plan {
  static constexpr int N = 1 << LOGN;
  static constexpr int P = plan_p(LOGN);
  static constexpr int N2 = 1 << plan_log_n2(LOGN);
  static constexpr int N1 = N / N2;
  static constexpr int P1 = plan_p1(LOGN, N1);          // phase-1 points per lane
  static constexpr int Q1 = N1 / P1;
  static constexpr int Q2 = N2 / P;
  static constexpr int UPS = N1 / 2;                   // units (column + mirror) per pair-segment
  static constexpr int NACC = P / 2;                   // accumulator bins per phase-2 lane
  static constexpr int NATIVE = UPS * N2 + 1;          // native accumulator bins per FFT pair (= N/2 + 1)
  static constexpr int THREADS = 256;                  // threads per CTA of both phase kernels
  static constexpr int WARPS = THREADS / 32;

  // phase 1: a warp owns CW columns; lane = q1 * CW + cw holds rows q1 + Q1 t
  static constexpr int CW = 32 / Q1;
  static constexpr int PQ = P1 / Q1;
  static constexpr bank::Ld2 L1 = bank::p1_layout(P1, Q1);
  static constexpr int LDP1 = L1.a, LDQ1 = L1.b;
  static constexpr int REGION1 = Q1 > 1 ? Q1 * LDQ1 : 0;  // float2 per warp
  static constexpr int TW1 = ((2 * P1 + 15) / 16) * 16;     // tensor-memory columns per lane (W_N1 twiddles)
  static constexpr int MINB1 = P1 <= 16 ? 3 : (P1 <= 32 ? 2 : 1);  // phase-1 CTAs per SM the registers aim at
  static constexpr int TCOLS1 = pow2_at_least((WARPS / 4) * TW1, 32);
  // CTA tiles of IPT * WARPS * CW columns inside one segment (Stage1<BITS>): the CTA stages
  // the tile's packed words (both IFs) in shared memory; otherwise (small N) every lane loads
  // its own words.  IPT column groups per warp per tile: two where the tile divides N2 and two
  // stage buffers still leave room for two CTAs per SM (fewer CTA barriers and less staging
  // work per column).  Four measured slower at 2^17: too few tiles per SM to balance.
  static constexpr size_t kSmemPerCta2 = (233472 - MINB1 * 1024) / MINB1;  // MINB1 CTAs per SM
  static constexpr size_t REGIONS1 = sizeof(float2) * (size_t)WARPS * REGION1;
  template <int BITS>
  struct Stage1 {
    static constexpr int tile_of(int ipt) { return ipt * WARPS * CW; }
    static constexpr int wpr_of(int ipt) { return tile_of(ipt) * BITS / 32; }
    // staged row: the tile's words of the two IFs interleaved (word w of IF a, of IF b, ...)
    // so that one 8-byte load fetches both, padded to an odd number of 8-byte pairs (rows of
    // distinct q1 then fall on distinct bank pairs)
    static constexpr int row_words(int ipt) { return 2 * wpr_of(ipt) + (wpr_of(ipt) % 2 ? 0 : 2); }
    static constexpr bool fits(int ipt, int bufs) {
      return REGIONS1 + 4 * (size_t)bufs * N1 * row_words(ipt) + 32 <= kSmemPerCta2;
    }
    // a tile of whole words that divides N2
    static constexpr bool aligned(int ipt) {
      return N2 % tile_of(ipt) == 0 && (tile_of(ipt) * BITS) % 32 == 0 && tile_of(ipt) * BITS >= 32;
    }
    static constexpr bool ok(int ipt) { return aligned(ipt) && tile_of(ipt) % 32 == 0 && fits(ipt, 2); }
    // Column groups per tile, 0 = not staged.  Tiles of 32 or more columns first; for
    // N1 >= 512 (warps of one or two columns, whose unstaged loads would each touch 32
    // sectors) any tile of whole words, preferring two stage buffers, then more columns.
    static constexpr int pick() {
      return ok(2)                                                 ? 2
             : (N2 % tile_of(1) == 0 && tile_of(1) % 32 == 0)     ? 1
             : N1 < 512                                           ? 0
             : (aligned(2) && fits(2, 2))                         ? 2
             : (aligned(1) && fits(1, 2))                         ? 1
             : (aligned(2) && fits(2, 1))                         ? 2
             : (aligned(1) && fits(1, 1))                         ? 1
                                                                  : 0;
    }
    static constexpr int IPT = pick() > 0 ? pick() : 1;
    static constexpr int TILE = IPT * WARPS * CW;
    static constexpr bool STAGED = pick() > 0;
    static constexpr int WPR = TILE * BITS / 32;  // words per IF per staged row
    static constexpr int RS = row_words(IPT);
    static constexpr int NB = fits(IPT, 2) ? 2 : 1;  // 2: the next tile in flight
    static constexpr int WORDS = STAGED ? NB * N1 * RS : 0;
    // TMA boxes are at most 256 rows: larger N1 moves by N1 / BOXR boxes per copy
    static constexpr int BOXR = N1 < 256 ? N1 : 256;
    // N1 <= 256: the warp's [N1][CW] output block leaves by one TMA store (rows of 32 bytes
    // or more).  N1 >= 512 (warps of one or two columns): the column group's [N1][WARPS CW]
    // block is assembled in the CTA's transpose regions, which it fits, and leaves by
    // N1 / BOXR TMA stores of 64- or 128-byte rows (swizzled in shared memory); per-warp
    // stores of 8- or 16-byte rows measured several times slower.
    static constexpr int JC = WARPS * CW;  // columns of the joint block
    static constexpr bool TMA_OUT = STAGED && Q1 > 1 && N1 <= 256;
    static constexpr bool JOINT_OUT = STAGED && Q1 > 1 && N1 >= 512 && (JC * 8 == 64 || JC * 8 == 128) &&
                                      (size_t)N1 * JC * 8 <= REGIONS1;
    static constexpr int JSW = JC * 8 == 128 ? 7 : 3;  // swizzle mask: 128-byte (SW128) or 64-byte (SW64) rows
    // the tile's input may be staged by TMA (two buffers, 16-byte box rows, one box of all
    // N1 rows: at N1 = 512 two boxes of 256 rows measured slower than cp.async staging)
    static constexpr bool TMA_IN = STAGED && NB == 2 && (WPR * 4) % 16 == 0 && N1 <= 256;
    static constexpr size_t SMEM = REGIONS1 + 4 * (size_t)WORDS + 16 + 16;  // + 2 mbarriers + TMEM slot
  };

  // phase 2: a warp owns UPW units; lane = (uw * 2 + e) * Q2 + q2 holds rows q2 + Q2 t
  static constexpr int UPW = 16 / Q2;
  static constexpr int PP = P / (2 * Q2);                  // p-values per lane after the joint transpose
  static constexpr int SL = UPW > UPS ? UPW / UPS : 1;     // segments in flight per warp (small N)
  static constexpr int UGW = UPW > UPS ? 1 : UPS / UPW;    // unit groups per pair-segment
  static constexpr bank::Ld2 L2 = bank::p2_layout(P, Q2);
  static constexpr int LDQ2 = L2.a, LDE2 = L2.b;
  // prefetch column padding (see PF2): Q2 values, at least two (16-byte aligned copies)
  static constexpr int PADC = UPW > 1 ? (Q2 >= 2 ? Q2 : 2) : 0;
  static constexpr int REGION2 =
      (2 * UPW * LDE2 > 2 * UPW * (N2 + PADC)) ? 2 * UPW * LDE2 : 2 * UPW * (N2 + PADC);
  // W_N2^k at k + k/32.  (A lane-contiguous [q][p] table has fewer bank conflicts but
  // measured slower in this kernel.)  With one p per lane (PP = 1), W_N2^{q p} by (p, q) at
  // p (Q2 + 1) + q instead: the lane's row, no index arithmetic per lookup, and rows of an odd
  // number of 8-byte entries put a half-warp's 16 rows on distinct bank pairs.
  static constexpr bool TWPQ = PP == 1;
  static constexpr int LDT2 = Q2 + 1;
  static constexpr int TWT = (TWPQ && P * LDT2 > N2 + N2 / 32 + 1) ? P * LDT2 : N2 + N2 / 32 + 1;
  static constexpr int TACC = ((2 * P + 15) / 16) * 16;    // tensor-memory columns per lane: accumulators
  static constexpr int TTW = ((2 * P + 15) / 16) * 16;     // and the lane's column twiddles W_N^{b u}
  static constexpr int TCOLS2 = pow2_at_least((WARPS / 4) * (TACC + TTW), 32);
  // phase 2 prefetches the next segment's 2 UPW columns (each unit's column and its mirror)
  // into the warp's region with bulk copies when a warp holds the units of one segment
  // (2^9 and up).  Column g sits at g (N2 + PADC): the Q2-lane groups of a half-warp then
  // start on distinct bank pairs (two-way conflicts at Q2 = 1, where the pad is 2).
  static constexpr bool PF2 = (SL == 1) && (UPW <= 16) && (PADC * 8) % 16 == 0 && (N2 * 8) % 16 == 0 &&
                              (2 * UPW * (N2 + PADC) <= REGION2);
  // regions | W_N2 table | tensor-memory slot (16 B) | one mbarrier per warp
  static constexpr size_t SMEM2 = sizeof(float2) * ((size_t)WARPS * REGION2 + TWT) + 16 + 8 * WARPS;

  static_assert(N1 * N2 == N, "plan");
  static_assert(Q1 >= 1 && Q1 <= 32 && P1 % Q1 == 0 && Q2 >= 1 && 2 * Q2 <= P && 16 % Q2 == 0, "plan bounds");
  static_assert(N1 <= 2048 && N2 <= 2048, "constant twiddle table covers L <= 2048");
  static_assert(UPS % UPW == 0 || UPW % UPS == 0, "units per warp");
  static_assert(TCOLS1 <= 256 && TCOLS2 <= 256, "tensor memory per CTA");
};

}  // namespace polaris
