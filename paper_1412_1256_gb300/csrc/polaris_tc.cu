// Tensor-core DFT spectrometer: the precision variant of the transform.
//
// One FFT pair (two IFs, pair-packed z = x + iy as in the FP32 path) per handle, whole
// segments (hop = N), N = 64^2 or 64^3.  The transform is taken as Stockham autosort passes
// of radix 64 (Ns = 1, 64, 4096 points already combined): every j < N/64 reads
// z[j + r N/64] (r < 64), multiplies by W_{64 Ns}^{r (j mod Ns)}, takes a 64-point DFT and
// writes output q to z[(j - j mod Ns) 64 + q Ns + j mod Ns].  A pass is one batch of
// 64-point DFTs, i.e. a GEMM: rows = the vectors j of all segments of a batch, K = the 64
// complex inputs as 128 reals [Re a | Im a], N = the 64 complex outputs as 128 reals, with
// the real 128 x 128 form of the DFT matrix F = W_64^{rq}:
//   Re b = Re a (Re F) + Im a (-Im F),  Im b = Re a (Im F) + Im a (Re F).
// The GEMM runs on the 5th-generation tensor cores (tcgen05.mma kind::f16, M = 128 rows,
// N = 128, K = 16 per instruction, FP32 accumulation in tensor memory).  Operands are
// 16-bit, so each FP32 operand x is split as x = hi + lo (hi = x rounded to 16 bits,
// lo = x - hi rounded again) and the product is taken as lo_a hi_b + hi_a lo_b +
// hi_a hi_b (the lo_a lo_b term is dropped):
//   BF16X3  bf16 halves: about 17 significant bits per operand
//   FP16X3  fp16 halves: about 22 bits; every row is scaled by an exact power of two so
//           that its largest value sits just under 2^15 (fp16 has no exponent range to spare)
//   BF16X1  hi_a hi_b alone: the plain 16-bit tensor-core product, for comparison
// Twiddles and the DFT matrix are computed in FP64 on the host; integration accumulators
// are FP64.  Pass kernels read their input with coalesced loads (a warp's lanes are
// consecutive j), the first pass decodes and windows the packed samples on the way; the
// first pass's output rows (64 consecutive values per row) go out through shared memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/polaris.h"
#include "polaris_device.cuh"

namespace polaris {
namespace tc {

constexpr int kR = 64;             // radix of a pass
constexpr int kRows = 128;         // GEMM M: vectors per tile, one per thread
constexpr int kK = 2 * kR;         // GEMM K and N in reals
constexpr int kGroups = 2;         // independent tile groups per CTA (their latencies overlap)
constexpr int kGroupThreads = kRows;
constexpr int kThreads = kGroups * kGroupThreads;
constexpr uint32_t kOpBytes = kRows * kK * 2;      // one 16-bit operand tile: 32 KB
constexpr uint32_t kLBO = 128;                     // core matrices (8 rows x 16 B) along K
constexpr uint32_t kSBO = (kK / 8) * 128;          // ... along M (or N)
constexpr uint32_t kStagePitch = kR + 1;           // first-pass output rows in shared memory (float2)
// shared memory: per group A hi | A lo (the first pass's output stage overlaps both), then the
// shared B hi | B lo, one barrier per group, the TMEM address slot
constexpr uint32_t kOffAh = 0, kOffAl = kOpBytes;
constexpr uint32_t kStageBytes = kRows * kStagePitch * 8;
constexpr uint32_t kGroupBytes = (kStageBytes + 127) / 128 * 128;
constexpr uint32_t kOffBh = kGroups * kGroupBytes, kOffBl = kOffBh + kOpBytes;
constexpr uint32_t kOffBar = kOffBl + kOpBytes, kOffSlot = kOffBar + 8 * kGroups;
constexpr uint32_t kSmemBytes = kOffSlot + 8;
constexpr uint32_t kTmemCols = 128 * kGroups;      // group g accumulates in columns [128 g, 128 g + 128)
constexpr uint32_t kWaitAfter = 1u << 24;

// element (row, k) of a [rows][128] 16-bit operand in the canonical no-swizzle K-major layout
__host__ __device__ constexpr uint32_t op_off(int row, int k) {
  return (uint32_t)(row >> 3) * kSBO + (uint32_t)(k >> 3) * kLBO + (uint32_t)(row & 7) * 16 + (uint32_t)(k & 7) * 2;
}

struct PassArgs {
  const uint32_t* in[2];  // first pass: the packed IF streams
  long long sample0;      // first pass: the batch's first sample
  const float* window;    // first pass: N taps
  const float2* src;      // later passes: previous output [nseg][N]
  float2* dst;            // [nseg][N]
  const float2* tw;       // per-pass twiddles: tw[r Ns + k - 1] = W_{64 Ns}^{r k}
  const uint4* bmat;      // DFT matrix, hi then lo, in the operand layout (2 x 32 KB)
  int N, m, Ns, nseg;     // m = N / 64 vectors per segment
  int* err;
  unsigned wait_limit;
};

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t op_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
         ((uint64_t)1 << 46);
}

__device__ __forceinline__ void mma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}

// barrier over the 128 threads of tile group g (named barrier 1 + g)
__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(1 + g), "r"(kGroupThreads) : "memory");
}
// the same barrier, returning whether any thread of the group passed `pred`
__device__ __forceinline__ bool group_any(int g, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(1 + g), "r"(kGroupThreads)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ bool wait_parity(uint32_t bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

template <int BITS>
__device__ __forceinline__ float tc_level(const uint32_t* __restrict__ in, long long idx) {
  if constexpr (BITS == 8) {
    return (float)(int)__ldg(reinterpret_cast<const signed char*>(in) + idx);
  } else {
    constexpr int SPW = 32 / BITS;
    return decode_level<BITS>(__ldg(in + idx / SPW), (uint32_t)(idx % SPW) * BITS);
  }
}

// 8 consecutive values -> 8 16-bit hi halves and 8 lo halves (x = hi + lo)
template <int PREC>
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if constexpr (PREC == POLARIS_TC_FP16X3) {
      const __half2 hh = __floats2half2_rn(v[2 * i], v[2 * i + 1]);
      const float2 hf = __half22float2(hh);
      const __half2 ll = __floats2half2_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
      h[i] = *reinterpret_cast<const uint32_t*>(&hh);
      l[i] = *reinterpret_cast<const uint32_t*>(&ll);
    } else {
      const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
      const float2 hf = __bfloat1622float2(hh);
      const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
      h[i] = *reinterpret_cast<const uint32_t*>(&hh);
      l[i] = *reinterpret_cast<const uint32_t*>(&ll);
    }
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// One radix-64 pass over all vectors of a batch (BITS > 0: the first pass, from the packed
// samples).  Persistent CTAs of two tile groups of 128 threads; tiles of 128 consecutive
// vectors (global vector v = segment * m + j) go round robin to the groups of all CTAs.
// Thread t of a group owns vector tile * 128 + t and TMEM lane t of the group's columns.
template <int PREC, int BITS>
__global__ void __launch_bounds__(kThreads, 1) k_tc_pass(PassArgs a) {
  extern __shared__ __align__(128) uint8_t sm[];
  const int gr = threadIdx.x / kGroupThreads, t = threadIdx.x % kGroupThreads, w = t >> 5;
  uint8_t* sg = sm + gr * kGroupBytes;
  const uint32_t bar = saddr(sm + kOffBar + 8 * gr);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kOffSlot);
  constexpr int NPROD = PREC == POLARIS_TC_BF16X1 ? 1 : 3;
  constexpr int NB = (PREC == POLARIS_TC_BF16X1 ? 1 : 2) * (int)kOpBytes / 16;
  for (int i = threadIdx.x; i < NB; i += kThreads) reinterpret_cast<uint4*>(sm + kOffBh)[i] = __ldg(a.bmat + i);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(saddr(slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tbase = *slot, tmem = tbase + 128u * gr;
  // D f32, A and B bf16 (1) or f16 (0), both K-major, N = 128, M = 128
  constexpr uint32_t fmt = PREC == POLARIS_TC_FP16X3 ? 0u : 1u;
  constexpr uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kK >> 3) << 17) |
                             ((uint32_t)(kRows >> 4) << 24);
  const long long rows = (long long)a.nseg * a.m;
  const int tiles = (int)((rows + kRows - 1) / kRows);
  const int worker = blockIdx.x * kGroups + gr, workers = gridDim.x * kGroups;
  uint32_t parity = 0;
  bool failed = false;
  for (int tile = worker; tile < tiles && !failed; tile += workers) {
    const long long g = (long long)tile * kRows + t;
    const bool valid = g < rows;
    const long long gv = valid ? g : 0;
    const int s = (int)(gv / a.m), j = (int)(gv - (long long)s * a.m);
    float v[kK];
    if constexpr (BITS > 0) {
      const long long base = a.sample0 + (long long)s * a.N + j;
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        const float wn = __ldg(a.window + j + r * a.m);
        v[r] = wn * tc_level<BITS>(a.in[0], base + (long long)r * a.m);
        v[kR + r] = wn * tc_level<BITS>(a.in[1], base + (long long)r * a.m);
      }
    } else {
      const float2* src = a.src + (long long)s * a.N + j;
      const int k = j & (a.Ns - 1);
#pragma unroll
      for (int r = 0; r < kR; ++r) {
        float2 z = __ldcg(src + (long long)r * a.m);
        if (r > 0) z = cmul(z, __ldg(a.tw + (r * a.Ns + k - 1)));
        v[r] = z.x;
        v[kR + r] = z.y;
      }
    }
    float inv_scale = 1.f;
    if constexpr (PREC == POLARIS_TC_FP16X3) {
      float amax = 0.f;
#pragma unroll
      for (int i = 0; i < kK; ++i) amax = fmaxf(amax, fabsf(v[i]));
      int e = 0;
      frexpf(amax, &e);  // amax = f 2^e, f in [0.5, 1); zero gives e = 0
      const float sc = ldexpf(1.f, 15 - e);
      inv_scale = ldexpf(1.f, e - 15);
#pragma unroll
      for (int i = 0; i < kK; ++i) v[i] *= sc;
    }
    if (!valid) {
#pragma unroll
      for (int i = 0; i < kK; ++i) v[i] = 0.f;
    }
#pragma unroll
    for (int kc = 0; kc < kK / 8; ++kc) {
      uint4 hi, lo;
      split8<PREC>(v + 8 * kc, hi, lo);
      *reinterpret_cast<uint4*>(sg + kOffAh + op_off(t, 8 * kc)) = hi;
      if constexpr (NPROD == 3) *reinterpret_cast<uint4*>(sg + kOffAl + op_off(t, 8 * kc)) = lo;
    }
    // operands visible to the tensor cores; the previous tile's TMEM reads are complete
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    group_sync(gr);
    if (t == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t ah = saddr(sg + kOffAh), al = saddr(sg + kOffAl);
      const uint32_t bh = saddr(sm + kOffBh), bl = saddr(sm + kOffBl);
      // small products first: lo_a hi_b, hi_a lo_b, then hi_a hi_b
      const uint32_t pa[3] = {NPROD == 3 ? al : ah, ah, ah};
      const uint32_t pb[3] = {bh, NPROD == 3 ? bl : bh, bh};
#pragma unroll
      for (int p = 3 - NPROD; p < 3; ++p)
#pragma unroll
        for (int ks = 0; ks < kK / 16; ++ks)
          mma_f16(tmem, op_desc(pa[p] + ks * 256), op_desc(pb[p] + ks * 256), idesc,
                  (p > 3 - NPROD || ks > 0) ? 1u : 0u);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                   : "memory");
    }
    // one decision for the whole group (every thread leaves the loop at the same tile)
    if (group_any(gr, !wait_parity(bar, parity, a.wait_limit))) {
      failed = true;
      if (t == 0 && a.err) atomicOr(a.err, 1);
      wait_parity(bar, parity, kWaitAfter);  // the products in flight land before the exit
    }
    parity ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // row t of D: Re b_q in columns q, Im b_q in columns 64 + q
#pragma unroll
    for (int c = 0; c < kK; c += 16) {
      uint32_t u[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]),
            "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
          : "r"(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c)
          : "memory");
#pragma unroll
      for (int i = 0; i < 16; ++i) v[c + i] = __uint_as_float(u[i]) * inv_scale;
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if constexpr (BITS > 0) {
      // output row g = 64 consecutive values at 64 g: through shared memory (pitch 65
      // float2), then 128 threads write the tile's 64 KB contiguously
      float2* stage = reinterpret_cast<float2*>(sg);
#pragma unroll
      for (int q = 0; q < kR; ++q) stage[t * kStagePitch + q] = make_float2(v[q], v[kR + q]);
      group_sync(gr);
      const long long out0 = (long long)tile * kRows * kR;
      const int nvals = (int)(min((long long)kRows, rows - (long long)tile * kRows) * kR);
      for (int e = t; e < nvals; e += kGroupThreads) __stcg(a.dst + out0 + e, stage[(e / kR) * kStagePitch + (e % kR)]);
    } else if (valid) {
      const int k = j & (a.Ns - 1);
      float2* dst = a.dst + (long long)s * a.N + (long long)(j - k) * kR + k;
#pragma unroll
      for (int q = 0; q < kR; ++q) __stcg(dst + (long long)q * a.Ns, make_float2(v[q], v[kR + q]));
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    group_sync(gr);  // stage reads and TMEM reads done before the next tile's operands
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(kTmemCols) : "memory");
}

// per bin k: X = (Z_k + conj Z_{N-k}) / 2, Y = (Z_k - conj Z_{N-k}) / 2i over the batch's
// segments; |X|^2, |Y|^2, X conj(Y) in FP32 with compensated (Kahan) sums over the batch,
// then added once to the FP64 accumulators [4][nbin]
__device__ __forceinline__ void kahan_add(float& sum, float& comp, float x) {
  const float y = x - comp;
  const float t = sum + y;
  comp = (t - sum) - y;
  sum = t;
}

__global__ void __launch_bounds__(256) k_tc_correlate(const float2* __restrict__ Z, int N, int nbin, int nseg,
                                                      double* __restrict__ acc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbin) return;
  const int km = (N - k) & (N - 1);
  float sm[4] = {0.f, 0.f, 0.f, 0.f}, cp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
  for (int s = 0; s < nseg; ++s) {
    const float2 a = __ldcg(Z + (long long)s * N + k), b = __ldcg(Z + (long long)s * N + km);
    const float xr = 0.5f * (a.x + b.x), xi = 0.5f * (a.y - b.y);
    const float yr = 0.5f * (a.y + b.y), yi = -0.5f * (a.x - b.x);
    kahan_add(sm[0], cp[0], fmaf(xr, xr, xi * xi));
    kahan_add(sm[1], cp[1], fmaf(yr, yr, yi * yi));
    kahan_add(sm[2], cp[2], fmaf(xr, yr, xi * yi));
    kahan_add(sm[3], cp[3], fmaf(xi, yr, -xr * yi));
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[(size_t)q * nbin + k] += (double)sm[q] - (double)cp[q];
}

// autos, cross and linear-feed Stokes (Eq. 2, psi = 0, unit gains); the accumulators clear
__global__ void __launch_bounds__(256) k_tc_readout(double* __restrict__ acc, int nbin, double* autos, double* cross,
                                                    double* stokes) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nbin) return;
  const double xx = acc[k], yy = acc[nbin + k], cr = acc[2 * (size_t)nbin + k], ci = acc[3 * (size_t)nbin + k];
  if (autos) {
    autos[k] = xx;
    autos[nbin + k] = yy;
  }
  if (cross) {
    cross[2 * (size_t)k] = cr;
    cross[2 * (size_t)k + 1] = ci;
  }
  if (stokes) {
    stokes[k] = 0.5 * (xx + yy);
    stokes[nbin + k] = 0.5 * (xx - yy);
    stokes[2 * (size_t)nbin + k] = cr;
    stokes[3 * (size_t)nbin + k] = ci;
  }
  acc[k] = 0.0;
  acc[nbin + k] = 0.0;
  acc[2 * (size_t)nbin + k] = 0.0;
  acc[3 * (size_t)nbin + k] = 0.0;
}

}  // namespace tc
}  // namespace polaris

using namespace polaris;
using namespace polaris::tc;

struct polaris_tc {
  int N = 0, m = 0, npass = 0, bits = 0, prec = 0, device = 0, nbin = 0, grid = 0, batch = 0;
  float* d_window = nullptr;
  float2* d_tw = nullptr;
  uint4* d_bmat = nullptr;
  float2* d_buf[2] = {nullptr, nullptr};
  double* d_acc = nullptr;
  int* d_err = nullptr;
  int64_t nseg = 0;
  unsigned wait_limit = 1u << 26;
  bool broken = false;
  std::string err;
};

static thread_local std::string g_tc_create_err;

static int tc_err(polaris_tc* h, int code, const std::string& m) {
  if (h) h->err = m;
  else g_tc_create_err = m;
  return code;
}

static uint16_t host_bf16(float x) {
  const __nv_bfloat16 b = __float2bfloat16_rn(x);
  uint16_t u;
  memcpy(&u, &b, 2);
  return u;
}
static float host_bf16_val(uint16_t u) {
  __nv_bfloat16 b;
  memcpy(&b, &u, 2);
  return __bfloat162float(b);
}
static uint16_t host_f16(float x) {
  const __half h = __float2half_rn(x);
  uint16_t u;
  memcpy(&u, &h, 2);
  return u;
}
static float host_f16_val(uint16_t u) {
  __half h;
  memcpy(&h, &u, 2);
  return __half2float(h);
}

template <int PREC, int BITS>
static cudaError_t tc_set_smem() {
  return cudaFuncSetAttribute(k_tc_pass<PREC, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
}

template <int PREC>
static cudaError_t tc_prepare(int bits) {
  cudaError_t e = tc_set_smem<PREC, 0>();
  if (e != cudaSuccess) return e;
  switch (bits) {
    case 1: return tc_set_smem<PREC, 1>();
    case 2: return tc_set_smem<PREC, 2>();
    case 4: return tc_set_smem<PREC, 4>();
    default: return tc_set_smem<PREC, 8>();
  }
}

template <int PREC>
static cudaError_t tc_launch_pass(int bits, const PassArgs& a, int grid, cudaStream_t st) {
  if (a.Ns == 1) {
    switch (bits) {
      case 1: k_tc_pass<PREC, 1><<<grid, kThreads, kSmemBytes, st>>>(a); break;
      case 2: k_tc_pass<PREC, 2><<<grid, kThreads, kSmemBytes, st>>>(a); break;
      case 4: k_tc_pass<PREC, 4><<<grid, kThreads, kSmemBytes, st>>>(a); break;
      default: k_tc_pass<PREC, 8><<<grid, kThreads, kSmemBytes, st>>>(a); break;
    }
  } else {
    k_tc_pass<PREC, 0><<<grid, kThreads, kSmemBytes, st>>>(a);
  }
  return cudaGetLastError();
}

static void tc_free(polaris_tc* h) {
  cudaFree(h->d_window);
  cudaFree(h->d_tw);
  cudaFree(h->d_bmat);
  cudaFree(h->d_buf[0]);
  cudaFree(h->d_buf[1]);
  cudaFree(h->d_acc);
  cudaFree(h->d_err);
}

extern "C" int polaris_tc_create(int64_t n_fft, int bits, int window, const float* taps, int precision, int device,
                                 polaris_tc** out) {
  if (!out) return POLARIS_EINVAL;
  *out = nullptr;
  if (n_fft != 4096 && n_fft != 262144) return tc_err(nullptr, POLARIS_EINVAL, "n_fft must be 64^2 = 4096 or 64^3 = 262144");
  if (bits != 1 && bits != 2 && bits != 4 && bits != 8) return tc_err(nullptr, POLARIS_EINVAL, "bits must be 1, 2, 4 or 8");
  if (precision != POLARIS_TC_BF16X3 && precision != POLARIS_TC_FP16X3 && precision != POLARIS_TC_BF16X1)
    return tc_err(nullptr, POLARIS_EINVAL, "unknown precision");
  if (window != POLARIS_WIN_RECT && window != POLARIS_WIN_HANN && window != POLARIS_WIN_CUSTOM)
    return tc_err(nullptr, POLARIS_EINVAL, "unknown window");
  if (window == POLARIS_WIN_CUSTOM && !taps) return tc_err(nullptr, POLARIS_EINVAL, "custom window needs taps");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return tc_err(nullptr, POLARIS_EINVAL, "no such CUDA device");
  }
  polaris_tc* h = new polaris_tc;
  h->N = (int)n_fft;
  h->m = h->N / kR;
  h->npass = h->N == 4096 ? 2 : 3;
  h->bits = bits;
  h->prec = precision;
  h->device = device;
  h->nbin = h->N / 2 + 1;
  h->batch = (int)std::max<int64_t>(2, (int64_t)(32u << 20) / ((int64_t)h->N * 8));  // 32 MB per buffer
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  int nsm = 0;
  cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) {
    switch (precision) {
      case POLARIS_TC_BF16X3: e = tc_prepare<POLARIS_TC_BF16X3>(bits); break;
      case POLARIS_TC_FP16X3: e = tc_prepare<POLARIS_TC_FP16X3>(bits); break;
      default: e = tc_prepare<POLARIS_TC_BF16X1>(bits); break;
    }
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaSetDevice(prev);
    delete h;
    return tc_err(nullptr, POLARIS_ECUDA, std::string("tensor-core kernels cannot be launched: ") + cudaGetErrorString(e));
  }
  h->grid = nsm;  // one CTA (two tile groups, 194 KB) per SM
  // window taps (FP64-computed, rounded once)
  std::vector<float> win(h->N);
  for (int n = 0; n < h->N; ++n) {
    if (window == POLARIS_WIN_RECT) win[n] = 1.f;
    else if (window == POLARIS_WIN_HANN) win[n] = (float)(0.5 - 0.5 * std::cos(2.0 * M_PI * n / h->N));
    else win[n] = taps[n];
  }
  // per-pass twiddles W_{64 Ns}^{r k} at r Ns + k - 1 (passes Ns = 64, 4096: offsets Ns - 1)
  std::vector<float2> tw(h->N, make_float2(0.f, 0.f));
  for (int Ns = kR; Ns < h->N; Ns *= kR)
    for (int r = 1; r < kR; ++r)
      for (int k = 0; k < Ns; ++k) {
        const double ang = -2.0 * M_PI * (double)r * (double)k / (double)(kR * Ns);
        tw[(size_t)r * Ns + k - 1] = make_float2((float)std::cos(ang), (float)std::sin(ang));
      }
  // the real 128 x 128 DFT-64 matrix as the N-major (K contiguous) operand, hi and lo
  std::vector<uint16_t> bm(2 * kOpBytes / 2, 0);
  for (int nn = 0; nn < kK; ++nn)
    for (int kk = 0; kk < kK; ++kk) {
      const int q = nn % kR, r = kk % kR;
      const double ang = 2.0 * M_PI * (double)((r * q) % kR) / kR;
      const double c = std::cos(ang), sn = std::sin(ang);  // F = c - i sn
      double val;
      if (nn < kR) val = kk < kR ? c : sn;   // Re b = Re a c + Im a sn
      else val = kk < kR ? -sn : c;          // Im b = -Re a sn + Im a c
      uint16_t hi, lo;
      if (precision == POLARIS_TC_FP16X3) {
        hi = host_f16((float)val);
        lo = host_f16((float)(val - (double)host_f16_val(hi)));
      } else {
        hi = host_bf16((float)val);
        lo = host_bf16((float)(val - (double)host_bf16_val(hi)));
      }
      bm[op_off(nn, kk) / 2] = hi;
      bm[(kOpBytes + op_off(nn, kk)) / 2] = lo;
    }
  const size_t buf = (size_t)h->batch * h->N * sizeof(float2);
  bool ok = cudaMalloc((void**)&h->d_window, h->N * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&h->d_tw, h->N * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&h->d_bmat, 2 * kOpBytes) == cudaSuccess &&
            cudaMalloc((void**)&h->d_buf[0], buf) == cudaSuccess && cudaMalloc((void**)&h->d_buf[1], buf) == cudaSuccess &&
            cudaMalloc((void**)&h->d_acc, 4 * (size_t)h->nbin * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&h->d_err, sizeof(int)) == cudaSuccess &&
            cudaMemcpy(h->d_window, win.data(), h->N * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(h->d_tw, tw.data(), h->N * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(h->d_bmat, bm.data(), 2 * kOpBytes, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemset(h->d_acc, 0, 4 * (size_t)h->nbin * sizeof(double)) == cudaSuccess &&
            cudaMemset(h->d_err, 0, sizeof(int)) == cudaSuccess;
  cudaSetDevice(prev);
  if (!ok) {
    cudaGetLastError();
    tc_free(h);
    delete h;
    return tc_err(nullptr, POLARIS_ENOMEM, "device allocation failed");
  }
  *out = h;
  return POLARIS_OK;
}

extern "C" void polaris_tc_destroy(polaris_tc* h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  tc_free(h);
  cudaSetDevice(prev);
  delete h;
}

extern "C" const char* polaris_tc_last_error(const polaris_tc* h) { return h ? h->err.c_str() : g_tc_create_err.c_str(); }

extern "C" int polaris_tc_set_wait_limit(polaris_tc* h, int64_t limit) {
  if (!h) return POLARIS_EINVAL;
  h->wait_limit = limit < 0 ? (1u << 26) : (unsigned)std::min<int64_t>(limit, 0xffffffffLL);
  return POLARIS_OK;
}

extern "C" int polaris_tc_feed(polaris_tc* h, const void* const* packed, int64_t n_samples, void* cuda_stream) {
  if (!h) return POLARIS_EINVAL;
  if (h->broken) return tc_err(h, POLARIS_ESTATE, "a device wait timed out earlier; the handle is unusable");
  if (!packed || !packed[0] || !packed[1]) return tc_err(h, POLARIS_EINVAL, "null input pointer");
  if (n_samples < 0 || n_samples % h->N) return tc_err(h, POLARIS_EINVAL, "n_samples must be a multiple of n_fft");
  const int64_t nseg = n_samples / h->N;
  if (nseg == 0) return POLARIS_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaSuccess;
  for (int64_t s0 = 0; s0 < nseg && e == cudaSuccess; s0 += h->batch) {
    const int nb = (int)std::min<int64_t>(h->batch, nseg - s0);
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.in[0] = static_cast<const uint32_t*>(packed[0]);
    a.in[1] = static_cast<const uint32_t*>(packed[1]);
    a.sample0 = s0 * h->N;
    a.window = h->d_window;
    a.tw = h->d_tw;
    a.bmat = h->d_bmat;
    a.N = h->N;
    a.m = h->m;
    a.nseg = nb;
    a.err = h->d_err;
    a.wait_limit = h->wait_limit;
    int cur = 0;
    for (int p = 0, Ns = 1; p < h->npass && e == cudaSuccess; ++p, Ns *= kR) {
      a.Ns = Ns;
      a.src = h->d_buf[cur ^ 1];
      a.dst = h->d_buf[cur];
      const int tiles = (int)(((int64_t)nb * h->m + kRows - 1) / kRows);
      const int grid = std::min((tiles + kGroups - 1) / kGroups, h->grid);
      switch (h->prec) {
        case POLARIS_TC_BF16X3: e = tc_launch_pass<POLARIS_TC_BF16X3>(h->bits, a, grid, st); break;
        case POLARIS_TC_FP16X3: e = tc_launch_pass<POLARIS_TC_FP16X3>(h->bits, a, grid, st); break;
        default: e = tc_launch_pass<POLARIS_TC_BF16X1>(h->bits, a, grid, st); break;
      }
      cur ^= 1;
    }
    if (e == cudaSuccess) {
      k_tc_correlate<<<(h->nbin + 255) / 256, 256, 0, st>>>(h->d_buf[cur ^ 1], h->N, h->nbin, nb, h->d_acc);
      e = cudaGetLastError();
    }
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) return tc_err(h, POLARIS_ECUDA, std::string("CUDA: ") + cudaGetErrorString(e));
  h->nseg += nseg;
  return POLARIS_OK;
}

extern "C" int polaris_tc_integrate(polaris_tc* h, double* autos, double* cross, double* stokes, int64_t* n_segments,
                                    void* cuda_stream) {
  if (!h) return POLARIS_EINVAL;
  if (h->broken) return tc_err(h, POLARIS_ESTATE, "a device wait timed out earlier; the handle is unusable");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  k_tc_readout<<<(h->nbin + 255) / 256, 256, 0, st>>>(h->d_acc, h->nbin, autos, cross, stokes);
  cudaError_t e = cudaGetLastError();
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaSetDevice(prev);
  if (e != cudaSuccess) return tc_err(h, POLARIS_ECUDA, std::string("CUDA: ") + cudaGetErrorString(e));
  if (n_segments) *n_segments = h->nseg;
  h->nseg = 0;
  if (herr) {
    h->broken = true;
    return tc_err(h, POLARIS_ETIMEOUT, "a tensor-core completion wait timed out");
  }
  return POLARIS_OK;
}
