// Leakage calibration: the segment kernels of the forward and window passes specialised per
// transform size N = 2^LOGN, kAdjSizedMin <= LOGN <= kAdjSizedMax, so that every index, pass
// and radix is a compile-time constant.  They compute what k_adj_forward and k_adj_window
// (polaris_adjoint.cu) compute, with the same per-CTA order of summation:
//   - one CTA of T = N/PPT threads per segment at a time, PPT points per thread (16; 32 at
//     N = 2^14, so that 512 threads of 128 registers hold them), radix-16 Stockham passes and
//     one pass of radix 2^(LOGN mod 4), in shared memory;
//   - the samples and window taps arrive by vector loads of 16 consecutive samples per
//     thread (inputs and window 16-byte aligned: the host routes other calls to the kernels
//     for any N);
//   - the per-CTA partial sums over the CTA's segments (per bin in the forward pass, per tap
//     in the window pass) stay in tensor memory, used as per-thread storage, and reach global
//     memory once, at the end (instead of a read and a write per segment);
//   - the twiddles of the passes with Ns <= 256 are a shared-memory copy of the host's table
//     (exact FP64 values rounded once); the last pass of N >= 2^13 (Ns = 4096) forms
//     W_N^{r j}, j = t + q T, as W_N^{r t} (from the table, once per thread) times the
//     constant W_PPT^{r q}: one rounding of two correctly rounded factors.
#include <cuda_runtime.h>

#include <algorithm>

#include "polaris_adjoint.cuh"
#include "polaris_kernels.cuh"  // tensor-memory helpers

namespace polaris {

template <int LOGN>
struct AdjPlan {
  static constexpr int N = 1 << LOGN, PPT = LOGN >= 14 ? 32 : 16, T = N / PPT, WARPS = T / 32, NBIN = N / 2 + 1;
  static constexpr int BPT = PPT / 2 + 1;  // bins per thread: k = t + T i (i < PPT/2), and N/2 for t = 0
  static constexpr int F = LOGN / 4, REM = LOGN % 4;     // F radix-16 passes, then one of radix 2^REM
  static constexpr int NS_LAST = 1 << (4 * F);           // Ns of that last pass
  static constexpr bool FLY = REM > 0 && NS_LAST > 256;  // its twiddles formed in registers
  static constexpr int RW = (REM > 0 ? (1 << REM) : 2) - 1;  // W_N^{r t}, r = 1 .. radix - 1, per thread
  static constexpr int NTAB = FLY ? NS_LAST - 1 : N - 1; // twiddle-table entries in shared memory
  static constexpr int DATA = adj_smem_points(N);
  static constexpr int SLOTS = WARPS >= 4 ? WARPS / 4 : 1;  // warps sharing a tensor-memory lane quadrant
  // tensor-memory columns per thread: forward, BPT bins x 4 sums in groups of 16 (four bins
  // each); window pass, the PPT taps of its sample groups
  static constexpr int FCOLS = 16 * ((4 * BPT + 15) / 16), WCOLS = PPT;
  static constexpr int TCOLS_F = pow2_at_least(SLOTS * FCOLS, 32), TCOLS_W = pow2_at_least(SLOTS * WCOLS, 32);
  static constexpr size_t SMEM = (size_t)(DATA + NTAB) * sizeof(float2) + 16;
  static_assert(T % 32 == 0 && (N / 2) / T == PPT / 2, "whole warps, PPT/2 bins per thread below N/2");
  static_assert(TCOLS_F <= 512 && TCOLS_W <= 512, "tensor memory");
};

// One Stockham pass of radix R with Ns = NS points already combined: every j < N/R reads
// z[j + r N/R] (r < R), multiplies by W_{NS R}^{r (j mod NS)}, takes an R-point DFT and writes
// output r to z[(j / NS) NS R + r NS + j mod NS].  All reads come before any write.
// Every compile-time part of the indices below (q T, r M, r NS) is a multiple of 16, so
// apad(x + c) = apad(x) + c + c/16: one padded base per lane and j, compile-time offsets.
template <int C>
__device__ __forceinline__ constexpr int apad_c() {
  static_assert(C % 16 == 0, "offset of whole 16-point groups");
  return C + C / 16;
}
template <int LOGN, int R, int NS>
__device__ __forceinline__ void adjs_pass(float2* z, const float2* __restrict__ tws,
                                          const float2 (&wt)[AdjPlan<LOGN>::RW], int tid) {
  using PL = AdjPlan<LOGN>;
  constexpr int T = PL::T, JPT = PL::PPT / R, M = PL::N / R;
  float2 v[JPT][R];
  const float2* zt = z + apad(tid);
  sfor<0, JPT>([&](auto q_) {
    constexpr int q = decltype(q_)::value;
    const int j = tid + q * T;
    const int k = j & (NS - 1);
    sfor<0, R>([&](auto r_) {
      constexpr int r = decltype(r_)::value;
      float2 x = zt[apad_c<q * T + r * M>()];  // z[apad(j + r M)]
      if constexpr (NS > 1 && r > 0) {
        if constexpr (NS <= 256) {
          x = cmul(x, tws[r * NS + k - 1]);
        } else {  // the last pass: k = j, W_N^{r j} = W_N^{r t} W_PPT^{r q} (T = N/PPT)
          constexpr int e = (r * q) % PL::PPT;
          float2 w = wt[r - 1];
          if constexpr (e != 0) {
            constexpr ct::CS cs = ct::cossin2pi(e, PL::PPT);
            w = cmul(w, make_float2((float)cs.c, (float)(-cs.s)));
          }
          x = cmul(x, w);
        }
      }
      v[q][ct::bitrev(r, R)] = x;
    });
  });
  __syncthreads();
  sfor<0, JPT>([&](auto q_) {
    constexpr int q = decltype(q_)::value;
    const int j = tid + q * T;
    dit<R>(v[q]);
    if constexpr (NS == 1) {  // base = 16 j, outputs r < 16: apad(16 j + r) = 17 j + r
      sfor<0, R>([&](auto r_) {
        constexpr int r = decltype(r_)::value;
        z[17 * j + r] = v[q][r];
      });
    } else {
      const int k = j & (NS - 1);
      float2* zb = z + apad((j - k) * R + k);
      sfor<0, R>([&](auto r_) {
        constexpr int r = decltype(r_)::value;
        zb[apad_c<r * NS>()] = v[q][r];  // z[apad(base + r NS)]
      });
    }
  });
  __syncthreads();
}

// forward DFT of the N points in z (natural order in and out); callers sync before
template <int LOGN>
__device__ __forceinline__ void adjs_fft(float2* z, const float2* __restrict__ tws,
                                         const float2 (&wt)[AdjPlan<LOGN>::RW], int tid) {
  using PL = AdjPlan<LOGN>;
  sfor<0, PL::F>([&](auto p_) { adjs_pass<LOGN, 16, (1 << (4 * decltype(p_)::value))>(z, tws, wt, tid); });
  if constexpr (PL::REM > 0) adjs_pass<LOGN, (1 << PL::REM), PL::NS_LAST>(z, tws, wt, tid);
}

// The levels of the 16 consecutive samples 16 g .. 16 g + 15 of segment s of one IF, from
// one vector load (16 B at 8 bits, 8 B at 4, 4 B at 2, 2 B at 1 bit; the caller guarantees
// 16-byte aligned inputs).  Sample i of a word sits at bits i BITS .. (i + 1) BITS - 1.
template <int LOGN, int BITS>
__device__ __forceinline__ void adjs_group_levels(const uint32_t* in, long long s, int g, float (&x)[16]) {
  const long long first = s * (1LL << LOGN) + 16LL * g;  // a multiple of 16 samples
  if constexpr (BITS == 8) {
    const int4 v = __ldg(reinterpret_cast<const int4*>(reinterpret_cast<const signed char*>(in) + first));
    const int w[4] = {v.x, v.y, v.z, v.w};
    sfor<0, 16>([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      x[i] = (float)((w[i / 4] << (24 - 8 * (i % 4))) >> 24);  // the byte, sign-extended
    });
  } else if constexpr (BITS == 4) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(in) + first / 16);
    sfor<0, 16>([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      x[i] = decode_level<4>(i < 8 ? v.x : v.y, (uint32_t)(i % 8) * 4);
    });
  } else if constexpr (BITS == 2) {
    const uint32_t v = __ldg(in + first / 16);
    sfor<0, 16>([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      x[i] = decode_level<2>(v, (uint32_t)i * 2);
    });
  } else {
    const uint32_t v = __ldg(reinterpret_cast<const unsigned short*>(in) + first / 16);
    sfor<0, 16>([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      x[i] = decode_level<1>(v, (uint32_t)i);
    });
  }
}

// z[n] = w[n] (x[n] + i y[n]) for segment s: thread t fills the groups g = t + T h (h <
// PPT/16) of 16 consecutive samples; apad(16 g + j) = 17 g + j, so the 16 lanes of a
// half-warp write distinct bank pairs
template <int LOGN, int BITS>
__device__ __forceinline__ void adjs_load(const AdjArgs& a, float2* z, long long s, int tid) {
  using PL = AdjPlan<LOGN>;
  sfor<0, PL::PPT / 16>([&](auto h_) {
    const int g = tid + decltype(h_)::value * PL::T;
    float x[16], y[16];
    adjs_group_levels<LOGN, BITS>(a.in[0], s, g, x);
    adjs_group_levels<LOGN, BITS>(a.in[1], s, g, y);
    const float4* wp = reinterpret_cast<const float4*>(a.window) + 4 * g;
    sfor<0, 4>([&](auto c_) {
      constexpr int c = decltype(c_)::value;
      const float4 w4 = __ldg(wp + c);
      const float w[4] = {w4.x, w4.y, w4.z, w4.w};
      sfor<0, 4>([&](auto i_) {
        constexpr int j = 4 * c + decltype(i_)::value;
        z[17 * g + j] = make_float2(w[j % 4] * x[j], w[j % 4] * y[j]);
      });
    });
  });
}

// the set-up both kernels share: the twiddle table in shared memory, this thread's W_N^{r t}
// for a last pass formed in registers, and the CTA's tensor memory (this thread's COLS columns
// zeroed); returns the address of those columns
template <int LOGN, int TCOLS, int COLS>
__device__ __forceinline__ uint32_t adjs_setup(const AdjArgs& a, float2* tws, uint32_t* tslot,
                                               float2 (&wt)[AdjPlan<LOGN>::RW], uint32_t& tbase, int tid) {
  using PL = AdjPlan<LOGN>;
  const int warp = tid >> 5;
  for (int i = tid; i < PL::NTAB; i += PL::T) tws[i] = __ldg(a.tw + i);
  sfor<0, PL::RW>([&](auto r_) {  // W_N^{r t}: the table's entry r, k = t of the last pass
    constexpr int r = decltype(r_)::value + 1;
    wt[r - 1] = PL::FLY ? __ldg(a.tw + r * PL::NS_LAST + tid - 1) : make_float2(1.f, 0.f);
  });
  tbase = cta_tmem_begin<TCOLS>(tslot, warp);  // (its barrier also publishes the table)
  const uint32_t tacc = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * COLS);
  float z16[16];
  sfor<0, 16>([&](auto i_) { z16[decltype(i_)::value] = 0.f; });
  sfor<0, COLS / 16>([&](auto c_) { tmem_st16(tacc + 16 * decltype(c_)::value, z16); });
  tmem_wait_st();
  return tacc;
}

template <int LOGN, int BITS>
__global__ void __launch_bounds__(AdjPlan<LOGN>::T) k_adjs_forward(AdjArgs a) {
  using PL = AdjPlan<LOGN>;
  constexpr int N = PL::N, T = PL::T;
  extern __shared__ __align__(16) float2 zs[];
  float2* z = zs;
  float2* tws = zs + PL::DATA;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tws + PL::NTAB);
  const int tid = threadIdx.x;
  float2 wt[PL::RW];
  uint32_t tbase;
  const uint32_t tacc = adjs_setup<LOGN, PL::TCOLS_F, PL::FCOLS>(a, tws, tslot, wt, tbase, tid);
#pragma unroll 1
  for (long long s = blockIdx.x; s < a.nseg; s += a.grid) {
    adjs_load<LOGN, BITS>(a, z, s, tid);
    __syncthreads();
    adjs_fft<LOGN>(z, tws, wt, tid);
    // X = (Z[k] + conj Z[N-k]) / 2, Y = (Z[k] - conj Z[N-k]) / 2i; the sums of bin i of this
    // thread at columns 4 i .. 4 i + 3
    sfor<0, PL::FCOLS / 16>([&](auto c_) {
      constexpr int cc = decltype(c_)::value;
      float acc[16];
      tmem_ld16(tacc + 16 * cc, acc);
      tmem_wait_ld();
      sfor<0, 4>([&](auto i_) {
        constexpr int i = 4 * cc + decltype(i_)::value;
        if constexpr (i < PL::BPT) {
          if (i < PL::BPT - 1 || tid == 0) {
            const int k = i < PL::BPT - 1 ? tid + T * i : N / 2;
            const float2 Zk = z[apad(k)], Zm = c_conj(z[apad((N - k) & (N - 1))]);
            const float2 X = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y + Zm.y));
            const float2 Y = make_float2(0.5f * (Zk.y - Zm.y), -0.5f * (Zk.x - Zm.x));
            constexpr int o = 4 * (i - 4 * cc);
            acc[o + 0] += fmaf(X.x, X.x, X.y * X.y);
            acc[o + 1] += fmaf(Y.x, Y.x, Y.y * Y.y);
            acc[o + 2] += fmaf(X.x, Y.x, X.y * Y.y);
            acc[o + 3] += fmaf(X.y, Y.x, -X.x * Y.y);
          }
        }
      });
      tmem_st16(tacc + 16 * cc, acc);
    });
    tmem_wait_st();
    __syncthreads();  // z is refilled by the next segment
  }
  float4* part = a.part + (size_t)blockIdx.x * PL::NBIN;
  sfor<0, PL::FCOLS / 16>([&](auto c_) {
    constexpr int cc = decltype(c_)::value;
    float acc[16];
    tmem_ld16(tacc + 16 * cc, acc);
    tmem_wait_ld();
    sfor<0, 4>([&](auto i_) {
      constexpr int i = 4 * cc + decltype(i_)::value;
      if constexpr (i < PL::BPT) {
        if (i < PL::BPT - 1 || tid == 0) {
          const int k = i < PL::BPT - 1 ? tid + T * i : N / 2;
          constexpr int o = 4 * (i - 4 * cc);
          part[k] = make_float4(acc[o], acc[o + 1], acc[o + 2], acc[o + 3]);
        }
      }
    });
  });
  cta_tmem_end<PL::TCOLS_F>(tbase, tid >> 5);
}

template <int LOGN, int BITS>
__global__ void __launch_bounds__(AdjPlan<LOGN>::T) k_adjs_window(AdjArgs a) {
  using PL = AdjPlan<LOGN>;
  constexpr int N = PL::N, T = PL::T;
  extern __shared__ __align__(16) float2 zs[];
  float2* z = zs;
  float2* tws = zs + PL::DATA;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tws + PL::NTAB);
  const int tid = threadIdx.x;
  float2 wt[PL::RW];
  uint32_t tbase;
  const uint32_t tacc = adjs_setup<LOGN, PL::TCOLS_W, PL::WCOLS>(a, tws, tslot, wt, tbase, tid);
#pragma unroll 1
  for (long long s = blockIdx.x; s < a.nseg; s += a.grid) {
    adjs_load<LOGN, BITS>(a, z, s, tid);
    __syncthreads();
    adjs_fft<LOGN>(z, tws, wt, tid);
    // G_X, G_Y per bin pair; conj of the Hermitian extension of G_X + i G_Y goes back into z
    // (the inverse transform is conj(DFT(conj H))).  This thread owns slots k and N - k.
#pragma unroll 1
    for (int k = tid; k < PL::NBIN; k += T) {  // (rolled: unrolled, its loads crowd the registers)
      {
        const int km = (N - k) & (N - 1);
        const float2 Zk = z[apad(k)], Zm = c_conj(z[apad(km)]);
        const float2 X = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y + Zm.y));
        const float2 Y = make_float2(0.5f * (Zk.y - Zm.y), -0.5f * (Zk.x - Zm.x));
        const float4 r0 = __ldg(a.mat + 2 * k), r1 = __ldg(a.mat + 2 * k + 1);
        const float2 GX = c_add(cmul(make_float2(r0.x, r0.y), X), cmul(make_float2(r0.z, r0.w), Y));
        const float2 GY = c_add(cmul(make_float2(r1.x, r1.y), X), cmul(make_float2(r1.z, r1.w), Y));
        if (k == 0 || 2 * k == N) {
          z[apad(k)] = make_float2(GX.x, -GY.x);  // H = Re G_X + i Re G_Y
        } else {
          const float2 hx = make_float2(0.5f * GX.x, 0.5f * GX.y), hy = make_float2(0.5f * GY.x, 0.5f * GY.y);
          // H[k] = hx + i hy, H[N-k] = conj(hx) + i conj(hy); store their conjugates
          z[apad(k)] = make_float2(hx.x - hy.y, -(hx.y + hy.x));
          z[apad(km)] = make_float2(hx.x + hy.y, hx.y - hy.x);
        }
      }
    }
    __syncthreads();
    adjs_fft<LOGN>(z, tws, wt, tid);
    // h = conj(F): dL/dw[n] += x[n] Re h[n] + y[n] Im h[n] = x F.x - y F.y
    // (this thread's taps are the samples of its groups: column 16 h + j holds n = 16 g + j)
    sfor<0, PL::PPT / 16>([&](auto h_) {
      constexpr int h = decltype(h_)::value;
      const int g = tid + h * T;
      float x[16], y[16];
      adjs_group_levels<LOGN, BITS>(a.in[0], s, g, x);
      adjs_group_levels<LOGN, BITS>(a.in[1], s, g, y);
      float acc[16];
      tmem_ld16(tacc + 16 * h, acc);
      tmem_wait_ld();
      sfor<0, 16>([&](auto j_) {
        constexpr int j = decltype(j_)::value;
        const float2 F = z[17 * g + j];
        acc[j] += fmaf(x[j], F.x, -y[j] * F.y);
      });
      tmem_st16(tacc + 16 * h, acc);
    });
    tmem_wait_st();
    __syncthreads();
  }
  float* gpart = a.gpart + (size_t)blockIdx.x * N;
  sfor<0, PL::PPT / 16>([&](auto h_) {
    constexpr int h = decltype(h_)::value;
    const int g = tid + h * T;
    float acc[16];
    tmem_ld16(tacc + 16 * h, acc);
    tmem_wait_ld();
    sfor<0, 4>([&](auto c_) {
      constexpr int c = decltype(c_)::value;
      reinterpret_cast<float4*>(gpart + 16 * g)[c] = make_float4(acc[4 * c], acc[4 * c + 1], acc[4 * c + 2], acc[4 * c + 3]);
    });
  });
  cta_tmem_end<PL::TCOLS_W>(tbase, tid >> 5);
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
template <int LOGN, int BITS>
static cudaError_t adjs_prepare(int* ctas_per_sm) {
  using PL = AdjPlan<LOGN>;
  const int smem = (int)PL::SMEM;
  cudaError_t e = cudaFuncSetAttribute(k_adjs_forward<LOGN, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adjs_window<LOGN, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int o1 = 0, o2 = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_adjs_forward<LOGN, BITS>, PL::T, PL::SMEM);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_adjs_window<LOGN, BITS>, PL::T, PL::SMEM);
  // CTAs that share an SM must find their tensor memory free (512 columns per SM)
  *ctas_per_sm = std::min(std::min(o1, o2), 512 / std::max(PL::TCOLS_F, PL::TCOLS_W));
  return e;
}

template <int LOGN, int BITS>
static cudaError_t adjs_launch(bool window_pass, const AdjArgs& a, cudaStream_t st) {
  using PL = AdjPlan<LOGN>;
  if (!window_pass) k_adjs_forward<LOGN, BITS><<<a.grid, PL::T, PL::SMEM, st>>>(a);
  else k_adjs_window<LOGN, BITS><<<a.grid, PL::T, PL::SMEM, st>>>(a);
  return cudaGetLastError();
}

template <int LOGN>
static cudaError_t adjs_dispatch(int bits, bool prepare, int* occ, bool window_pass, const AdjArgs* a,
                                 cudaStream_t st) {
  switch (bits) {
    case 1: return prepare ? adjs_prepare<LOGN, 1>(occ) : adjs_launch<LOGN, 1>(window_pass, *a, st);
    case 2: return prepare ? adjs_prepare<LOGN, 2>(occ) : adjs_launch<LOGN, 2>(window_pass, *a, st);
    case 4: return prepare ? adjs_prepare<LOGN, 4>(occ) : adjs_launch<LOGN, 4>(window_pass, *a, st);
    default: return prepare ? adjs_prepare<LOGN, 8>(occ) : adjs_launch<LOGN, 8>(window_pass, *a, st);
  }
}

static cudaError_t adjs_any(int log2n, int bits, bool prepare, int* occ, bool window_pass, const AdjArgs* a,
                            cudaStream_t st) {
  switch (log2n) {
    case 9: return adjs_dispatch<9>(bits, prepare, occ, window_pass, a, st);
    case 10: return adjs_dispatch<10>(bits, prepare, occ, window_pass, a, st);
    case 11: return adjs_dispatch<11>(bits, prepare, occ, window_pass, a, st);
    case 12: return adjs_dispatch<12>(bits, prepare, occ, window_pass, a, st);
    case 13: return adjs_dispatch<13>(bits, prepare, occ, window_pass, a, st);
    case 14: return adjs_dispatch<14>(bits, prepare, occ, window_pass, a, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t adj_sized_prepare(int log2n, int bits, int* ctas_per_sm) {
  return adjs_any(log2n, bits, true, ctas_per_sm, false, nullptr, nullptr);
}

cudaError_t adj_sized_launch(int log2n, int bits, bool window_pass, const AdjArgs& a, cudaStream_t st) {
  return adjs_any(log2n, bits, false, nullptr, window_pass, &a, st);
}

}  // namespace polaris
