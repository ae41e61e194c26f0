// Hot-path kernels (sm_103a), templated on log2(N):
//
//   k_phase1  data translation (codes -> levels, Fig. 2 caption), window (Sec. 3.1),
//             first half of the segment FFT: for every column b of n = N2 a + b a DFT of
//             length N1 over the rows a, done in registers (P points per thread) with one
//             transpose through shared memory.  Writes the N complex partial transforms of
//             each pair-segment to an L2-resident scratch slab, row b contiguous in c.
//
//   k_phase2  second half of the FFT and the correlator (Fig. 1 caption: XX*, YY*, XY*;
//             Table 1; accumulation over the integration): for every output column c the
//             twiddle W_N^{b c} and a DFT of length N2 over b, again in registers with one
//             shared-memory transpose.  Column c and its mirror N1 - c are transformed
//             together (the mirror conjugated), so each thread ends with Z_k and
//             conj(Z_{N-k}) of the packed pair z = x + i y, from which
//               2 X_k = Z_k + conj(Z_{N-k}),  2i Y_k = Z_k - conj(Z_{N-k}).
//             |X|^2, |Y|^2 and X conj(Y) are accumulated in registers over all segments
//             of the tile and added once to the integration accumulators: no per-segment
//             spectrum is written to memory.
#pragma once
#include <cuda_runtime.h>

#include "polaris_device.cuh"

namespace polaris {

// W_1024^k = e^{-2 pi i k / 1024}, k in [0, 1024), from the compile-time series.
struct TwTable {
  float2 v[1024];
};
constexpr TwTable make_tw1024() {
  TwTable t{};
  for (int k = 0; k < 1024; ++k) {
    const ct::CS cs = ct::cossin2pi(k, 1024);
    t.v[k].x = (float)cs.c;
    t.v[k].y = (float)(-cs.s);
  }
  return t;
}
static __constant__ TwTable c_tw = make_tw1024();

// twiddle W_L^k for L <= 1024 (power of two), k any integer
template <int L>
__device__ __forceinline__ float2 tw_small(int k) {
  return c_tw.v[(k & (L - 1)) * (1024 / L)];
}

constexpr int kMaxIF = 8;

// Where segment s of the current feed starts, per IF: segments [0, n0) in src0 (the staging
// copy that joins carried samples to the new ones), the rest in src1 (the new data).
struct SegSrc {
  const uint32_t* src0[kMaxIF];
  const uint32_t* src1[kMaxIF];
  long long hop_w;  // 32-bit words between segment starts
  int n0;
};

struct BatchArgs {
  SegSrc in;
  int fa[kMaxIF];  // FFT pair f transforms IF fa[f] (real part) and IF fb[f] (imag part; < 0: zero)
  int fb[kMaxIF];
  int n_fpair;
  int seg0;             // first feed segment of this batch
  int nseg;             // segments in this batch
  const float* taps;    // window taps (N) or nullptr for the rectangular window
  float2* scratch;      // [nseg * n_fpair][N2][N1]
  const float2* tw;     // [N2][UPS + 1]: W_N^{b u}
  void* acc;            // native accumulators [n_fpair][N/2 + 1] of float4 (or double4 if fp64)
  int fp64;
  int bits;
  int num_sms;
};

__device__ __forceinline__ const uint32_t* seg_ptr(const SegSrc& in, int ifx, int s) {
  return s < in.n0 ? in.src0[ifx] + (long long)s * in.hop_w : in.src1[ifx] + (long long)(s - in.n0) * in.hop_w;
}

// ------------------------------------------------------------------------------------------
// phase 1
// ------------------------------------------------------------------------------------------
template <int LOGN, int BITS>
__device__ __forceinline__ void p1_load(const BatchArgs& a, int g, int b, int q1, float2 (&v)[Plan<LOGN>::P]) {
  using PL = Plan<LOGN>;
  constexpr int P = PL::P, N2 = PL::N2, Q1 = PL::Q1;
  const int s_local = g / a.n_fpair, f = g - s_local * a.n_fpair;
  const int s = a.seg0 + s_local;
  const int ia = a.fa[f], ib = a.fb[f];
  const uint32_t* pa = seg_ptr(a.in, ia, s);
  const uint32_t* pb = ib >= 0 ? seg_ptr(a.in, ib, s) : nullptr;
  const float* taps = a.taps;
  const uint32_t base = (uint32_t)(N2 * q1 + b);  // sample index of t = 0 within the segment
  sfor<0, P>([&](auto t_) {
    constexpr int t = decltype(t_)::value;
    const uint32_t n = base + (uint32_t)(N2 * Q1 * t);
    uint32_t word_i, shift;
    if constexpr (((long)N2 * Q1 * BITS) % 32 == 0) {
      word_i = ((base * BITS) >> 5) + (uint32_t)(((long)N2 * Q1 * BITS / 32) * t);
      shift = (base * BITS) & 31u;
    } else {
      word_i = (n * BITS) >> 5;
      shift = (n * BITS) & 31u;
    }
    float x = decode_level<BITS>(__ldg(pa + word_i), shift);
    float y = pb ? decode_level<BITS>(__ldg(pb + word_i), shift) : 0.0f;
    if (taps) {
      const float wv = __ldg(taps + n);
      x *= wv;
      y *= wv;
    }
    v[ct::bitrev(t, P)] = make_float2(x, y);
  });
}

template <int LOGN, int BITS>
__global__ void __launch_bounds__(Plan<LOGN>::T1, 1) k_phase1(BatchArgs a) {
  using PL = Plan<LOGN>;
  constexpr int P = PL::P, N1 = PL::N1, N2 = PL::N2, Q1 = PL::Q1, W = PL::W, LD = PL::S1_LD;
  extern __shared__ float2 sm1[];
  const int tid = threadIdx.x;
  const long long total_cols = (long long)a.nseg * a.n_fpair * N2;
  {
    const int q1 = tid / W, w = tid % W;
    const long long gc = (long long)blockIdx.x * W + w;
    float2 v[P];
    if (gc < total_cols) {
      p1_load<LOGN, BITS>(a, (int)(gc / N2), (int)(gc % N2), q1, v);
    } else {
      sfor<0, P>([&](auto t_) { v[decltype(t_)::value] = make_float2(0.f, 0.f); });
    }
    dit<P>(v);
    if constexpr (Q1 > 1) {
      sfor<1, P>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        v[p] = cmul(v[p], tw_small<N1>(q1 * p));
      });
    }
    sfor<0, P>([&](auto p_) {
      constexpr int p = decltype(p_)::value;
      sm1[(q1 * P + p) * LD + w] = v[p];
    });
  }
  __syncthreads();
  {
    constexpr int CPT = P / Q1;  // columns per thread in the second step
    const int p = tid % P, wg = tid / P;
    sfor<0, CPT>([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      const int w = wg * CPT + i;
      const long long gc = (long long)blockIdx.x * W + w;
      float2 u[Q1];
      sfor<0, Q1>([&](auto q_) {
        constexpr int q = decltype(q_)::value;
        u[ct::bitrev(q, Q1)] = sm1[(q * P + p) * LD + w];
      });
      dit<Q1>(u);
      if (gc < total_cols) {
        const long long g = gc / N2, b = gc % N2;
        float2* dst = a.scratch + ((size_t)g * N2 + b) * N1 + p;
        sfor<0, Q1>([&](auto m_) {
          constexpr int m = decltype(m_)::value;
          dst[m * P] = u[m];
        });
      }
    });
  }
}

// ------------------------------------------------------------------------------------------
// phase 2
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void corr_acc(float (&acc)[4], float2 U, float2 V) {
  // S = 2X, D = 2iY;  |S|^2, |D|^2, Re/Im of i S conj(D) (= 4 X conj(Y))
  const float sx = U.x + V.x, sy = U.y + V.y, dx = U.x - V.x, dy = U.y - V.y;
  acc[0] = fmaf(sx, sx, fmaf(sy, sy, acc[0]));
  acc[1] = fmaf(dx, dx, fmaf(dy, dy, acc[1]));
  acc[2] = fmaf(sx, dy, fmaf(-sy, dx, acc[2]));
  acc[3] = fmaf(sx, dx, fmaf(sy, dy, acc[3]));
}

template <int LOGN>
__global__ void __launch_bounds__(Plan<LOGN>::T2, 1) k_phase2(BatchArgs a, int seg_per_tile, int n_chunks) {
  using PL = Plan<LOGN>;
  constexpr int P = PL::P, N1 = PL::N1, N2 = PL::N2, Q2 = PL::Q2, U = PL::U, UPS = PL::UPS;
  constexpr int SLOTS = PL::SLOTS, NUB = PL::NUB, PP = PL::PP, NACC = PL::NACC, LD = PL::S2_LD;
  extern __shared__ float2 sm2[];
  float2* sp = sm2 + Q2 * P * LD;  // mirror area for the special unit: [SLOTS][2][N2]
  const int tid = threadIdx.x;

  const int chunk = blockIdx.x % n_chunks;
  const int fub = blockIdx.x / n_chunks;
  const int ub = fub % NUB, f = fub / NUB;
  const int s_begin = chunk * seg_per_tile;
  const int s_end = min(a.nseg, s_begin + seg_per_tile);

  // step-1 mapping: lanes over the tile's 2U columns, q2 over warps
  const int col = tid % (2 * U), q2 = tid / (2 * U);
  const int e1 = col / U, i1 = col % U;
  const int so1 = (U > UPS) ? i1 / UPS : 0;
  const int u1 = (U > UPS) ? i1 % UPS : ub * U + i1;
  const int c1 = (u1 == 0) ? (e1 ? N1 / 2 : 0) : (e1 ? N1 - u1 : u1);
  const int tu1 = (u1 == 0 && e1) ? N1 / 2 : u1;
  const bool cj1 = e1 && u1 != 0;
  // step-2 mapping: one unit per 2 Q2 threads, p-values j2 * PP + r
  const int j2 = tid % (2 * Q2), i2 = tid / (2 * Q2);
  const int so2 = (U > UPS) ? i2 / UPS : 0;
  const int u2 = (U > UPS) ? i2 % UPS : ub * U + i2;
  const bool special2 = (u2 == 0);
  const bool tile_special = (U > UPS) || (ub == 0);

  float acc[NACC][4];
  float extra[4] = {0.f, 0.f, 0.f, 0.f};
  sfor<0, NACC>([&](auto k_) {
    constexpr int k = decltype(k_)::value;
    acc[k][0] = acc[k][1] = acc[k][2] = acc[k][3] = 0.f;
  });

  const int n_iter = (s_end - s_begin + SLOTS - 1) / SLOTS;
  for (int it = 0; it < n_iter; ++it) {
    {
      const int s = s_begin + it * SLOTS + so1;
      const bool act = s < s_end;
      const float2* src = a.scratch + ((size_t)(act ? s : 0) * a.n_fpair + f) * N2 * N1 + c1;
      const float2* twp = a.tw + tu1;
      float2 v[P];
      sfor<0, P>([&](auto t_) {
        constexpr int t = decltype(t_)::value;
        const int b = q2 + Q2 * t;
        const float2 z = act ? __ldcg(src + (size_t)b * N1) : make_float2(0.f, 0.f);
        const float2 w = __ldg(twp + b * (UPS + 1));
        v[ct::bitrev(t, P)] = cj1 ? cmulc(z, w) : cmul(z, w);
      });
      dit<P>(v);
      if constexpr (Q2 > 1) {
        sfor<1, P>([&](auto p_) {
          constexpr int p = decltype(p_)::value;
          v[p] = cmul(v[p], tw_small<N2>(q2 * p));
        });
      }
      __syncthreads();  // previous iteration's readers are done with sm2
      sfor<0, P>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        sm2[(q2 * P + p) * LD + col] = v[p];
      });
    }
    __syncthreads();
    // step 2: DFT-Q2 for both members (e) of the unit and PP p-values
    float2 wv[2 * PP * Q2];
    sfor<0, 2>([&](auto e_) {
      constexpr int e = decltype(e_)::value;
      sfor<0, PP>([&](auto r_) {
        constexpr int r = decltype(r_)::value;
        const int p = j2 * PP + r;
        sfor<0, Q2>([&](auto q_) {
          constexpr int q = decltype(q_)::value;
          wv[(e * PP + r) * Q2 + ct::bitrev(q, Q2)] = sm2[(q * P + p) * LD + e * U + i2];
        });
        dit<Q2, (e * PP + r) * Q2, 1>(wv);
      });
    });
    const int s2 = s_begin + it * SLOTS + so2;
    const bool act2 = s2 < s_end;
    if (tile_special) {  // uniform per tile
      if (special2) {
        sfor<0, 2>([&](auto e_) {
          constexpr int e = decltype(e_)::value;
          sfor<0, PP>([&](auto r_) {
            constexpr int r = decltype(r_)::value;
            sfor<0, Q2>([&](auto m_) {
              constexpr int m = decltype(m_)::value;
              const int d = j2 * PP + r + P * m;
              sp[(so2 * 2 + e) * N2 + d] = wv[(e * PP + r) * Q2 + m];
            });
          });
        });
      }
      __syncthreads();
    }
    if (act2) {
      if (!special2) {
        sfor<0, PP>([&](auto r_) {
          constexpr int r = decltype(r_)::value;
          sfor<0, Q2>([&](auto m_) {
            constexpr int m = decltype(m_)::value;
            corr_acc(acc[r * Q2 + m], wv[r * Q2 + m], wv[(PP + r) * Q2 + m]);
          });
        });
      } else {
        const float2* s0 = sp + (so2 * 2 + 0) * N2;  // column 0
        const float2* sh = sp + (so2 * 2 + 1) * N2;  // column N1/2
        sfor<0, PP>([&](auto r_) {
          constexpr int r = decltype(r_)::value;
          sfor<0, Q2>([&](auto m_) {
            constexpr int m = decltype(m_)::value;
            const int d = j2 * PP + r + P * m;
            float2 Uv, Vv;
            if (d <= N2 / 2) {  // column 0: bins N1 d, mirror N1 (N2 - d)
              Uv = s0[d];
              const float2 t = s0[(N2 - d) & (N2 - 1)];
              Vv = make_float2(t.x, -t.y);
            } else {  // column N1/2 at dh = d - N2/2 - 1: bins N1/2 + N1 dh, mirror dh' = N2 - 1 - dh
              const int dh = d - N2 / 2 - 1;
              Uv = sh[dh];
              const float2 t = sh[N2 - 1 - dh];
              Vv = make_float2(t.x, -t.y);
            }
            corr_acc(acc[r * Q2 + m], Uv, Vv);
          });
        });
        if (j2 == 0) {  // the one extra bin: column N1/2 at dh = N2/2 - 1
          const float2 t = sh[N2 / 2];
          corr_acc(extra, sh[N2 / 2 - 1], make_float2(t.x, -t.y));
        }
      }
    }
  }

  // flush: one atomic add per bin into the integration accumulators (native order)
  const bool had_work = (s_begin + so2) < s_end;
  if (!had_work) return;
  const size_t base = (size_t)f * PL::NATIVE;
  if (!a.fp64) {
    float4* accp = reinterpret_cast<float4*>(a.acc) + base;
    sfor<0, PP>([&](auto r_) {
      constexpr int r = decltype(r_)::value;
      sfor<0, Q2>([&](auto m_) {
        constexpr int m = decltype(m_)::value;
        const int d = j2 * PP + r + P * m;
        const float* q = acc[r * Q2 + m];
        atomicAdd(accp + (size_t)u2 * N2 + d, make_float4(q[0], q[1], q[2], q[3]));
      });
    });
    if (special2 && j2 == 0) atomicAdd(accp + (size_t)UPS * N2, make_float4(extra[0], extra[1], extra[2], extra[3]));
  } else {
    double* accp = reinterpret_cast<double*>(a.acc) + 4 * base;
    sfor<0, PP>([&](auto r_) {
      constexpr int r = decltype(r_)::value;
      sfor<0, Q2>([&](auto m_) {
        constexpr int m = decltype(m_)::value;
        const int d = j2 * PP + r + P * m;
        const float* q = acc[r * Q2 + m];
        double* o = accp + 4 * ((size_t)u2 * N2 + d);
        atomicAdd(o + 0, (double)q[0]);
        atomicAdd(o + 1, (double)q[1]);
        atomicAdd(o + 2, (double)q[2]);
        atomicAdd(o + 3, (double)q[3]);
      });
    });
    if (special2 && j2 == 0) {
      double* o = accp + 4 * (size_t)UPS * N2;
      atomicAdd(o + 0, (double)extra[0]);
      atomicAdd(o + 1, (double)extra[1]);
      atomicAdd(o + 2, (double)extra[2]);
      atomicAdd(o + 3, (double)extra[3]);
    }
  }
}

// ------------------------------------------------------------------------------------------
// host-side launcher for one batch of segments (instantiated once per N)
// ------------------------------------------------------------------------------------------
template <int LOGN, int BITS>
static cudaError_t launch_phase1(const BatchArgs& a, cudaStream_t st) {
  using PL = Plan<LOGN>;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k_phase1<LOGN, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::SMEM1);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  const long long cols = (long long)a.nseg * a.n_fpair * PL::N2;
  const int grid = (int)((cols + PL::W - 1) / PL::W);
  k_phase1<LOGN, BITS><<<grid, PL::T1, PL::SMEM1, st>>>(a);
  return cudaGetLastError();
}

// phase 1 of one batch
template <int LOGN>
cudaError_t run_phase1(const BatchArgs& a, cudaStream_t st) {
  if (a.nseg <= 0) return cudaSuccess;
  switch (a.bits) {
    case 1: return launch_phase1<LOGN, 1>(a, st);
    case 2: return launch_phase1<LOGN, 2>(a, st);
    case 4: return launch_phase1<LOGN, 4>(a, st);
    case 8: return launch_phase1<LOGN, 8>(a, st);
    default: return cudaErrorInvalidValue;
  }
}

// phase 2 of one batch: tiles = (FFT pair, unit block, chunk of segments), ~2 tiles per SM
template <int LOGN>
cudaError_t run_phase2(const BatchArgs& a, cudaStream_t st) {
  using PL = Plan<LOGN>;
  if (a.nseg <= 0) return cudaSuccess;
  static int attr_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k_phase2<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::SMEM2);
    if (e != cudaSuccess) return e;
    attr_dev = dev;
  }
  const int per_chunk_tiles = a.n_fpair * PL::NUB;
  const int max_chunks = (a.nseg + PL::SLOTS - 1) / PL::SLOTS;
  int want = (2 * a.num_sms + per_chunk_tiles - 1) / per_chunk_tiles;
  if (want < 1) want = 1;
  if (want > max_chunks) want = max_chunks;
  int seg_per_tile = (a.nseg + want - 1) / want;
  seg_per_tile = ((seg_per_tile + PL::SLOTS - 1) / PL::SLOTS) * PL::SLOTS;
  const int n_chunks = (a.nseg + seg_per_tile - 1) / seg_per_tile;
  k_phase2<LOGN><<<per_chunk_tiles * n_chunks, PL::T2, PL::SMEM2, st>>>(a, seg_per_tile, n_chunks);
  return cudaGetLastError();
}

}  // namespace polaris

#define POLARIS_INSTANTIATE(LOGN)                                                          \
  template cudaError_t polaris::run_phase1<LOGN>(const polaris::BatchArgs&, cudaStream_t); \
  template cudaError_t polaris::run_phase2<LOGN>(const polaris::BatchArgs&, cudaStream_t);
