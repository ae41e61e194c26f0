// Differentiable leakage calibration: forward model and hand-written adjoint.
//
// Model (ours: the paper calibrates gains offline, Sec. 2.1, and says nothing about
// polarisation leakage).  Two IFs R and L (circular feeds), segments of N samples at hop N,
// window w:
//   X_s[k] = sum_n w[n] x_s[n] e^{-2 pi i n k / N}, Y_s[k] likewise, k = 0..N/2
//   Xt = gR (X + DR[k] Y),  Yt = gL (Y + DL[k] X)
//   RR = sum_s |Xt|^2, LL = sum_s |Yt|^2, RL = sum_s Xt conj(Yt)
//   I = (RR + LL)/2, V = (RR - LL)/2, Q = Re RL, U = Im RL
//   loss = sum_k sum_S (S[k] - T_S[k])^2
//
// The mixing is linear per bin, so RR, LL and RL are quadratic forms of the plain sums
//   A = sum_s |X|^2, B = sum_s |Y|^2, C = sum_s X conj(Y):
//   P_R = sum|X + DR Y|^2 = A + |DR|^2 B + 2 Re(conj(DR) C)
//   P_L = sum|Y + DL X|^2 = B + |DL|^2 A + 2 Re(DL C)
//   Qm  = sum (X + DR Y) conj(Y + DL X) = C + conj(DL) A + DR B + DR conj(DL) conj(C)
//   RR = |gR|^2 P_R, LL = |gL|^2 P_L, RL = gR conj(gL) Qm.
// Gradients use G = dL/d re + i dL/d im for every complex parameter.  With r_S = 2 (S - T_S),
// a = (r_I + r_V)/2, b = (r_I - r_V)/2, c = r_Q + i r_U:
//   G_gR = sum_k 2a P_R gR + c gL conj(Qm)          G_gL = sum_k 2b P_L gL + conj(c) gR Qm
//   G_DR[k] = 2a |gR|^2 (B DR + C) + c conj(gR) gL (B + DL C)
//   G_DL[k] = 2b |gL|^2 (A DL + conj(C)) + conj(c) gR conj(gL) (A + DR conj(C))
// so neither needs the segments again.  The window does: per segment the spectral
// gradients are G_X = m11 X + m12 Y, G_Y = m21 X + m22 Y with a per-bin 2 x 2 matrix (from
// G_Xt = 2a Xt + c Yt, G_Yt = 2b Yt + conj(c) Xt pulled back through the mixing), and
//   dL/dw[n] = sum_s x_s[n] Re(sum_k G_X e^{+2 pi i n k/N}) + y_s[n] Re(sum_k G_Y e^{+...}),
// the real inverse transforms of the Hermitian extensions of G_X and G_Y, taken together
// as one complex inverse transform of H_X + i H_Y.  Segments are transformed again in the
// adjoint pass, not stored.
//
// Kernels (no atomics; every sum has a fixed order, so runs are bitwise reproducible):
//   k_adj_forward  a grid of G CTAs, each over segments b, b + G, ...: decode, window, a
//                  radix-16 Stockham transform of the pair x + i y in shared memory, split
//                  into X and Y, per-CTA partial sums of |X|^2, |Y|^2, X conj(Y)
//                  (N = 2^9 .. 2^14: k_adjs_forward, the same per size at compile time,
//                  polaris_adjoint_sized.cu; likewise k_adjs_window)
//   k_adj_bins     per bin: partials summed (fp32 slices, added in fp64), the model,
//                  Stokes and loss in fp64, the gain and leakage gradients and the
//                  window-adjoint matrix in fp32
//   k_adj_finish   block partials of the loss and gain gradients summed in order
//   k_adj_window   per segment again: forward transform, G_X and G_Y, inverse transform,
//                  per-CTA partials of the window gradient
//   k_adj_wsum     the window-gradient partials summed per tap
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/polaris.h"
#include "polaris_adjoint.cuh"

namespace polaris {

constexpr int kMaxCtasPerSm = 8;

// One Stockham autosort pass of radix R (Ns = product of the radices already applied), in
// place in z: every j < N/R reads z[j + r N/R] (r < R), multiplies by W_{Ns R}^{r (j mod Ns)}
// (from the pass's own table, where consecutive j read consecutive entries),
// takes an R-point DFT and writes output q to z[(j / Ns) Ns R + q Ns + j mod Ns].  All reads
// of the pass finish before any write.  The block has exactly T = N/16 threads and each
// holds 16 points: one j for R = 16, j = t, t + T, ... for smaller radices, always < N/R
// (a bounds test here would push the point arrays into local memory).
template <int R>
__device__ __forceinline__ void stockham_pass(float2* z, int N, int Ns, const float2* __restrict__ tw, int T) {
  constexpr int JPT = 16 / R;
  const int m = N / R;
  float2 v[JPT][R];
#pragma unroll
  for (int q = 0; q < JPT; ++q) {
    const int j = threadIdx.x + q * T;
    const int k = j & (Ns - 1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float2 a = z[apad(j + r * m)];
      if (r > 0 && Ns > 1) a = cmul(a, __ldg(tw + r * Ns + k - 1));
      v[q][ct::bitrev(r, R)] = a;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < JPT; ++q) {
    const int j = threadIdx.x + q * T;
    dit<R>(v[q]);
    const int k = j & (Ns - 1);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) z[apad(base + r * Ns)] = v[q][r];
  }
  __syncthreads();
}

// forward DFT of the N points in z (natural order in and out); callers sync before
__device__ __forceinline__ void adj_fft(float2* z, int N, int log2n, const float2* __restrict__ tw, int T) {
  int Ns = 1;
#pragma unroll 1
  for (int p = 0; p < (log2n >> 2); ++p, Ns <<= 4) stockham_pass<16>(z, N, Ns, tw, T);
  switch (log2n & 3) {
    case 1: stockham_pass<2>(z, N, Ns, tw, T); break;
    case 2: stockham_pass<4>(z, N, Ns, tw, T); break;
    case 3: stockham_pass<8>(z, N, Ns, tw, T); break;
    default: break;
  }
}

// z[n] = w[n] (x[n] + i y[n]) for segment s; thread t fills n = t + T e, e < 16, so that
// every load is coalesced and the stores are conflict-free
template <int BITS>
__device__ __forceinline__ void adj_load_segment(const AdjArgs& a, float2* z, long long s) {
  const long long base = s * a.N;
#pragma unroll 8
  for (int e = 0; e < 16; ++e) {
    const int n = threadIdx.x + e * a.threads;
    const float w = __ldg(a.window + n);
    z[apad(n)] = make_float2(w * adj_level<BITS>(a.in[0], base + n), w * adj_level<BITS>(a.in[1], base + n));
  }
}

// one segment of the forward pass
template <int BITS>
__device__ __forceinline__ void adj_forward_segment(const AdjArgs& a, float2* z, long long s, bool first) {
  const int N = a.N, nbin = a.nbin;
  float4* part = a.part + (size_t)blockIdx.x * nbin;
  adj_load_segment<BITS>(a, z, s);
  __syncthreads();
  adj_fft(z, N, a.log2n, a.tw, a.threads);
  // X = (Z[k] + conj Z[N-k]) / 2, Y = (Z[k] - conj Z[N-k]) / 2i
#pragma unroll 1
  for (int k = threadIdx.x; k < nbin; k += a.threads) {
    const float2 Zk = z[apad(k)], Zm = c_conj(z[apad((N - k) & (N - 1))]);
    const float2 X = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y + Zm.y));
    const float2 Y = make_float2(0.5f * (Zk.y - Zm.y), -0.5f * (Zk.x - Zm.x));
    const float4 v = make_float4(fmaf(X.x, X.x, X.y * X.y), fmaf(Y.x, Y.x, Y.y * Y.y), fmaf(X.x, Y.x, X.y * Y.y),
                                fmaf(X.y, Y.x, -X.x * Y.y));
    if (first) {
      part[k] = v;
    } else {
      const float4 o = part[k];
      part[k] = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
    }
  }
  __syncthreads();
}

template <int BITS>
__global__ void __launch_bounds__(1024) k_adj_forward(AdjArgs a) {
  extern __shared__ float2 z[];
#pragma unroll 1
  for (long long s = blockIdx.x; s < a.nseg; s += a.grid) adj_forward_segment<BITS>(a, z, s, s == blockIdx.x);
}

// one segment of the window-gradient pass
template <int BITS>
__device__ __forceinline__ void adj_window_segment(const AdjArgs& a, float2* z, long long s, bool first) {
  const int N = a.N, nbin = a.nbin;
  float* gpart = a.gpart + (size_t)blockIdx.x * N;
  adj_load_segment<BITS>(a, z, s);
  __syncthreads();
  adj_fft(z, N, a.log2n, a.tw, a.threads);
  // G_X, G_Y per bin pair; conj of the Hermitian extension of G_X + i G_Y goes back into z
  // (the inverse transform is conj(DFT(conj H))).  Thread k owns slots k and N - k.
#pragma unroll 1
  for (int k = threadIdx.x; k < nbin; k += a.threads) {
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
  __syncthreads();
  adj_fft(z, N, a.log2n, a.tw, a.threads);
  // h = conj(F): dL/dw[n] += x[n] Re h[n] + y[n] Im h[n] = x F.x - y F.y
  const long long base = s * N;
#pragma unroll 8
  for (int e = 0; e < 16; ++e) {
    const int n = threadIdx.x + e * a.threads;
    const float2 F = z[apad(n)];
    const float g = fmaf(adj_level<BITS>(a.in[0], base + n), F.x, -adj_level<BITS>(a.in[1], base + n) * F.y);
    gpart[n] = first ? g : gpart[n] + g;
  }
  __syncthreads();
}

template <int BITS>
__global__ void __launch_bounds__(1024) k_adj_window(AdjArgs a) {
  extern __shared__ float2 z[];
#pragma unroll 1
  for (long long s = blockIdx.x; s < a.nseg; s += a.grid) adj_window_segment<BITS>(a, z, s, s == blockIdx.x);
}

struct dc {
  double x, y;
};
__device__ __forceinline__ dc dmul(dc a, dc b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ dc dconj(dc a) { return {a.x, -a.y}; }
__device__ __forceinline__ dc dadd(dc a, dc b) { return {a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ dc dscale(dc a, double s) { return {a.x * s, a.y * s}; }
__device__ __forceinline__ double dnorm(dc a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float2 fscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float fnorm(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

struct BinArgs {
  const float4* part;
  int grid, nbin;
  const float* gains;
  const float* leak;
  const float* target;
  float* stokes;
  float* grad_leak;
  float4* mat;
  double* bpart;  // [blocks][5]: loss, G_gR re/im, G_gL re/im
};

// A block covers kBinsPerBlock bins; its kSlices warps sum the per-CTA partials of the
// segment kernel (one 16-byte load per CTA and bin) over interleaved slices of CTAs in fp32
// (many loads in flight), the slice sums are added in fp64 in slice order, then one warp
// evaluates the model per bin: the sums, Stokes and loss in fp64, the gradients and the
// window-adjoint matrix in fp32.
constexpr int kBinsPerBlock = 32, kSlices = 8;

__global__ void __launch_bounds__(kBinsPerBlock * kSlices) k_adj_bins(BinArgs a) {
  __shared__ float red[kSlices][4][kBinsPerBlock];
  const int nbin = a.nbin;
  const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int k = blockIdx.x * kBinsPerBlock + lane;
  float s4[4] = {0.f, 0.f, 0.f, 0.f};
  if (k < nbin) {
#pragma unroll 8
    for (int g = sl; g < a.grid; g += kSlices) {
      const float4 v = __ldcg(a.part + (size_t)g * nbin + k);
      s4[0] += v.x;
      s4[1] += v.y;
      s4[2] += v.z;
      s4[3] += v.w;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) red[sl][q][lane] = s4[q];
  __syncthreads();
  if (sl != 0) return;
  double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (k < nbin) {
    double t4[4] = {0.0, 0.0, 0.0, 0.0};
    for (int w = 0; w < kSlices; ++w)
      for (int q = 0; q < 4; ++q) t4[q] += (double)red[w][q][lane];
    const double A = t4[0], B = t4[1];
    const dc C = {t4[2], t4[3]};
    const dc gR = {a.gains[0], a.gains[1]}, gL = {a.gains[2], a.gains[3]};
    const dc DR = {a.leak[2 * k], a.leak[2 * k + 1]};
    const dc DL = {a.leak[2 * (nbin + k)], a.leak[2 * (nbin + k) + 1]};
    const double PR = A + dnorm(DR) * B + 2.0 * dmul(dconj(DR), C).x;
    const double PL = B + dnorm(DL) * A + 2.0 * dmul(DL, C).x;
    const dc Qm = dadd(dadd(C, dscale(dconj(DL), A)), dadd(dscale(DR, B), dmul(dmul(DR, dconj(DL)), dconj(C))));
    const double RR = dnorm(gR) * PR, LL = dnorm(gL) * PL;
    const dc RL = dmul(dmul(gR, dconj(gL)), Qm);
    const double S[4] = {0.5 * (RR + LL), RL.x, RL.y, 0.5 * (RR - LL)};
    if (a.stokes)
      for (int q = 0; q < 4; ++q) a.stokes[q * nbin + k] = (float)S[q];
    if (a.target) {
      float r[4];
      for (int q = 0; q < 4; ++q) {
        const double d = S[q] - (double)a.target[q * nbin + k];
        acc[0] += d * d;
        r[q] = (float)(2.0 * d);
      }
      if (a.mat) {
        const float ca = 0.5f * (r[0] + r[3]), cb = 0.5f * (r[0] - r[3]);
        const float2 c = make_float2(r[1], r[2]), cc = c_conj(c);
        const float2 fgR = make_float2(a.gains[0], a.gains[1]), fgL = make_float2(a.gains[2], a.gains[3]);
        const float2 fDR = make_float2((float)DR.x, (float)DR.y), fDL = make_float2((float)DL.x, (float)DL.y);
        const float2 fC = make_float2((float)C.x, (float)C.y), fQ = make_float2((float)Qm.x, (float)Qm.y);
        const float fA = (float)A, fB = (float)B;
        const float2 ggR = c_add(fscale(fgR, 2.f * ca * (float)PR), cmul(cmul(c, fgL), c_conj(fQ)));
        const float2 ggL = c_add(fscale(fgL, 2.f * cb * (float)PL), cmul(cmul(cc, fgR), fQ));
        acc[1] = ggR.x;
        acc[2] = ggR.y;
        acc[3] = ggL.x;
        acc[4] = ggL.y;
        const float2 gDR = c_add(fscale(c_add(fscale(fDR, fB), fC), 2.f * ca * fnorm(fgR)),
                                 cmul(cmul(c, cmulc(fgR, fgL)), c_add(make_float2(fB, 0.f), cmul(fDL, fC))));
        const float2 gDL = c_add(fscale(c_add(fscale(fDL, fA), c_conj(fC)), 2.f * cb * fnorm(fgL)),
                                 cmul(cmul(cc, cmulc(fgL, fgR)), c_add(make_float2(fA, 0.f), cmul(fDR, c_conj(fC)))));
        a.grad_leak[2 * k] = gDR.x;
        a.grad_leak[2 * k + 1] = gDR.y;
        a.grad_leak[2 * (nbin + k)] = gDL.x;
        a.grad_leak[2 * (nbin + k) + 1] = gDL.y;
        // G_Xt = al1 X + be1 Y, G_Yt = al2 X + be2 Y; G_X = conj(gR) G_Xt + conj(gL DL) G_Yt,
        // G_Y = conj(gR DR) G_Xt + conj(gL) G_Yt
        const float2 gLDL = cmul(fgL, fDL), gRDR = cmul(fgR, fDR);
        const float2 al1 = c_add(fscale(fgR, 2.f * ca), cmul(c, gLDL));
        const float2 be1 = c_add(fscale(gRDR, 2.f * ca), cmul(c, fgL));
        const float2 al2 = c_add(fscale(gLDL, 2.f * cb), cmul(cc, fgR));
        const float2 be2 = c_add(fscale(fgL, 2.f * cb), cmul(cc, gRDR));
        const float2 m11 = c_add(cmulc(fgR, al1), cmulc(gLDL, al2)), m12 = c_add(cmulc(fgR, be1), cmulc(gLDL, be2));
        const float2 m21 = c_add(cmulc(gRDR, al1), cmulc(fgL, al2)), m22 = c_add(cmulc(gRDR, be1), cmulc(fgL, be2));
        a.mat[2 * k] = make_float4(m11.x, m11.y, m12.x, m12.y);
        a.mat[2 * k + 1] = make_float4(m21.x, m21.y, m22.x, m22.y);
      }
    }
  }
  if (a.bpart) {
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      double v = acc[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) a.bpart[5 * blockIdx.x + q] = v;
    }
  }
}

// five warps, one per quantity: block partials summed lane-strided, then across the warp
// (the last block of k_adj_bins to finish doing this instead, elected by an atomic ticket
// after a memory fence, measured slower: 20.6 us against 13.4 + 3.7 us)
__global__ void __launch_bounds__(160) k_adj_finish(const double* bpart, int blocks, double* loss, float* grad_gains) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double t = 0.0;
  for (int b = lane; b < blocks; b += 32) t += bpart[5 * b + q];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  if (lane == 0) {
    if (q == 0) {
      if (loss) *loss = t;
    } else if (grad_gains) {
      grad_gains[q - 1] = (float)t;
    }
  }
}

// window-gradient partials summed per tap: 32 taps per block, kSlices warps over the CTAs
// (four taps per lane with one 16-byte load per CTA ran slower: 9.7 against 7.4 us, a
// quarter of the blocks)
__global__ void __launch_bounds__(kBinsPerBlock * kSlices) k_adj_wsum(const float* gpart, int grid, int N,
                                                                      float* grad_w) {
  __shared__ float red[kSlices][kBinsPerBlock];
  const int lane = threadIdx.x & 31, sl = threadIdx.x >> 5;
  const int n = blockIdx.x * kBinsPerBlock + lane;
  float t = 0.f;
  if (n < N) {
#pragma unroll 4
    for (int g = sl; g < grid; g += kSlices) t += __ldcg(gpart + (size_t)g * N + n);
  }
  red[sl][lane] = t;
  __syncthreads();
  if (sl == 0 && n < N) {
    double u = 0.0;
    for (int w = 0; w < kSlices; ++w) u += (double)red[w][lane];
    grad_w[n] = (float)u;
  }
}

}  // namespace polaris

using namespace polaris;

struct polaris_adj {
  int N = 0, log2n = 0, nbin = 0, bits = 0, device = 0, threads = 0, grid_max = 0, bin_blocks = 0;
  bool sized = false;  // the size-specialised segment kernels (polaris_adjoint_sized.cu)
  size_t smem = 0;
  float2* d_tw = nullptr;
  float4* d_part = nullptr;  // [grid_max][nbin]
  float* d_gpart = nullptr;  // [grid_max][N]
  float4* d_mat = nullptr;   // [nbin][2]
  double* d_bpart = nullptr; // [bin_blocks][5]
  std::string err;
};

static thread_local std::string g_adj_create_err;

static int adj_err(polaris_adj* h, int code, const char* msg, const char* detail = "") {
  std::string m = std::string(msg) + detail;
  if (h) h->err = m;
  else g_adj_create_err = m;
  return code;
}

template <int BITS>
static cudaError_t adj_prepare(polaris_adj* h, int* ctas_per_sm) {
  const int smem = (int)h->smem;
  cudaError_t e = cudaFuncSetAttribute(k_adj_forward<BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_window<BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  int o1 = 0, o2 = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, k_adj_forward<BITS>, h->threads, h->smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, k_adj_window<BITS>, h->threads, h->smem);
  *ctas_per_sm = std::min(o1, o2);
  return e;
}

static void adj_free(polaris_adj* h) {
  cudaFree(h->d_tw);
  cudaFree(h->d_part);
  cudaFree(h->d_gpart);
  cudaFree(h->d_mat);
  cudaFree(h->d_bpart);
}

extern "C" int polaris_adj_create(int64_t n_fft, int bits, int device, polaris_adj** out) {
  if (!out) return POLARIS_EINVAL;
  *out = nullptr;
  if (bits != 1 && bits != 2 && bits != 4 && bits != 8)
    return adj_err(nullptr, POLARIS_EINVAL, "bits must be 1, 2, 4 or 8");
  if (n_fft < 32 || n_fft > 16384 || (n_fft & (n_fft - 1)))
    return adj_err(nullptr, POLARIS_EINVAL, "n_fft must be a power of two in [32, 16384]");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return adj_err(nullptr, POLARIS_EINVAL, "no such CUDA device");
  }
  polaris_adj* h = new polaris_adj;
  h->N = (int)n_fft;
  while ((1 << h->log2n) < h->N) ++h->log2n;
  h->nbin = h->N / 2 + 1;
  h->bits = bits;
  h->device = device;
  h->threads = h->N / 16;
  h->sized = h->log2n >= kAdjSizedMin && h->log2n <= kAdjSizedMax;
  h->smem = (size_t)adj_smem_points(h->N) * sizeof(float2);
  h->bin_blocks = (h->nbin + kBinsPerBlock - 1) / kBinsPerBlock;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  int nsm = 0, occ = 0;
  cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  // the kernels for any N always (they also take calls whose buffers are not 16-byte
  // aligned), the size-specialised ones where they exist; both run on the same grid
  if (e == cudaSuccess) {
    switch (bits) {
      case 1: e = adj_prepare<1>(h, &occ); break;
      case 2: e = adj_prepare<2>(h, &occ); break;
      case 4: e = adj_prepare<4>(h, &occ); break;
      default: e = adj_prepare<8>(h, &occ); break;
    }
  }
  if (e == cudaSuccess && h->sized) {
    int occ_sized = 0;
    e = adj_sized_prepare(h->log2n, bits, &occ_sized);
    occ = std::min(occ, occ_sized);
  }
  if (e != cudaSuccess || occ < 1) {
    cudaGetLastError();
    cudaSetDevice(prev);
    delete h;
    return adj_err(nullptr, POLARIS_ECUDA, "adjoint kernels cannot be launched: ",
                   e != cudaSuccess ? cudaGetErrorString(e) : "zero occupancy");
  }
  h->grid_max = nsm * std::min(occ, kMaxCtasPerSm);
  // per-pass twiddles of the Stockham passes (radix 16, then 2, 4 or 8): pass with Ns
  // points done and radix R keeps W_{Ns R}^{r k} at r Ns + k - 1 (1 <= r < R, k < Ns); the
  // offsets Ns - 1 telescope, so the N - 1 entries tile [0, N - 1) exactly
  std::vector<float2> tw(h->N);
  for (int Ns = 1; Ns < h->N;) {
    const int R = std::min(16, h->N / Ns);
    for (int r = 1; r < R; ++r)
      for (int k = 0; k < Ns; ++k) {
        const double ang = -2.0 * M_PI * (double)r * (double)k / (double)(Ns * R);
        tw[r * Ns + k - 1] = make_float2((float)std::cos(ang), (float)std::sin(ang));
      }
    Ns *= R;
  }
  bool ok = cudaMalloc((void**)&h->d_tw, tw.size() * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&h->d_part, (size_t)h->grid_max * h->nbin * sizeof(float4)) == cudaSuccess &&
            cudaMalloc((void**)&h->d_gpart, (size_t)h->grid_max * h->N * sizeof(float)) == cudaSuccess &&
            cudaMalloc((void**)&h->d_mat, (size_t)h->nbin * 2 * sizeof(float4)) == cudaSuccess &&
            cudaMalloc((void**)&h->d_bpart, (size_t)h->bin_blocks * 5 * sizeof(double)) == cudaSuccess &&
            cudaMemcpy(h->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    adj_free(h);
    cudaSetDevice(prev);
    delete h;
    return adj_err(nullptr, POLARIS_ENOMEM, "device allocation failed");
  }
  cudaSetDevice(prev);
  *out = h;
  return POLARIS_OK;
}

extern "C" void polaris_adj_destroy(polaris_adj* h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  adj_free(h);
  cudaSetDevice(prev);
  delete h;
}

extern "C" const char* polaris_adj_last_error(const polaris_adj* h) {
  return h ? h->err.c_str() : g_adj_create_err.c_str();
}

template <int BITS>
static cudaError_t adj_segments(const AdjArgs& a, size_t smem, bool window_pass, cudaStream_t st) {
  if (!window_pass) k_adj_forward<BITS><<<a.grid, a.threads, smem, st>>>(a);
  else k_adj_window<BITS><<<a.grid, a.threads, smem, st>>>(a);
  return cudaGetLastError();
}

static cudaError_t adj_segments_bits(int bits, const AdjArgs& a, size_t smem, bool window_pass, bool sized,
                                     cudaStream_t st) {
  if (sized) return adj_sized_launch(a.log2n, bits, window_pass, a, st);
  switch (bits) {
    case 1: return adj_segments<1>(a, smem, window_pass, st);
    case 2: return adj_segments<2>(a, smem, window_pass, st);
    case 4: return adj_segments<4>(a, smem, window_pass, st);
    default: return adj_segments<8>(a, smem, window_pass, st);
  }
}

extern "C" int polaris_adj_run(polaris_adj* h, const void* const* packed, int64_t n_samples, const float* window,
                               const float* gains, const float* leak, const float* target, float* stokes,
                               double* loss, float* grad_window, float* grad_gains, float* grad_leak,
                               void* cuda_stream) {
  if (!h) return POLARIS_EINVAL;
  if (!packed || !packed[0] || !packed[1] || !window || !gains || !leak)
    return adj_err(h, POLARIS_EINVAL, "null input pointer");
  if (n_samples < h->N || n_samples % h->N)
    return adj_err(h, POLARIS_EINVAL, "n_samples must be a positive multiple of n_fft (whole segments, hop = n_fft)");
  if (n_samples / h->N > 0x7fffffff) return adj_err(h, POLARIS_EINVAL, "too many segments");
  const bool grads = grad_window || grad_gains || grad_leak;
  if ((grads || loss) && !target) return adj_err(h, POLARIS_EINVAL, "loss and gradients need a target");
  if (grads && !(grad_window && grad_gains && grad_leak))
    return adj_err(h, POLARIS_EINVAL, "gradients come as a set: grad_window, grad_gains and grad_leak");
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  AdjArgs a;
  memset(&a, 0, sizeof a);
  a.in[0] = static_cast<const uint32_t*>(packed[0]);
  a.in[1] = static_cast<const uint32_t*>(packed[1]);
  a.N = h->N;
  a.log2n = h->log2n;
  a.nbin = h->nbin;
  a.nseg = (int)(n_samples / h->N);
  a.grid = std::min(a.nseg, h->grid_max);
  a.threads = h->threads;
  a.tw = h->d_tw;
  a.window = window;
  a.part = h->d_part;
  a.mat = h->d_mat;
  a.gpart = h->d_gpart;
  // the size-specialised kernels read the inputs and the window by 16-byte vector loads
  auto aligned16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  const bool sized = h->sized && aligned16(packed[0]) && aligned16(packed[1]) && aligned16(window);
  cudaError_t e = adj_segments_bits(h->bits, a, h->smem, false, sized, st);
  if (e == cudaSuccess) {
    BinArgs b;
    b.part = h->d_part;
    b.grid = a.grid;
    b.nbin = h->nbin;
    b.gains = gains;
    b.leak = leak;
    b.target = target;
    b.stokes = stokes;
    b.grad_leak = grads ? grad_leak : nullptr;
    b.mat = grads ? h->d_mat : nullptr;
    b.bpart = (loss || grads) ? h->d_bpart : nullptr;
    k_adj_bins<<<h->bin_blocks, kBinsPerBlock * kSlices, 0, st>>>(b);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && (loss || grads)) {
    k_adj_finish<<<1, 160, 0, st>>>(h->d_bpart, h->bin_blocks, loss, grads ? grad_gains : nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && grads) {
    e = adj_segments_bits(h->bits, a, h->smem, true, sized, st);
    if (e == cudaSuccess) {
      k_adj_wsum<<<(h->N + kBinsPerBlock - 1) / kBinsPerBlock, kBinsPerBlock * kSlices, 0, st>>>(h->d_gpart, a.grid, h->N, grad_window);
      e = cudaGetLastError();
    }
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) return adj_err(h, POLARIS_ECUDA, "CUDA: ", cudaGetErrorString(e));
  return POLARIS_OK;
}
