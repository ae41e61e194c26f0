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
// Adjoint: with r_S = 2 (S - T_S), a = (r_I + r_V)/2, b = (r_I - r_V)/2, c = r_Q + i r_U,
//   G_Xt = 2a Xt + c Yt,  G_Yt = 2b Yt + conj(c) Xt          (G = 2 dL/d conj(z))
//   G_X = conj(gR) G_Xt + conj(gL DL) G_Yt,  G_Y = conj(gR DR) G_Xt + conj(gL) G_Yt
//   grad gR = sum conj(X + DR Y) G_Xt,  grad gL = sum conj(Y + DL X) G_Yt
//   grad DR[k] = sum_s conj(gR Y) G_Xt,  grad DL[k] = sum_s conj(gL X) G_Yt
//   grad w[n] = sum_s x[n] Re(sum_k G_X[k] e^{+2 pi i n k/N}) + y[n] Re(sum_k G_Y[k] e^{+...})
// The last sums are real inverse transforms of the one-sided G: the Hermitian extensions of
// G_X and G_Y go through one complex inverse FFT as H_X + i H_Y.  Segments are transformed
// again in the adjoint pass, not stored.
//
// Kernels: one CTA per segment holds the segment's N complex points in shared memory
// (N <= 16384: 128 KB) and runs an in-place radix-2 transform; the pair x + i y is
// transformed once.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/polaris.h"
#include "polaris_device.cuh"

namespace polaris {

constexpr int kAdjThreads = 1024;

struct AdjArgs {
  const uint32_t* in[2];  // the two IFs' packed words
  int N, log2n, nbin, nseg;
  const float2* tw;       // W_N^j, j < N/2
  const float* window;    // N
  const float* gains;     // gR re, gR im, gL re, gL im
  const float* leak;      // DR then DL, nbin (re, im) each
  double* acc;            // RR, LL, RL re, RL im (4 x nbin)
  const float4* res;      // per bin (a, b, c re, c im)
  float* grad_w;          // N
  float* grad_leak;       // 2 x nbin x 2
  double* grad_g;         // 4
};

__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_scale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

__device__ __forceinline__ unsigned bitrev_n(unsigned v, int log2n) { return __brev(v) >> (32 - log2n); }

template <int BITS>
__device__ __forceinline__ float adj_level(const uint32_t* words, long long n) {
  constexpr int SPW = 32 / BITS;
  return decode_level<BITS>(words[n / SPW], (uint32_t)((n % SPW) * BITS));
}

// in-place radix-2 DIT over z (input in bit-reversed order, output natural); sign -1 forward
__device__ void adj_fft(float2* z, int N, const float2* tw, bool inverse) {
  for (int half = 1; half < N; half <<= 1) {
    const int step = N / (2 * half);
    for (int b = threadIdx.x; b < N / 2; b += kAdjThreads) {
      const int j = b & (half - 1);
      const int base = ((b / half) * 2 * half) + j;
      float2 w = __ldg(tw + j * step);
      if (inverse) w.y = -w.y;
      const float2 u = z[base], v = c_mul(z[base + half], w);
      z[base] = c_add(u, v);
      z[base + half] = make_float2(u.x - v.x, u.y - v.y);
    }
    __syncthreads();
  }
}

// MODE 0: accumulate RR, LL, RL.  MODE 1: adjoint (gain, leakage and window gradients).
template <int BITS, int MODE>
__global__ void __launch_bounds__(kAdjThreads) k_adj_segment(AdjArgs a) {
  extern __shared__ float2 z[];
  __shared__ double red[4][kAdjThreads / 32];
  const int N = a.N, nbin = a.nbin, s = blockIdx.x;
  const long long n0 = (long long)s * N;
  // windowed levels of the pair as z = w (x + i y), in bit-reversed order
  for (int n = threadIdx.x; n < N; n += kAdjThreads) {
    const float wn = __ldg(a.window + n);
    z[bitrev_n((unsigned)n, a.log2n)] =
        make_float2(wn * adj_level<BITS>(a.in[0], n0 + n), wn * adj_level<BITS>(a.in[1], n0 + n));
  }
  __syncthreads();
  adj_fft(z, N, a.tw, false);
  const float2 gR = make_float2(__ldg(a.gains + 0), __ldg(a.gains + 1));
  const float2 gL = make_float2(__ldg(a.gains + 2), __ldg(a.gains + 3));
  double gg[4] = {0.0, 0.0, 0.0, 0.0};
  // one thread per bin pair (k, N - k): both are read before either is rewritten
  for (int k = threadIdx.x; k < nbin; k += kAdjThreads) {
    const int km = (N - k) & (N - 1);
    const float2 Zk = z[k], Zm = c_conj(z[km]);
    const float2 X = make_float2(0.5f * (Zk.x + Zm.x), 0.5f * (Zk.y + Zm.y));
    const float2 Y = make_float2(0.5f * (Zk.y - Zm.y), -0.5f * (Zk.x - Zm.x));  // (Zk - Zm) / 2i
    const float2 DR = make_float2(__ldg(a.leak + 2 * k), __ldg(a.leak + 2 * k + 1));
    const float2 DL = make_float2(__ldg(a.leak + 2 * (nbin + k)), __ldg(a.leak + 2 * (nbin + k) + 1));
    const float2 uR = c_add(X, c_mul(DR, Y)), uL = c_add(Y, c_mul(DL, X));
    const float2 Xt = c_mul(gR, uR), Yt = c_mul(gL, uL);
    if constexpr (MODE == 0) {
      const float2 rl = c_mul(Xt, c_conj(Yt));
      atomicAdd(a.acc + k, (double)Xt.x * Xt.x + (double)Xt.y * Xt.y);
      atomicAdd(a.acc + nbin + k, (double)Yt.x * Yt.x + (double)Yt.y * Yt.y);
      atomicAdd(a.acc + 2 * nbin + k, (double)rl.x);
      atomicAdd(a.acc + 3 * nbin + k, (double)rl.y);
    } else {
      const float4 r = __ldg(a.res + k);  // a, b, c
      const float2 c = make_float2(r.z, r.w);
      const float2 GXt = c_add(c_scale(Xt, 2.f * r.x), c_mul(c, Yt));
      const float2 GYt = c_add(c_scale(Yt, 2.f * r.y), c_mul(c_conj(c), Xt));
      const float2 GX = c_add(c_mul(c_conj(gR), GXt), c_mul(c_conj(c_mul(gL, DL)), GYt));
      const float2 GY = c_add(c_mul(c_conj(c_mul(gR, DR)), GXt), c_mul(c_conj(gL), GYt));
      const float2 ggR = c_mul(c_conj(uR), GXt), ggL = c_mul(c_conj(uL), GYt);
      gg[0] += ggR.x;
      gg[1] += ggR.y;
      gg[2] += ggL.x;
      gg[3] += ggL.y;
      const float2 gDR = c_mul(c_conj(c_mul(gR, Y)), GXt), gDL = c_mul(c_conj(c_mul(gL, X)), GYt);
      atomicAdd(a.grad_leak + 2 * k, gDR.x);
      atomicAdd(a.grad_leak + 2 * k + 1, gDR.y);
      atomicAdd(a.grad_leak + 2 * (nbin + k), gDL.x);
      atomicAdd(a.grad_leak + 2 * (nbin + k) + 1, gDL.y);
      // Hermitian extensions of G_X, G_Y packed as H_X + i H_Y
      if (k == 0 || k == N / 2) {
        z[k] = make_float2(GX.x, GY.x);  // Re(G) at the self-mirrored bins
      } else {
        const float2 hx = c_scale(GX, 0.5f), hy = c_scale(GY, 0.5f);
        z[k] = make_float2(hx.x - hy.y, hx.y + hy.x);    // hx + i hy
        z[km] = make_float2(hx.x + hy.y, -hx.y + hy.x);  // conj(hx) + i conj(hy)
      }
    }
  }
  if constexpr (MODE == 1) {
    // gain gradients: block sum, one double atomic per component
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double v = gg[q];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((threadIdx.x & 31) == 0) red[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
      double t = 0.0;
      for (int w = 0; w < kAdjThreads / 32; ++w) t += red[threadIdx.x][w];
      atomicAdd(a.grad_g + threadIdx.x, t);
    }
    // bit-reverse in place, inverse transform, then the window gradient
    for (int i = threadIdx.x; i < N; i += kAdjThreads) {
      const int j = (int)bitrev_n((unsigned)i, a.log2n);
      if (i < j) {
        const float2 t = z[i];
        z[i] = z[j];
        z[j] = t;
      }
    }
    __syncthreads();
    adj_fft(z, N, a.tw, true);
    for (int n = threadIdx.x; n < N; n += kAdjThreads) {
      const float2 v = z[n];
      atomicAdd(a.grad_w + n, adj_level<BITS>(a.in[0], n0 + n) * v.x + adj_level<BITS>(a.in[1], n0 + n) * v.y);
    }
  }
}

// per bin: Stokes, residual coefficients (a, b, c), loss
__global__ void k_adj_residual(const double* acc, const float* target, int nbin, float* stokes, float4* res,
                               double* loss) {
  __shared__ double red[8];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (k < nbin) {
    const double RR = acc[k], LL = acc[nbin + k];
    const double S[4] = {0.5 * (RR + LL), acc[2 * nbin + k], acc[3 * nbin + k], 0.5 * (RR - LL)};
    if (stokes)
      for (int q = 0; q < 4; ++q) stokes[q * nbin + k] = (float)S[q];
    if (target) {
      double r[4];
      for (int q = 0; q < 4; ++q) {
        const double d = S[q] - (double)target[q * nbin + k];
        l += d * d;
        r[q] = 2.0 * d;
      }
      res[k] = make_float4((float)(0.5 * (r[0] + r[3])), (float)(0.5 * (r[0] - r[3])), (float)r[1], (float)r[2]);
    }
  }
  if (loss) {
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      atomicAdd(loss, t);
    }
  }
}

__global__ void k_adj_gains_out(const double* g, float* out) {
  if (threadIdx.x < 4) out[threadIdx.x] = (float)g[threadIdx.x];
}

}  // namespace polaris

using namespace polaris;

struct polaris_adj {
  int N = 0, log2n = 0, nbin = 0, bits = 0, device = 0;
  float2* d_tw = nullptr;
  double* d_acc = nullptr;  // 4 x nbin, then 4 gain-gradient doubles
  float4* d_res = nullptr;
  std::string err;
};

static thread_local std::string g_adj_create_err;

static int adj_err(polaris_adj* h, int code, const char* msg, const char* detail = "") {
  std::string m = std::string(msg) + detail;
  if (h) h->err = m;
  else g_adj_create_err = m;
  return code;
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
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(device);
  std::vector<float2> tw(h->N / 2);
  for (int j = 0; j < h->N / 2; ++j) {
    const double ang = -2.0 * M_PI * (double)j / (double)h->N;
    tw[j] = make_float2((float)std::cos(ang), (float)std::sin(ang));
  }
  bool ok = cudaMalloc((void**)&h->d_tw, tw.size() * sizeof(float2)) == cudaSuccess &&
            cudaMalloc((void**)&h->d_acc, (4 * (size_t)h->nbin + 4) * sizeof(double)) == cudaSuccess &&
            cudaMalloc((void**)&h->d_res, (size_t)h->nbin * sizeof(float4)) == cudaSuccess &&
            cudaMemcpy(h->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice) == cudaSuccess;
  cudaSetDevice(prev);
  if (!ok) {
    cudaGetLastError();
    cudaFree(h->d_tw);
    cudaFree(h->d_acc);
    cudaFree(h->d_res);
    delete h;
    return adj_err(nullptr, POLARIS_ENOMEM, "device allocation failed");
  }
  *out = h;
  return POLARIS_OK;
}

extern "C" void polaris_adj_destroy(polaris_adj* h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaFree(h->d_tw);
  cudaFree(h->d_acc);
  cudaFree(h->d_res);
  cudaSetDevice(prev);
  delete h;
}

extern "C" const char* polaris_adj_last_error(const polaris_adj* h) {
  return h ? h->err.c_str() : g_adj_create_err.c_str();
}

template <int BITS>
static cudaError_t adj_launch(const AdjArgs& a, bool grads, cudaStream_t st) {
  const size_t smem = (size_t)a.N * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(k_adj_segment<BITS, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_adj_segment<BITS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (!grads) {
    k_adj_segment<BITS, 0><<<a.nseg, kAdjThreads, smem, st>>>(a);
  } else {
    k_adj_segment<BITS, 1><<<a.nseg, kAdjThreads, smem, st>>>(a);
  }
  return cudaGetLastError();
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
  const int nbin = h->nbin;
  AdjArgs a;
  memset(&a, 0, sizeof a);
  a.in[0] = static_cast<const uint32_t*>(packed[0]);
  a.in[1] = static_cast<const uint32_t*>(packed[1]);
  a.N = h->N;
  a.log2n = h->log2n;
  a.nbin = nbin;
  a.nseg = (int)(n_samples / h->N);
  a.tw = h->d_tw;
  a.window = window;
  a.gains = gains;
  a.leak = leak;
  a.acc = h->d_acc;
  a.res = h->d_res;
  a.grad_w = grad_window;
  a.grad_leak = grad_leak;
  a.grad_g = h->d_acc + 4 * (size_t)nbin;
  cudaError_t e = cudaMemsetAsync(h->d_acc, 0, (4 * (size_t)nbin + 4) * sizeof(double), st);
  if (e == cudaSuccess && loss) e = cudaMemsetAsync(loss, 0, sizeof(double), st);
  if (e == cudaSuccess) {
    switch (h->bits) {  // forward: accumulate RR, LL, RL
      case 1: e = adj_launch<1>(a, false, st); break;
      case 2: e = adj_launch<2>(a, false, st); break;
      case 4: e = adj_launch<4>(a, false, st); break;
      default: e = adj_launch<8>(a, false, st); break;
    }
  }
  if (e == cudaSuccess) {
    k_adj_residual<<<(nbin + 255) / 256, 256, 0, st>>>(h->d_acc, target, nbin, stokes, h->d_res, loss);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && grads) {
    e = cudaMemsetAsync(grad_window, 0, (size_t)h->N * sizeof(float), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(grad_leak, 0, 4 * (size_t)nbin * sizeof(float), st);
    if (e == cudaSuccess) {
      switch (h->bits) {  // adjoint: transforms again, gradients
        case 1: e = adj_launch<1>(a, true, st); break;
        case 2: e = adj_launch<2>(a, true, st); break;
        case 4: e = adj_launch<4>(a, true, st); break;
        default: e = adj_launch<8>(a, true, st); break;
      }
    }
    if (e == cudaSuccess) {
      k_adj_gains_out<<<1, 32, 0, st>>>(a.grad_g, grad_gains);
      e = cudaGetLastError();
    }
  }
  cudaSetDevice(prev);
  if (e != cudaSuccess) return adj_err(h, POLARIS_ECUDA, "CUDA: ", cudaGetErrorString(e));
  return POLARIS_OK;
}
