// Leakage calibration (forward model and adjoint): what the segment kernels share.  The
// model, its gradients and the kernel sequence are described in polaris_adjoint.cu; the
// transforms of N = 2^9 .. 2^14 run in size-specialised kernels (polaris_adjoint_sized.cu),
// the smaller ones in polaris_adjoint.cu's kernels for any N.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "polaris_device.cuh"

namespace polaris {

struct AdjArgs {
  const uint32_t* in[2];  // the two IFs' packed words
  int N, log2n, nbin, nseg, grid, threads;
  const float2* tw;       // per-pass twiddles: tw[r Ns + k - 1] = W_{Ns R}^{r k} (N - 1 entries)
  const float* window;    // N
  float4* part;           // [grid][nbin]: (|X|^2, |Y|^2, Re X conj(Y), Im X conj(Y)) per bin
  const float4* mat;      // per bin (m11, m12), (m21, m22)
  float* gpart;           // [grid][N] window-gradient partials
};

// shared-memory layout of the N points: one float2 of padding after every 16 keeps the
// stride-16 writes of the first pass, and every other access, free of bank conflicts
__host__ __device__ __forceinline__ int apad(int i) { return i + (i >> 4); }
__host__ __device__ constexpr int adj_smem_points(int N) { return N + N / 16; }

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }

// level of sample idx of one IF
template <int BITS>
__device__ __forceinline__ float adj_level(const uint32_t* __restrict__ in, long long idx) {
  if constexpr (BITS == 8) {
    return (float)(int)__ldg(reinterpret_cast<const signed char*>(in) + idx);
  } else {
    constexpr int SPW = 32 / BITS;
    return decode_level<BITS>(__ldg(in + idx / SPW), (uint32_t)(idx % SPW) * BITS);
  }
}

// Size-specialised segment kernels (polaris_adjoint_sized.cu) for log2 N in
// [kAdjSizedMin, kAdjSizedMax].  adj_sized_prepare: sets the kernels' shared-memory limit
// for this device (current) and returns how many CTAs of the pair may share an SM
// (occupancy and tensor memory); adj_sized_launch: one segment kernel (forward or window
// pass) on a.grid CTAs.
constexpr int kAdjSizedMin = 9, kAdjSizedMax = 14;
cudaError_t adj_sized_prepare(int log2n, int bits, int* ctas_per_sm);
cudaError_t adj_sized_launch(int log2n, int bits, bool window_pass, const AdjArgs& a, cudaStream_t st);

}  // namespace polaris
