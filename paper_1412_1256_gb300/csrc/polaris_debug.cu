// Bit-exactness check of the staged data translation (Fig. 2 caption: integer codes to
// floats).  From N = 2^13 up, phase 1 decodes from a shared-memory stage of each tile's
// packed words, with a rotation per column and both IFs of an FFT pair in one packed
// subtraction (p1_stage_decode).  k_unpack_staged fills a stage of the same layout as phase 1
// (interleaved for cp.async staging, dense for TMA staging) tile by tile and decodes every
// sample through that same device function, so the levels phase 1 transforms can be
// compared with the oracle's decode bit for bit.
#include "polaris_kernels.cuh"

namespace polaris {

// One CTA per tile (segment s, first column b0): stage the tile's N1 rows x WPR words of IF a
// (and IF b), then decode row, col -> sample n = s N + row N2 + b0 + col.
template <int LOGN, int BITS>
__global__ void __launch_bounds__(256) k_unpack_staged(const uint32_t* __restrict__ pa, const uint32_t* __restrict__ pb,
                                                       int dense, float* __restrict__ oa, float* __restrict__ ob) {
  using PL = Plan<LOGN>;
  using ST = typename PL::template Stage1<BITS>;
  constexpr int N = PL::N, N1 = PL::N1, N2 = PL::N2, TILE = ST::TILE, WPR = ST::WPR, RS = ST::RS;
  constexpr int SEGW = N * BITS / 32, ROWW = N2 * BITS / 32;  // words per segment, per row
  extern __shared__ uint32_t stg[];
  constexpr int TPS = N2 / TILE;  // tiles per segment
  const int s = blockIdx.x / TPS, b0 = (blockIdx.x % TPS) * TILE;
  const uint32_t* sa = pa + (size_t)s * SEGW + (b0 * BITS) / 32;
  const uint32_t* sbp = pb ? pb + (size_t)s * SEGW + (b0 * BITS) / 32 : nullptr;
  for (int k = threadIdx.x; k < N1 * WPR; k += blockDim.x) {
    const int row = k / WPR, w = k % WPR;
    const uint32_t va = sa[row * ROWW + w], vb = sbp ? sbp[row * ROWW + w] : va;
    if (dense) {
      stg[row * WPR + w] = va;
      stg[N1 * WPR + row * WPR + w] = vb;
    } else {
      stg[row * RS + 2 * w] = va;
      stg[row * RS + 2 * w + 1] = vb;  // (IF a again when the pair has no IF b, as phase 1 stages it)
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < N1 * TILE; e += blockDim.x) {
    const int row = e / TILE, col = e % TILE;
    const int wd = p1_col_word<BITS>(col);
    const uint32_t rot = p1_col_rot<BITS>(col);
    float2 z;
    if (dense) {
      z = sbp ? p1_stage_decode<BITS, true, true, N1, WPR, RS>(stg, row, wd, rot)
              : p1_stage_decode<BITS, true, false, N1, WPR, RS>(stg, row, wd, rot);
    } else {
      z = sbp ? p1_stage_decode<BITS, false, true, N1, WPR, RS>(stg, row, wd, rot)
              : p1_stage_decode<BITS, false, false, N1, WPR, RS>(stg, row, wd, rot);
    }
    const size_t n = (size_t)s * N + (size_t)row * N2 + b0 + col;
    oa[n] = z.x;
    if (sbp) ob[n] = z.y;
  }
}

template <int LOGN, int BITS>
static cudaError_t launch_unpack_staged_t(const uint32_t* pa, const uint32_t* pb, long long nseg, int dense, float* oa,
                                          float* ob, cudaStream_t st) {
  using PL = Plan<LOGN>;
  using ST = typename PL::template Stage1<BITS>;
  if constexpr (!ST::STAGED) {
    return cudaErrorInvalidValue;
  } else {
    const size_t smem_i = (size_t)PL::N1 * ST::RS * 4, smem_d = (size_t)2 * PL::N1 * ST::WPR * 4;
    const size_t smem = smem_i > smem_d ? smem_i : smem_d;
    cudaError_t e = cudaFuncSetAttribute(k_unpack_staged<LOGN, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const long long grid = nseg * (PL::N2 / ST::TILE);
    k_unpack_staged<LOGN, BITS><<<(unsigned)grid, 256, smem, st>>>(pa, pb, dense, oa, ob);
    return cudaGetLastError();
  }
}

template <int LOGN>
static cudaError_t launch_unpack_staged_n(int bits, const uint32_t* pa, const uint32_t* pb, long long nseg, int dense,
                                          float* oa, float* ob, cudaStream_t st) {
  switch (bits) {
    case 1: return launch_unpack_staged_t<LOGN, 1>(pa, pb, nseg, dense, oa, ob, st);
    case 2: return launch_unpack_staged_t<LOGN, 2>(pa, pb, nseg, dense, oa, ob, st);
    case 4: return launch_unpack_staged_t<LOGN, 4>(pa, pb, nseg, dense, oa, ob, st);
    case 8: return launch_unpack_staged_t<LOGN, 8>(pa, pb, nseg, dense, oa, ob, st);
    default: return cudaErrorInvalidValue;
  }
}

template <int LOGN, int BITS>
static constexpr bool staged_t() {
  return Plan<LOGN>::template Stage1<BITS>::STAGED;
}
template <int LOGN>
static constexpr bool staged_n(int bits) {
  return bits == 1 ? staged_t<LOGN, 1>() : bits == 2 ? staged_t<LOGN, 2>() : bits == 4 ? staged_t<LOGN, 4>()
                                                                            : staged_t<LOGN, 8>();
}

// true when phase 1 stages its input (and decodes through p1_stage_decode) at this size
bool phase1_staged(int logn, int bits) {
  switch (logn) {
#define POLARIS_ST(L) \
  case L: return staged_n<L>(bits);
    POLARIS_ST(4) POLARIS_ST(5) POLARIS_ST(6) POLARIS_ST(7) POLARIS_ST(8) POLARIS_ST(9) POLARIS_ST(10)
    POLARIS_ST(11) POLARIS_ST(12) POLARIS_ST(13) POLARIS_ST(14) POLARIS_ST(15) POLARIS_ST(16) POLARIS_ST(17)
    POLARIS_ST(18) POLARIS_ST(19) POLARIS_ST(20)
#undef POLARIS_ST
    default: return false;
  }
}

// decode nseg whole segments of IF a (and IF b, may be null) through the staged decoder
cudaError_t launch_unpack_staged(int logn, int bits, const uint32_t* pa, const uint32_t* pb, long long nseg, int dense,
                                 float* oa, float* ob, cudaStream_t st) {
  switch (logn) {
#define POLARIS_US(L) \
  case L: return launch_unpack_staged_n<L>(bits, pa, pb, nseg, dense, oa, ob, st);
    POLARIS_US(13) POLARIS_US(14) POLARIS_US(15) POLARIS_US(16) POLARIS_US(17) POLARIS_US(18) POLARIS_US(19)
    POLARIS_US(20)
#undef POLARIS_US
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace polaris
