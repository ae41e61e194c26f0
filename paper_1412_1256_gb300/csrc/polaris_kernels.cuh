// Hot-path kernels (sm_103a), templated on log2(N):
//
//   k_phase1  data translation (codes -> levels, Fig. 2 caption), window (Sec. 3.1),
//             first half of the segment FFT: for every column b of n = N2 a + b a DFT of
//             length N1 over the rows a, done in registers (P points per thread) with one
//             warp-local transpose through shared memory.  Writes the N complex partial
//             transforms of each pair-segment to a scratch slab [pair-segment][c][b].
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

#include <cuda.h>
#include <type_traits>
#include <cudaTypedefs.h>

#include "polaris_device.cuh"

namespace polaris {

// W_2048^k = e^{-2 pi i k / 2048}, k in [0, 2048), from the compile-time series.  The table
// sits in global memory (read through the read-only cache): the kernels' set-up reads a
// different entry in every lane, which a __constant__ bank would serialise per distinct
// address (that cost 8 us of a 45 us phase-1 launch at 2^17).
constexpr int kTwL = 2048;
struct TwTable {
  float2 v[kTwL];
};
constexpr TwTable make_tw_table() {
  TwTable t{};
  for (int k = 0; k < kTwL; ++k) {
    const ct::CS cs = ct::cossin2pi(k, kTwL);
    t.v[k].x = (float)cs.c;
    t.v[k].y = (float)(-cs.s);
  }
  return t;
}
static __device__ TwTable g_tw = make_tw_table();

// twiddle W_L^k for L <= 2048 (power of two), k any integer
template <int L>
__device__ __forceinline__ float2 tw_small(int k) {
  static_assert(L <= kTwL && kTwL % L == 0, "twiddle table");
  return __ldg(&g_tw.v[(k & (L - 1)) * (kTwL / L)]);
}

constexpr int kMaxIF = 8;

// Where segment s of the current feed starts, per IF: segments [0, n0) in src0 (the staging
// copy that joins carried samples to the new ones), the rest in src1 (the new data).
struct SegSrc {
  const uint32_t* src0[kMaxIF];
  const uint32_t* src1[kMaxIF];
  long long hop_w;  // 32-bit words between segment starts
  int n0;
  long long in_words0, in_words1;  // words reachable from src0 / src1 (read by the checked build)
};

struct BatchArgs {
  SegSrc in;
  int fa[kMaxIF];  // FFT pair f transforms IF fa[f] (real part) and IF fb[f] (imag part; < 0: zero)
  int fb[kMaxIF];
  int n_fpair;
  int seg0;             // first feed segment of this batch
  int nseg;             // segments in this batch
  const float* taps;    // window taps (N) or nullptr for the rectangular window
  float2* scratch;      // slab [nseg * n_fpair][N1][N2]: row c (phase-1 output index), b contiguous
  const float2* tw;     // [UPS + 1][N2]: W_N^{b u} (unit-major)
  void* acc;            // native accumulators [acc_copies][n_fpair][N/2 + 1] of float4 (double4 if fp64)
  int acc_copies;       // 1, or K: segment range r of a (pair, unit group) adds into copy r % K
  int fp64;
  int bits;
  int num_sms;
  int cap1, cap2;       // CTAs per SM of phase 1 / phase 2 at most (0: as many as fit)
  int* err;             // device status word: set to 1 when a bounded wait ran out (see k_phase2)
  unsigned wait_limit;  // iterations of a bounded mbarrier wait before it counts as timed out
  // buffer extents, read only by the bounds-checked build (POLARIS_CHECK): float2 elements of
  // this pass's slab, accumulator slots (float4 or double4) over all copies
  long long slab_elems, acc_slots;
};

// Bounds-checked build (-DPOLARIS_CHECK): every global-memory index of the hot-path kernels
// that is not checked by the hardware (tensor-map copies are) is tested against its buffer's
// extent; an index outside sets the device status word to kErrBounds and the access is
// skipped (a load gives zero).  Nothing traps.  In the normal build the test is compiled out.
constexpr int kErrBounds = 2;
#ifdef POLARIS_CHECK
__device__ __forceinline__ bool in_bounds(int* err, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  if (err) atomicExch(err, kErrBounds);
  return false;
}
#else
__device__ __forceinline__ constexpr bool in_bounds(int*, long long, long long) { return true; }
#endif
// word offset of segment s's first word from the start of its source (src0 or src1), and
// that source's extent
__device__ __forceinline__ long long seg_word0(const SegSrc& in, int s) {
  return s < in.n0 ? (long long)s * in.hop_w : (long long)(s - in.n0) * in.hop_w;
}

// Tensor maps of the packed input for phase 1's TMA staging: m[0][i] views IF i's staged
// segments [0, n0) and m[1][i] its segments from n0 on, each as words x rows x segments.
// use = 0: the kernel stages with cp.async instead (layouts a tensor map cannot describe).
struct InMaps {
  CUtensorMap m[2][kMaxIF];
  int use;
};

__device__ __forceinline__ const uint32_t* seg_ptr(const SegSrc& in, int ifx, int s) {
  return s < in.n0 ? in.src0[ifx] + (long long)s * in.hop_w : in.src1[ifx] + (long long)(s - in.n0) * in.hop_w;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
// L2 eviction policies for the copy engine: the slab is written by phase 1 and read once by
// phase 2 (kept in L2 in preference: evict_last); the packed input is read once (evict_first)
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
// TMA store of a 2-D box (x = column, y = row) from shared memory, issued by one elected lane
// of the (converged) warp as one bulk group; predicated, so the warp never branches apart
__device__ __forceinline__ void tma_store_2d_elect(const CUtensorMap* map, const void* src, int x, int y,
                                                   uint64_t policy) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b32 r;\n elect.sync r|p, 0xffffffff;\n"
      " @p cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%2, %3}], [%1], %4;\n"
      " @p cp.async.bulk.commit_group;\n}\n" ::"l"(map),
      "r"(smem_addr(src)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}
// TMA store of a 2-D box by the calling thread alone (the caller commits the group)
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y, uint64_t policy) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%2, %3}], [%1], %4;\n" ::"l"(
                   map),
               "r"(src), "r"(x), "r"(y), "l"(policy)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
// wait until this thread's bulk groups have finished reading shared memory (a lane that
// issued none returns at once)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
// mbarrier + bulk copies (phase-2 prefetch): one barrier per warp, expected-transaction
// counting; every wait is bounded by an iteration count
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
// one elected lane of the converged warp: announce `bytes`, then copy two contiguous blocks
// global -> shared, both completing on `bar`
__device__ __forceinline__ void bulk_load2_elect(uint32_t bar, uint32_t dst0, const void* src0, uint32_t dst1,
                                                 const void* src1, uint32_t bytes_each) {
  asm volatile(
      "{\n .reg .pred p;\n .reg .b32 r;\n elect.sync r|p, 0xffffffff;\n"
      " @p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %5;\n"
      " @p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%1], [%2], %6, [%0];\n"
      " @p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%3], [%4], %6, [%0];\n}\n" ::"r"(bar),
      "r"(dst0), "l"(src0), "r"(dst1), "l"(src1), "r"(2 * bytes_each), "r"(bytes_each)
      : "memory");
}
// one bulk copy global -> shared completing on mbarrier `bar` (the caller has announced the bytes)
__device__ __forceinline__ void bulk_load(uint32_t bar, uint32_t dst, const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// true once the barrier's phase `parity` has completed; false after `limit` polls
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (__any_sync(0xffffffffu, done != 0)) return true;  // phases only move forward
  }
  return false;
}
constexpr uint32_t kWaitAfterTimeout = 1u << 24;  // second, fixed bound: copies in flight land

// programmatic dependent launch: a kernel launched with programmatic stream serialisation may
// start before its predecessor in the stream ends; pdl_wait() returns once the predecessor
// has completed and its memory operations are visible (at once for an ordinary launch).
// pdl_trigger() lets the successor's CTAs be scheduled as soon as every CTA of this grid has
// triggered or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// ------------------------------------------------------------------------------------------
// tensor memory (TMEM) as per-thread storage: warp w reaches lanes 32 (w % 4) .. +31; a
// thread owns one lane and a range of 32-bit columns.  All tcgen05 calls below are
// warp-wide (.sync.aligned) and are made by converged warps only.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {  // one warp
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {  // the allocating warp
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory"); }
// 16 consecutive columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&r)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]), "=r"(u[7]), "=r"(u[8]),
        "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]), "=r"(u[14]), "=r"(u[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) r[i] = __uint_as_float(u[i]);
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
          taddr),
      "r"(__float_as_uint(r[0])), "r"(__float_as_uint(r[1])), "r"(__float_as_uint(r[2])), "r"(__float_as_uint(r[3])),
      "r"(__float_as_uint(r[4])), "r"(__float_as_uint(r[5])), "r"(__float_as_uint(r[6])), "r"(__float_as_uint(r[7])),
      "r"(__float_as_uint(r[8])), "r"(__float_as_uint(r[9])), "r"(__float_as_uint(r[10])),
      "r"(__float_as_uint(r[11])), "r"(__float_as_uint(r[12])), "r"(__float_as_uint(r[13])),
      "r"(__float_as_uint(r[14])), "r"(__float_as_uint(r[15]))
      : "memory");
}

// ------------------------------------------------------------------------------------------
// phase 1
// ------------------------------------------------------------------------------------------
template <int LOGN, int BITS>
__device__ __forceinline__ void p1_load(const BatchArgs& a, int g, int b, int q1, float2 (&v)[Plan<LOGN>::P1]) {
  using PL = Plan<LOGN>;
  constexpr int P = PL::P1, N2 = PL::N2, Q1 = PL::Q1;
  const int s_local = g / a.n_fpair, f = g - s_local * a.n_fpair;
  const int s = a.seg0 + s_local;
  const int ia = a.fa[f], ib = a.fb[f];
  const uint32_t* pa = seg_ptr(a.in, ia, s);
  const uint32_t* pb = ib >= 0 ? seg_ptr(a.in, ib, s) : nullptr;
  const long long w0 = seg_word0(a.in, s), wext = s < a.in.n0 ? a.in.in_words0 : a.in.in_words1;
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
    const bool ok = in_bounds(a.err, w0 + word_i, wext);
    float x = decode_level<BITS>(ok ? __ldg(pa + word_i) : 0u, shift);
    float y = pb ? decode_level<BITS>(ok ? __ldg(pb + word_i) : 0u, shift) : 0.0f;
    if (taps) {
      const float wv = __ldg(taps + n);
      x *= wv;
      y *= wv;
    }
    v[ct::bitrev(t, P)] = make_float2(x, y);
  });
}

// Data translation of the staged phase 1 (N >= 2^13), shared with the bit-exactness check
// (k_unpack_staged): column `col` of a tile starts at word p1_col_word(col) of each staged row,
// and its code sits at rotation p1_col_rot(col) of that word.
template <int BITS>
__device__ __forceinline__ int p1_col_word(int col) { return (col * BITS) >> 5; }
template <int BITS>
__device__ __forceinline__ uint32_t p1_col_rot(int col) { return decode_rot<BITS>((uint32_t)((col * BITS) & 31)); }
// The codes of staged row `row` at word wd, decoded at rotation rot, before the window:
// (level of IF a, level of IF b) for a pair with an IF b (HB), else (level of IF a, 0).
// Interleaved stage (cp.async, TL false): word w of IF a at 2w, of IF b at 2w + 1 of the
// row's RS words.  Dense stage (TMA, TL true): [IF][row][WPR].
template <int BITS, bool TL, bool HB, int N1, int WPR, int RS>
__device__ __forceinline__ float2 p1_stage_decode(const uint32_t* sb, int row, int wd, uint32_t rot) {
  uint32_t wa, wb = 0;
  if constexpr (TL) {
    wa = sb[row * WPR + wd];
    if constexpr (HB) wb = sb[N1 * WPR + row * WPR + wd];
  } else {
    const uint2 w = *reinterpret_cast<const uint2*>(sb + row * RS + 2 * wd);  // IF a, IF b
    wa = w.x;
    wb = w.y;
  }
  if constexpr (HB) {
    return decode_pair_rot<BITS>(wa, wb, rot);
  } else {
    return make_float2(decode_level_rot<BITS>(wa, rot), 0.0f);
  }
}

__device__ __forceinline__ void corr_acc(float (&acc)[4], float2 U, float2 V) {
  // S = 2X, D = 2iY;  |S|^2, |D|^2, Re/Im of i S conj(D) (= 4 X conj(Y)).  S and D by packed
  // operations (each component rounds once, as the scalar sum and difference would)
  const float2 S = __fadd2_rn(U, V), D = __ffma2_rn(V, make_float2(-1.f, -1.f), U);
  const float sx = S.x, sy = S.y, dx = D.x, dy = D.y;
  acc[0] = fmaf(sx, sx, fmaf(sy, sy, acc[0]));
  acc[1] = fmaf(dx, dx, fmaf(dy, dy, acc[1]));
  acc[2] = fmaf(sx, dy, fmaf(-sy, dx, acc[2]));
  acc[3] = fmaf(sx, dx, fmaf(sy, dy, acc[3]));
}



// ------------------------------------------------------------------------------------------
// warp-owned work: no CTA-wide barrier inside the loops.  Each warp allocates nothing; the
// CTA takes its tensor memory once (warp 0) and gives it back at the end.
// ------------------------------------------------------------------------------------------
template <int TCOLS>
__device__ __forceinline__ uint32_t cta_tmem_begin(uint32_t* slot, int warp) {
  if (warp == 0) tmem_alloc(slot, TCOLS);
  tmem_fence_before();
  __syncthreads();
  tmem_fence_after();
  return *slot;
}
template <int TCOLS>
__device__ __forceinline__ void cta_tmem_end(uint32_t tbase, int warp) {
  tmem_fence_before();
  __syncthreads();
  if (warp == 0) {
    tmem_fence_after();
    tmem_dealloc(tbase, TCOLS);
  }
}

// ------------------------------------------------------------------------------------------
// phase 1: a warp owns CW = 32/Q1 adjacent columns of the slab; lane (q1, cw) loads rows
// q1 + Q1 t of column cw, runs the P-point DFT in registers, twiddles by W_N1^{q1 p} (held in
// its tensor-memory lane), transposes through the warp's shared-memory region and finishes
// the N1-point DFT with Q1-point register DFTs.  Output slab layout: [pair-segment][c][b].
// ------------------------------------------------------------------------------------------
template <int LOGN, int BITS>
__global__ void __launch_bounds__(Plan<LOGN>::THREADS, Plan<LOGN>::MINB1)
    k_phase1(BatchArgs a, const __grid_constant__ CUtensorMap slab_map, const __grid_constant__ InMaps in_maps) {
  using PL = Plan<LOGN>;
  constexpr int P = PL::P1, N1 = PL::N1, N2 = PL::N2, Q1 = PL::Q1, CW = PL::CW, PQ = PL::PQ;
  constexpr int LDP = PL::LDP1, LDQ = PL::LDQ1;
  using ST = typename PL::template Stage1<BITS>;
  constexpr bool STAGED = ST::STAGED;
  constexpr int TILE = ST::TILE, IPT = ST::IPT, WPR = STAGED ? ST::WPR : 1;  // words per IF per tile row
  // the warp's [N1][CW] output block leaves by one TMA store (TMA_OUT), or the column
  // group's [N1][JC] block, assembled over all warps' regions, by N1 / BOXR (JOINT)
  constexpr bool TMA_OUT = ST::TMA_OUT, JOINT = ST::JOINT_OUT;
  constexpr int BOXR = ST::BOXR, JC = ST::JC;
  static_assert(!TMA_OUT || (Q1 > 1 && N1 == BOXR && (CW * 8) % 16 == 0 && N1 * CW <= PL::REGION1 &&
                             (PL::REGION1 * 8) % 128 == 0),
                "TMA output tile");
  static_assert(!JOINT || (N1 % BOXR == 0 && (BOXR * JC * 8) % 1024 == 0 && (size_t)N1 * JC * 8 <= PL::REGIONS1),
                "joint output block");
  extern __shared__ __align__(1024) float2 sm1[];
  // (warp index and tensor-memory base broadcast from lane 0: uniform registers, as in phase 2)
  const int tid = threadIdx.x, warp = __shfl_sync(0xffffffffu, tid >> 5, 0), lane = tid & 31;
  if constexpr (JOINT) {
    // the swizzled joint block needs a 1024-byte aligned base (the declaration asks for it);
    // should that ever not hold, report and leave the work undone rather than misplace data
    if ((smem_addr(sm1) & 1023u) != 0) {
      if (tid == 0 && a.err) atomicExch(a.err, 1);
      return;
    }
  }
  const int q1 = lane / CW, cw = lane % CW;
  float2* region = sm1 + warp * PL::REGION1;
  uint32_t* stage = reinterpret_cast<uint32_t*>(sm1 + PL::WARPS * PL::REGION1);  // stage buffers
  const uint32_t bar0 = smem_addr(stage + ST::WORDS);  // two mbarriers (TMA staging), then the TMEM slot
  uint32_t* tslot = stage + ST::WORDS + 4;
  // TMA staging of the input: possible for this plan (two buffers, 16-byte box rows) and
  // chosen by the host for this launch
  constexpr bool TIN = ST::TMA_IN;
  static_assert(!TIN || (N1 % BOXR == 0 && (BOXR * WPR * 4) % 128 == 0), "TMA input boxes");
  const bool tin = TIN && in_maps.use != 0;
  if (TIN && tin && tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_async_shared();
  }

  uint32_t tbase = 0, t_tw = 0;
  if constexpr (Q1 > 1) {
    tbase = __shfl_sync(0xffffffffu, cta_tmem_begin<PL::TCOLS1>(tslot, warp), 0);
    t_tw = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * PL::TW1);
    // this lane's twiddles W_N1^{q1 p}, p < P
    sfor<0, PL::TW1 / 16>([&](auto c_) {
      constexpr int cc = decltype(c_)::value;
      float w16[16];
      sfor<0, 8>([&](auto k_) {
        constexpr int k = decltype(k_)::value;
        const float2 w = tw_small<N1>(q1 * (8 * cc + k));
        w16[2 * k] = w.x;
        w16[2 * k + 1] = w.y;
      });
      tmem_st16(t_tw + 16 * cc, w16);
    });
    tmem_wait_st();
  }
  pdl_wait();  // the input and the slab may be touched from here on (dependent launch)

  // Slab rows c > N1/2 are read by phase 2 only as the mirror column of unit N1 - c, which
  // enters its transform conjugated: phase 1 stores them conjugated (an exact sign flip).
  auto slab_val = [](float2 x, int c) { return c > N1 / 2 ? make_float2(x.x, -x.y) : x; };
  // the second half of the work on one column group: twiddle, transpose, Q1-point DFTs, store.
  // After the transpose lane (q1, cw) holds, for p = r Q1 + q1, the Q1 values of row p; its
  // DFT gives rows c = p + P m of the slab.
  auto finish = [&](float2 (&v)[P], bool act, long long g, long long b, int xcol) {
    dit<P>(v);
    if constexpr (Q1 > 1) {
      sfor<0, P / 8>([&](auto c_) {
        constexpr int cc = decltype(c_)::value;
        float w16[16];
        tmem_ld16(t_tw + 16 * cc, w16);
        tmem_wait_ld();
        sfor<0, 8>([&](auto k_) {
          constexpr int k = decltype(k_)::value;
          constexpr int p = 8 * cc + k;
          if constexpr (p > 0) v[p] = cmul(v[p], make_float2(w16[2 * k], w16[2 * k + 1]));
        });
      });
      if constexpr (TMA_OUT) {
        bulk_wait_read();  // the previous output tile has left the region
        __syncwarp();
      }
      if constexpr (JOINT) {
        if (tid == 0) bulk_wait_read();  // the previous joint block has left the regions
        __syncthreads();
      }
      sfor<0, P>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        region[q1 * LDQ + p * LDP + cw] = v[p];
      });
      __syncwarp();
      if constexpr (JOINT) {
        sfor<0, PQ>([&](auto r_) {
          constexpr int r = decltype(r_)::value;
          const int p = r * Q1 + q1;
          sfor<0, Q1>([&](auto q_) {
            constexpr int q = decltype(q_)::value;
            v[r * Q1 + ct::bitrev(q, Q1)] = region[q * LDQ + p * LDP + cw];
          });
          dit<Q1, r * Q1, 1>(v);
        });
        __syncthreads();  // every warp has read its transpose: the regions take the joint block
        // joint block [c][JC] of 8-byte values, JC * 8 = 64 or 128 bytes per row, with the
        // TMA swizzle of that row width: 16-byte chunk k of row c sits at chunk k ^ (row
        // bits of the byte offset), so the 16 or 32 rows one store instruction writes fall
        // on distinct chunks
        // Row c = C0 + q1 with C0 = r Q1 + P m a multiple of 8: the row bits the swizzle
        // takes (bits 7-9 of the offset for 128-byte rows, 7-8 for 64-byte rows) are those
        // of the lane's own first row, and C0's part of the offset has no bits below the
        // ninth, so the swizzled offset is the lane's swizzled base plus C0's part.
        static_assert(Q1 % 8 == 0 && P % 8 == 0, "joint block swizzle per lane");
        char* jb = reinterpret_cast<char*>(sm1);
        const uint32_t jl = (uint32_t)((q1 * JC + warp * CW + cw) * 8);
        char* jlane = jb + (jl ^ (((jl >> 7) & (uint32_t)ST::JSW) << 4));
        sfor<0, PQ>([&](auto r_) {
          constexpr int r = decltype(r_)::value;
          sfor<0, Q1>([&](auto m_) {
            constexpr int m = decltype(m_)::value;
            *reinterpret_cast<float2*>(jlane + (r * Q1 + P * m) * JC * 8) =
                slab_val(v[r * Q1 + m], r * Q1 + q1 + P * m);
          });
        });
        fence_async_shared();
        __syncthreads();
        if (tid == 0 && act) {  // xcol of warp 0 = the column group's first column
          sfor<0, N1 / BOXR>([&](auto h_) {
            constexpr int h = decltype(h_)::value;
            tma_store_2d(&slab_map, smem_addr(jb + h * BOXR * JC * 8), xcol, (int)(g * N1 + h * BOXR),
                         l2_evict_last());
          });
          bulk_commit();
        }
      } else if constexpr (TMA_OUT) {
        sfor<0, PQ>([&](auto r_) {
          constexpr int r = decltype(r_)::value;
          const int p = r * Q1 + q1;
          sfor<0, Q1>([&](auto q_) {
            constexpr int q = decltype(q_)::value;
            v[r * Q1 + ct::bitrev(q, Q1)] = region[q * LDQ + p * LDP + cw];
          });
        });
        __syncwarp();  // region consumed: it now takes the output tile [c][cw]
        sfor<0, PQ>([&](auto r_) {
          constexpr int r = decltype(r_)::value;
          dit<Q1, r * Q1, 1>(v);
          sfor<0, Q1>([&](auto m_) {
            constexpr int m = decltype(m_)::value;
            region[(r * Q1 + q1 + P * m) * CW + cw] = slab_val(v[r * Q1 + m], r * Q1 + q1 + P * m);
          });
        });
        fence_async_shared();
        __syncwarp();
        if (act) tma_store_2d_elect(&slab_map, region, xcol, (int)(g * N1), l2_evict_last());
      } else {
        sfor<0, PQ>([&](auto r_) {
          constexpr int r = decltype(r_)::value;
          const int p = r * Q1 + q1;
          float2 u[Q1];
          sfor<0, Q1>([&](auto q_) {
            constexpr int q = decltype(q_)::value;
            u[ct::bitrev(q, Q1)] = region[q * LDQ + p * LDP + cw];
          });
          dit<Q1>(u);
          if (act) {
            float2* dst = a.scratch + ((size_t)g * N1 + p) * N2 + b;
            sfor<0, Q1>([&](auto m_) {
              constexpr int m = decltype(m_)::value;
              if (in_bounds(a.err, ((long long)g * N1 + p + (long long)m * P) * N2 + b, a.slab_elems))
                dst[(size_t)m * P * N2] = slab_val(u[m], p + m * P);
            });
          }
        });
        __syncwarp();  // region free for the next item
      }
    } else {
      if (act) {
        float2* dst = a.scratch + (size_t)g * N1 * N2 + b;
        sfor<0, P>([&](auto p_) {
          constexpr int p = decltype(p_)::value;
          if (in_bounds(a.err, (long long)g * N1 * N2 + (long long)p * N2 + b, a.slab_elems))
            dst[(size_t)p * N2] = slab_val(v[p], p);
        });
      }
    }
  };

  const long long total_cols = (long long)a.nseg * a.n_fpair * N2;
  if constexpr (!STAGED) {
    // small N: each warp item = CW global columns, each lane loads its own words
    const long long n_items = (total_cols + CW - 1) / CW;
    const long long nw = (long long)gridDim.x * PL::WARPS;
    for (long long item = (long long)blockIdx.x * PL::WARPS + warp; item < n_items; item += nw) {
      const long long gc = item * CW + cw;
      const bool act = gc < total_cols;
      const long long g = gc / N2, b = gc % N2;
      float2 v[P];
      if (act) {
        p1_load<LOGN, BITS>(a, (int)g, (int)b, q1, v);
      } else {
        sfor<0, P>([&](auto t_) { v[decltype(t_)::value] = make_float2(0.f, 0.f); });
      }
      finish(v, act, g, b, 0);
    }
  } else {
    // CTA tiles of TILE columns of one pair-segment.  The packed words of a tile (both IFs)
    // are staged in shared memory with cp.async, double-buffered so that the next tile's
    // words are in flight while the warps work on this one; every warp decodes its CW
    // columns from the stage.
    constexpr int RS = ST::RS;   // words per staged row
    constexpr int SB = N1 * RS;  // words per stage buffer
    constexpr int NB = ST::NB;   // 2: next tile in flight
    const long long n_tiles = total_cols / TILE;
    const uint32_t stage_a = smem_addr(stage);
    // this thread's share of a tile's words: source offsets (words from the tile's first word
    // of its row 0) and stage offsets (bytes), the same for every tile
    constexpr int KW = N1 * WPR, KPT = (KW + PL::THREADS - 1) / PL::THREADS;
    uint32_t soff[KPT], doff[KPT];
    sfor<0, KPT>([&](auto i_) {
      constexpr int i = decltype(i_)::value;
      const int k = (int)threadIdx.x + i * PL::THREADS;
      const int row = k / WPR, wd = k % WPR;
      soff[i] = (uint32_t)(row * (N2 * BITS / 32) + wd);
      doff[i] = 4u * (uint32_t)(row * RS + 2 * wd);
    });
    auto issue = [&](long long tile, int buf) {
      const int g = (int)(tile / (N2 / TILE)), b0 = (int)(tile % (N2 / TILE)) * TILE;
      const int s_local = g / a.n_fpair, f = g - s_local * a.n_fpair;
      const int sg = a.seg0 + s_local;
      const int ia = a.fa[f], ib = a.fb[f];
      const uint32_t* pa = seg_ptr(a.in, ia, sg) + (b0 * BITS) / 32;
      const uint32_t* pb = ib >= 0 ? seg_ptr(a.in, ib, sg) + (b0 * BITS) / 32 : pa;
      const uint32_t dst0 = stage_a + 4u * (uint32_t)(buf * SB);
      const long long w0 = seg_word0(a.in, sg) + (b0 * BITS) / 32;
      const long long wext = sg < a.in.n0 ? a.in.in_words0 : a.in.in_words1;
      sfor<0, KPT>([&](auto i_) {
        constexpr int i = decltype(i_)::value;
        if (KW % PL::THREADS == 0 || (int)threadIdx.x + i * PL::THREADS < KW) {
          if (in_bounds(a.err, w0 + soff[i], wext)) {
            cp_async4(dst0 + doff[i], pa + soff[i]);
            cp_async4(dst0 + doff[i] + 4u, pb + soff[i]);  // (IF a again when the pair has no IF b)
          }
        }
      });
      cp_async_commit();
    };
    // TMA staging: one thread loads the tile's words of each IF (N1 rows x WPR words, in
    // boxes of BOXR rows) into a dense [IF][row][word] stage and the CTA waits on that
    // buffer's mbarrier (bounded)
    auto issue_tma = [&](long long tile, int buf) {
      const int g = (int)(tile / (N2 / TILE)), b0 = (int)(tile % (N2 / TILE)) * TILE;
      const int s_local = g / a.n_fpair, f = g - s_local * a.n_fpair;
      const int sg = a.seg0 + s_local;
      const int ia = a.fa[f], ib = a.fb[f];
      const int src = sg < a.in.n0 ? 0 : 1, z = sg < a.in.n0 ? sg : sg - a.in.n0;
      const uint32_t bar = bar0 + 8u * (uint32_t)buf, dst = stage_a + 4u * (uint32_t)(buf * SB);
      const uint32_t box = (uint32_t)(N1 * WPR * 4), sub = (uint32_t)(BOXR * WPR * 4);  // bytes per IF, per box
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar),
                   "r"(ib >= 0 ? 2 * box : box)
                   : "memory");
      const int x = (b0 * BITS) / 32;
      const uint64_t pol_in = l2_evict_first();
      sfor<0, N1 / BOXR>([&](auto h_) {
        constexpr int h = decltype(h_)::value;
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
            "{%2, %3, %4}], [%5], %6;\n" ::"r"(dst + h * sub),
            "l"(&in_maps.m[src][ia]), "r"(x), "r"(h * BOXR), "r"(z), "r"(bar), "l"(pol_in)
            : "memory");
        if (ib >= 0)
          asm volatile(
              "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, "
              "{%2, %3, %4}], [%5], %6;\n" ::"r"(dst + box + h * sub),
              "l"(&in_maps.m[src][ib]), "r"(x), "r"(h * BOXR), "r"(z), "r"(bar), "l"(pol_in)
              : "memory");
      });
    };
    // Work units: whole tiles for the complete rounds over the grid, then, for the last,
    // partial round, half tiles (one column group per warp; the whole tile is staged), so
    // that the last round spreads over twice as many CTAs.
    const long long G = gridDim.x;
    long long F = n_tiles;  // units [0, F) are whole tiles, [F, ...) halves of the rest
    if (IPT == 2 && n_tiles % G != 0) F = (n_tiles / G) * G;
    const long long n_units = F + (n_tiles - F) * (IPT == 2 ? 2 : 1);
    auto unit_tile = [&](long long u) { return u < F ? u : F + (u - F) / 2; };
    uint32_t par[2] = {0u, 0u};
    long long unit = blockIdx.x;
    if (unit < n_units) {
      if (tin) {
        if (tid == 0) issue_tma(unit_tile(unit), 0);
      } else {
        issue(unit_tile(unit), 0);
      }
    }
    for (int buf = 0; unit < n_units; unit += G, buf = (NB == 2) ? buf ^ 1 : 0) {
      const long long tile = unit_tile(unit);
      const int it_begin = unit < F ? 0 : (int)((unit - F) & 1), it_end = unit < F ? IPT : it_begin + 1;
      int timed_out = 0;
      if (tin) {
        const uint32_t bar = bar0 + 8u * (uint32_t)buf;
        if (!mbar_wait_bounded(bar, par[buf], a.wait_limit)) {
          timed_out = 1;
          if (lane == 0 && a.err) atomicExch(a.err, 1);
          mbar_wait_bounded(bar, par[buf], kWaitAfterTimeout);  // the copy in flight lands first
        }
        par[buf] ^= 1u;
      } else {
        cp_async_wait_all();
      }
      // this tile's words are staged; every warp is done with the other buffer
      if (__syncthreads_or(timed_out)) break;
      const long long next = unit + G;
      if constexpr (NB == 2) {
        if (next < n_units) {
          if (tin) {
            if (tid == 0) {
              fence_async_shared();  // the CTA's reads of that buffer come before the copy
              issue_tma(unit_tile(next), buf ^ 1);
            }
          } else {
            issue(unit_tile(next), buf ^ 1);
          }
        }
      }
      if (next >= n_units) pdl_trigger();  // this CTA's last unit: phase 2 may be scheduled
      const int g = (int)(tile / (N2 / TILE)), b0 = (int)(tile % (N2 / TILE)) * TILE;
      const int f = g % a.n_fpair;
      const bool has_b = a.fb[f] >= 0;
      // IPT column groups per warp per tile: group it of warp w holds columns (it WARPS + w) CW + cw
      // (a rolled loop: one copy of the decode variants and of the transform in the code)
#pragma unroll 1
      for (int it = it_begin; it < it_end; ++it) {
        const int col = (it * PL::WARPS + warp) * CW + cw;  // column inside the tile
        const long long b = b0 + col;
        const int wd = p1_col_word<BITS>(col);
        const uint32_t rot = p1_col_rot<BITS>(col);
        const uint32_t* sb = stage + buf * SB;
        float2 v[P];
        // decode the lane's rows; the stage layout (TL), the pair's shape (HB) and the
        // window (TP) are uniform per tile
        auto decode = [&](auto tl_, auto hb_, auto tp_) {
          constexpr bool TL = decltype(tl_)::value, HB = decltype(hb_)::value, TP = decltype(tp_)::value;
          sfor<0, P>([&](auto t_) {
            constexpr int t = decltype(t_)::value;
            const int row = q1 + Q1 * t;
            float2 z = p1_stage_decode<BITS, TL, HB, N1, WPR, RS>(sb, row, wd, rot);
            if constexpr (TP) {
              const float tv = __ldg(a.taps + row * N2 + b);
              z.x *= tv;
              z.y *= tv;
            }
            v[ct::bitrev(t, P)] = z;
          });
        };
        using T_ = std::true_type;
        using F_ = std::false_type;
        auto decode_tl = [&](auto tl) {
          if (a.taps) {
            if (has_b) decode(tl, T_{}, T_{});
            else decode(tl, F_{}, T_{});
          } else {
            if (has_b) decode(tl, T_{}, F_{});
            else decode(tl, F_{}, F_{});
          }
        };
        if constexpr (TIN) {
          if (tin) decode_tl(T_{});
          else decode_tl(F_{});
        } else {
          decode_tl(F_{});
        }
        if constexpr (NB == 1) {
          if (it == it_end - 1) {
            __syncthreads();  // every warp has decoded the tile: the single buffer is free
            if (next < n_units) issue(unit_tile(next), 0);
          }
        }
        finish(v, true, g, b, b0 + (it * PL::WARPS + warp) * CW);
      }
    }
    cp_async_wait_all();
  }
  if constexpr (TMA_OUT || JOINT) {
    bulk_wait_all();  // output tiles written before the CTA's shared memory goes
  }
  if constexpr (Q1 > 1) cta_tmem_end<PL::TCOLS1>(tbase, warp);
}

// ------------------------------------------------------------------------------------------
// phase 2 and the correlator.  A warp owns UPW units (column u and its mirror N1 - u; unit 0
// = columns 0 and N1/2) over a range of segments.  Lane (uw, e, q2) loads rows q2 + Q2 t of
// its column (a mirror column arrives conjugated: phase 1 stores rows c > N1/2 so), applies
// W_N^{b u} (its tensor-memory twiddles), runs the
// P-point DFT, transposes through the warp's region (the two members of a unit together),
// applies W_N2^{q p} and runs the Q2-point DFTs, so that lane (uw, j) holds Z_k and
// conj(Z_{N-k}) for bins k = u + N1 d, d = j PP + r + P m.  |S|^2, |D|^2 and i S conj(D)
// (S = 2X, D = 2iY) are accumulated in its tensor-memory lane over the range and added once
// to the integration accumulators.
// ------------------------------------------------------------------------------------------
template <int LOGN>
__global__ void __launch_bounds__(Plan<LOGN>::THREADS, 2) k_phase2(BatchArgs a, int range_len) {
  using PL = Plan<LOGN>;
  constexpr int P = PL::P, N1 = PL::N1, N2 = PL::N2, Q2 = PL::Q2, UPS = PL::UPS, UPW = PL::UPW;
  constexpr int SL = PL::SL, UGW = PL::UGW, PP = PL::PP, NACC = PL::NACC;
  constexpr int LDQ = PL::LDQ2, LDE = PL::LDE2, TACC = PL::TACC;
  extern __shared__ float2 sm2[];
  // (the warp index and the tensor-memory base broadcast from lane 0: values the compiler can
  // keep in uniform registers, which the tensor-memory loads and stores address by)
  const int tid = threadIdx.x, warp = __shfl_sync(0xffffffffu, tid >> 5, 0), lane = tid & 31;
  float2* region = sm2 + warp * PL::REGION2;
  float2* tw2 = sm2 + PL::WARPS * PL::REGION2;  // skewed table: W_N2^k at k + k/32
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tw2 + PL::TWT);
  // prefetch (PF): the next segment's columns arrive in the warp's region by bulk copy
  constexpr bool PF = PL::PF2;
  const uint32_t bar = smem_addr(reinterpret_cast<uint64_t*>(tslot + 4) + warp);
  if constexpr (PF) {
    if (lane == 0) mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    fence_async_shared();
    __syncwarp();
  }
  uint32_t parity = 0;
  bool stop = false;  // a bounded wait ran out: no further work, no flush
  // column c_ of segment s_ of pair f_; in the checked build an out-of-range column is recorded
  // and read from the slab's start instead (the barrier still receives its bytes)
  auto colp = [&](int f_, int s_, int c_) -> const float2* {
    const long long o = (((long long)s_ * a.n_fpair + f_) * N1 + c_) * N2;
    return a.scratch + (in_bounds(a.err, o + N2 - 1, a.slab_elems) ? o : 0);
  };
  // the columns of units ug_ UPW .. ug_ UPW + UPW - 1 of segment s_ of FFT pair f_: unit w's
  // column c and mirror N1 - c (0 and N1/2 for unit 0) at region columns 2w, 2w + 1
  auto prefetch = [&](int f_, int ug_, int s_) {
    if constexpr (UPW == 1) {
      const int u_ = ug_;
      const int c0 = (u_ == 0) ? 0 : u_, c1 = (u_ == 0) ? N1 / 2 : N1 - u_;
      bulk_load2_elect(bar, smem_addr(region), colp(f_, s_, c0), smem_addr(region + N2), colp(f_, s_, c1),
                       (uint32_t)(N2 * sizeof(float2)));
    } else {
      if (lane == 0) {
        constexpr uint32_t bytes = (uint32_t)(N2 * sizeof(float2));
        mbar_expect_tx(bar, 2 * UPW * bytes);
        sfor<0, UPW>([&](auto w_) {
          constexpr int w = decltype(w_)::value;
          const int u_ = ug_ * UPW + w;
          const int c0 = (u_ == 0) ? 0 : u_, c1 = (u_ == 0) ? N1 / 2 : N1 - u_;
          bulk_load(bar, smem_addr(region + (2 * w) * (N2 + PL::PADC)), colp(f_, s_, c0), bytes);
          bulk_load(bar, smem_addr(region + (2 * w + 1) * (N2 + PL::PADC)), colp(f_, s_, c1), bytes);
        });
      }
      __syncwarp();
    }
  };

  // lane roles: step 1 (uw, e, q2); step 2 (uw, j)
  const int uw = lane / (2 * Q2), e1 = (lane / Q2) & 1, q2 = lane % Q2, j = lane % (2 * Q2);
  // Once a segment's columns have landed in shared memory their slab lines are dead (every
  // column is read by exactly one warp, and the slab is rewritten before it is read again):
  // drop them from L2 without a write-back, so that the slab's round trip costs no DRAM write
  // for the lines still cached when they are read.  A column is N2 / 16 lines of 128 bytes;
  // its Q2 lanes take P / 16 lines each.
  static_assert(!PF || (P % 16 == 0 && (N2 * 8) % 128 == 0), "whole lines per lane");
  auto discard = [&](int f_, int s_, int c_) {
    const char* col = reinterpret_cast<const char*>(colp(f_, s_, c_));
    sfor<0, P / 16>([&](auto i_) {
      asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(col + (q2 + Q2 * decltype(i_)::value) * 128) : "memory");
    });
  };

  const int so = (SL > 1) ? uw / UPS : 0;
  const int uoff = (SL > 1) ? uw % UPS : uw;

  if constexpr (PL::TWPQ) {
    for (int i = tid; i < P * Q2; i += PL::THREADS) {
      const int pp = i / Q2, qq = i % Q2;
      tw2[pp * PL::LDT2 + qq] = tw_small<N2>((qq * pp) & (N2 - 1));
    }
  } else {
    for (int k = tid; k < N2; k += PL::THREADS) tw2[k + (k >> 5)] = tw_small<N2>(k);
  }
  const uint32_t tbase = __shfl_sync(0xffffffffu, cta_tmem_begin<PL::TCOLS2>(tslot, warp), 0);  // (its barrier also publishes tw2)
  // (pdl_wait -- the slab written by phase 1 and the accumulators cleared by the readout are
  // visible -- comes after the first item's tensor-memory set-up, which reads neither)
  bool waited = false;
  const uint32_t t_acc = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * (PL::TCOLS2 / 2));
  const uint32_t t_tw = t_acc + TACC;

  const int R = (a.nseg + SL - 1) / SL;                // rounds of SL segments
  const int NRG = (R + range_len - 1) / range_len;     // ranges per (pair, unit group)
  const long long n_items = (long long)a.n_fpair * UGW * NRG;
  const long long nw = (long long)gridDim.x * PL::WARPS;
  for (long long item = (long long)blockIdx.x * PL::WARPS + warp; item < n_items; item += nw) {
    const int rg = (int)(item % NRG);
    const long long fug = item / NRG;
    const int r_begin = rg * range_len, r_end = min(R, r_begin + range_len);
    const int ug = (int)(fug % UGW), f = (int)(fug / UGW);
    const int u = (SL > 1) ? uoff : ug * UPW + uoff;
    const int c = (u == 0) ? (e1 ? N1 / 2 : 0) : (e1 ? N1 - u : u);
    const int tu = (u == 0 && e1) ? N1 / 2 : u;
    const bool special = (u == 0);
    const bool warp_special = (SL > 1) || (ug == 0);  // some lane of this warp holds unit 0
    // tensor memory: zero the accumulators, load this lane's twiddles W_N^{b tu}, b = q2 + Q2 t
    sfor<0, TACC / 16>([&](auto c_) {
      constexpr int cc = decltype(c_)::value;
      float z16[16];
      sfor<0, 16>([&](auto k_) { z16[decltype(k_)::value] = 0.f; });
      tmem_st16(t_acc + 16 * cc, z16);
    });
    sfor<0, PL::TTW / 16>([&](auto c_) {
      constexpr int cc = decltype(c_)::value;
      float w16[16];
      sfor<0, 8>([&](auto k_) {
        constexpr int k = decltype(k_)::value;
        constexpr int t = 8 * cc + k;
        float2 w = make_float2(0.f, 0.f);
        if constexpr (t < P) w = __ldg(a.tw + (size_t)tu * N2 + (q2 + Q2 * t));
        w16[2 * k] = w.x;
        w16[2 * k + 1] = w.y;
      });
      tmem_st16(t_tw + 16 * cc, w16);
    });
    tmem_wait_st();
    if (!waited) {
      pdl_wait();
      waited = true;
    }
    float extra[4] = {0.f, 0.f, 0.f, 0.f};
    bool worked = false;
    if constexpr (PF) {
      if (r_begin < r_end) {
        fence_async_shared();  // the previous item's shared reads of the region come first
        __syncwarp();
        prefetch(f, ug, r_begin);
      }
    }
    // after the region is free: start the next segment's copy
    auto next_prefetch = [&](int rnd_) {
      if constexpr (PF) {
        if (rnd_ + 1 < r_end) {
          fence_async_shared();  // this warp's shared reads before the copy's writes
          __syncwarp();
          prefetch(f, ug, rnd_ + 1);
        }
      }
    };
    for (int rnd = r_begin; rnd < r_end; ++rnd) {
      const int s = rnd * SL + so;
      const bool act = s < a.nseg;
      worked |= act;
      // step 1: load the column, twiddle, P-point DFT
      float2 v[P];
      if constexpr (PF) {
        if (!mbar_wait_bounded(bar, parity, a.wait_limit)) {
          if (lane == 0 && a.err) atomicExch(a.err, 1);
          mbar_wait_bounded(bar, parity, kWaitAfterTimeout);  // the copy in flight lands first
          stop = true;
        }
        parity ^= 1u;
        if (stop) break;
        sfor<0, P>([&](auto t_) {
          constexpr int t = decltype(t_)::value;
          v[ct::bitrev(t, P)] = region[(uw * 2 + e1) * (N2 + PL::PADC) + q2 + Q2 * t];
        });
        __syncwarp();  // every lane has its column before the transpose overwrites the region
      } else {
        const long long so = ((long long)(act ? s : 0) * a.n_fpair + f) * N1 * N2 + (long long)c * N2 + q2;
        const float2* src = a.scratch + so;
        sfor<0, P>([&](auto t_) {
          constexpr int t = decltype(t_)::value;
          v[ct::bitrev(t, P)] = (act && in_bounds(a.err, so + Q2 * t, a.slab_elems)) ? __ldcg(src + Q2 * t)
                                                                                       : make_float2(0.f, 0.f);
        });
      }
      sfor<0, (P + 7) / 8>([&](auto c_) {
        constexpr int cc = decltype(c_)::value;
        float w16[16];
        tmem_ld16(t_tw + 16 * cc, w16);
        tmem_wait_ld();
        sfor<0, 8>([&](auto k_) {
          constexpr int k = decltype(k_)::value;
          constexpr int t = 8 * cc + k;
          if constexpr (t < P) {  // (a mirror column arrives conjugated from phase 1)
            v[ct::bitrev(t, P)] = cmul(v[ct::bitrev(t, P)], make_float2(w16[2 * k], w16[2 * k + 1]));
          }
        });
      });
      dit<P>(v);
      // joint transpose through the warp's region
      sfor<0, P>([&](auto p_) {
        constexpr int p = decltype(p_)::value;
        region[(uw * 2 + e1) * LDE + p * LDQ + q2] = v[p];
      });
      __syncwarp();
      float2 wv[2 * PP * Q2];
      sfor<0, PP>([&](auto r_) {
        constexpr int r = decltype(r_)::value;
        const int p = j * PP + r;
        sfor<0, Q2>([&](auto q_) {
          constexpr int q = decltype(q_)::value;
          float2 w = make_float2(1.f, 0.f);
          if constexpr (q > 0) {
            if constexpr (PL::TWPQ) {
              w = tw2[p * PL::LDT2 + q];
            } else {
              const int k = (q * p) & (N2 - 1);
              w = tw2[k + (k >> 5)];
            }
          }
          sfor<0, 2>([&](auto e_) {
            constexpr int e = decltype(e_)::value;
            const float2 z = region[(uw * 2 + e) * LDE + p * LDQ + q];
            wv[(e * PP + r) * Q2 + ct::bitrev(q, Q2)] = (q > 0) ? cmul(z, w) : z;
          });
        });
        sfor<0, 2>([&](auto e_) {
          constexpr int e = decltype(e_)::value;
          dit<Q2, (e * PP + r) * Q2, 1>(wv);
        });
      });
      __syncwarp();  // region consumed
      if (!warp_special) next_prefetch(rnd);
      float2* s0 = region + (uw * 2 + 0) * N2;  // unit 0 mirror exchange: column 0
      float2* sh = region + (uw * 2 + 1) * N2;  //                         column N1/2
      if (warp_special) {
        if (special) {
          sfor<0, 2>([&](auto e_) {
            constexpr int e = decltype(e_)::value;
            sfor<0, PP>([&](auto r_) {
              constexpr int r = decltype(r_)::value;
              sfor<0, Q2>([&](auto m_) {
                constexpr int m = decltype(m_)::value;
                region[(uw * 2 + e) * N2 + j * PP + r + P * m] = wv[(e * PP + r) * Q2 + m];
              });
            });
          });
        }
        __syncwarp();
      }
      // correlate into the tensor-memory accumulators.  SP: this lane's unit is unit 0
      // (column 0 and N1/2, from the mirror area); with one unit per warp and one segment per
      // round that, and act, are the same for the whole warp and are decided once per segment.
      auto correlate = [&](auto sp_) {
        constexpr int SPK = decltype(sp_)::value;  // 0: not special, 1: special, 2: decided per lane
        sfor<0, (NACC + 3) / 4>([&](auto c_) {
          constexpr int cc = decltype(c_)::value;
          float a16[16];
          tmem_ld16(t_acc + 16 * cc, a16);
          tmem_wait_ld();
          if (act) {
            sfor<0, 4>([&](auto k_) {
              constexpr int slot = 4 * cc + decltype(k_)::value;
              if constexpr (slot < NACC) {
                constexpr int r = slot / Q2, m = slot % Q2;
                float(&q)[4] = *reinterpret_cast<float(*)[4]>(a16 + 4 * (slot - 4 * cc));
                auto special_bin = [&]() {
                  const int d = j * PP + r + P * m;
                  float2 Uv, Vv;
                  if (d <= N2 / 2) {  // column 0: bins N1 d, mirror N1 (N2 - d)
                    Uv = s0[d];
                    const float2 t = s0[(N2 - d) & (N2 - 1)];
                    Vv = make_float2(t.x, -t.y);
                  } else {  // column N1/2 at dh = d - N2/2 - 1: bins N1/2 + N1 dh, mirror N2 - 1 - dh
                    const int dh = d - N2 / 2 - 1;
                    Uv = sh[dh];
                    const float2 t = sh[N2 - 1 - dh];
                    Vv = make_float2(t.x, -t.y);
                  }
                  corr_acc(q, Uv, Vv);
                };
                if constexpr (SPK == 0) {
                  corr_acc(q, wv[r * Q2 + m], wv[(PP + r) * Q2 + m]);
                } else if constexpr (SPK == 1) {
                  special_bin();
                } else {
                  if (!special) corr_acc(q, wv[r * Q2 + m], wv[(PP + r) * Q2 + m]);
                  else special_bin();
                }
              }
            });
          }
          tmem_st16(t_acc + 16 * cc, a16);
        });
      };
      if constexpr (UPW == 1 && SL == 1) {
        if (special) correlate(std::integral_constant<int, 1>{});
        else correlate(std::integral_constant<int, 0>{});
      } else {
        correlate(std::integral_constant<int, 2>{});
      }
      tmem_wait_st();
      if (act && special && j == 0) {  // the one extra bin: column N1/2 at dh = N2/2 - 1
        const float2 t = sh[N2 / 2];
        corr_acc(extra, sh[N2 / 2 - 1], make_float2(t.x, -t.y));
      }
      if (warp_special) {
        __syncwarp();  // mirror area read before the next transpose
        next_prefetch(rnd);
      }
      if constexpr (PF) discard(f, s, c);  // (this segment's copy completed at the wait above)
    }
    if (stop) break;
    // flush this lane's sums into the integration accumulators (native order; the range's copy)
    const int copy = a.acc_copies > 1 ? rg % a.acc_copies : 0;
    const size_t base = ((size_t)copy * a.n_fpair + f) * PL::NATIVE;
    sfor<0, (NACC + 3) / 4>([&](auto c_) {
      constexpr int cc = decltype(c_)::value;
      float a16[16];
      tmem_ld16(t_acc + 16 * cc, a16);
      tmem_wait_ld();
      if (worked) {
        sfor<0, 4>([&](auto k_) {
          constexpr int slot = 4 * cc + decltype(k_)::value;
          if constexpr (slot < NACC) {
            constexpr int r = slot / Q2, m = slot % Q2;
            const int d = j * PP + r + P * m;
            const float* q = a16 + 4 * (slot - 4 * cc);
            const size_t o = base + (size_t)u * N2 + d;
            if (!in_bounds(a.err, (long long)o, a.acc_slots)) {
            } else if (!a.fp64) {
              atomicAdd(reinterpret_cast<float4*>(a.acc) + o, make_float4(q[0], q[1], q[2], q[3]));
            } else {
              double* op = reinterpret_cast<double*>(a.acc) + 4 * o;
              atomicAdd(op + 0, (double)q[0]);
              atomicAdd(op + 1, (double)q[1]);
              atomicAdd(op + 2, (double)q[2]);
              atomicAdd(op + 3, (double)q[3]);
            }
          }
        });
      }
    });
    if (worked && special && j == 0 && in_bounds(a.err, (long long)(base + (size_t)UPS * N2), a.acc_slots)) {
      const size_t o = base + (size_t)UPS * N2;
      if (!a.fp64) {
        atomicAdd(reinterpret_cast<float4*>(a.acc) + o, make_float4(extra[0], extra[1], extra[2], extra[3]));
      } else {
        double* op = reinterpret_cast<double*>(a.acc) + 4 * o;
        atomicAdd(op + 0, (double)extra[0]);
        atomicAdd(op + 1, (double)extra[1]);
        atomicAdd(op + 2, (double)extra[2]);
        atomicAdd(op + 3, (double)extra[3]);
      }
    }
  }
  pdl_trigger();
  cta_tmem_end<PL::TCOLS2>(tbase, warp);
}

// ------------------------------------------------------------------------------------------
// host-side launchers (instantiated once per N): persistent grids, as many CTAs as fit
// ------------------------------------------------------------------------------------------
// CTAs of `kernel` that fit on one SM at once: the larger of the occupancy API's answer and
// a direct count from the kernel's registers and shared memory (the API has been seen to
// return 1 for these kernels although two fit).  The kernels never wait on one another, so
// a CTA beyond what fits simply starts later.
template <typename K>
static int ctas_per_sm(K kernel, int threads, size_t smem, int tmem_cols) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  cudaFuncAttributes fa;
  int manual = 1;
  int dev = 0, regs_sm = 65536, smem_sm = 233472;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess && fa.numRegs > 0) {
    const int by_regs = regs_sm / (fa.numRegs * threads);
    const int by_smem = smem_sm / (int)(smem + fa.sharedSizeBytes + 1024);
    const int by_threads = 2048 / threads;
    manual = by_regs < by_smem ? by_regs : by_smem;
    manual = manual < by_threads ? manual : by_threads;
  } else {
    cudaGetLastError();
  }
  n = n > manual ? n : manual;
  const int by_tmem = 512 / tmem_cols;  // each CTA holds tmem_cols of the SM's 512 columns
  n = n < by_tmem ? n : by_tmem;
  return n < 1 ? 1 : n;
}

// Tensor map over the slab of one batch, rows (pair-segment, c) x columns b of 8-byte
// complex values; box = box_cols columns x box_rows rows of an output block, laid out in
// shared memory with the given swizzle.
static cudaError_t encode_slab_map(CUtensorMap* map, float2* slab, long long rows, int n2, int box_cols, int box_rows,
                                   CUtensorMapSwizzle swizzle) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)n2, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n2 * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, slab, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map over one IF's packed input: 32-bit words x rows (row_bytes apart) x segments
// (seg_bytes apart); box = one tile's words of box_rows rows of one segment.  Fails (and
// phase 1 then stages with cp.async) for an address that is not 16-byte aligned.
static cudaError_t encode_input_map(CUtensorMap* map, const uint32_t* base, int words_per_row, int rows, int box_rows,
                                    long long segs, long long row_bytes, long long seg_bytes, int box_words) {
  if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return cudaErrorMisalignedAddress;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
      return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[3] = {(cuuint64_t)words_per_row, (cuuint64_t)rows, (cuuint64_t)segs};
  const cuuint64_t strides[2] = {(cuuint64_t)row_bytes, (cuuint64_t)seg_bytes};
  const cuuint32_t box[3] = {(cuuint32_t)box_words, (cuuint32_t)box_rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, const_cast<uint32_t*>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int LOGN, int BITS>
static cudaError_t launch_phase1(const BatchArgs& a, cudaStream_t st, bool pdl) {
  using PL = Plan<LOGN>;
  static int attr_dev = -1, per_sm = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k_phase1<LOGN, BITS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PL::template Stage1<BITS>::SMEM);
    if (e != cudaSuccess) return e;
    per_sm = ctas_per_sm(k_phase1<LOGN, BITS>, PL::THREADS, PL::template Stage1<BITS>::SMEM, PL::TCOLS1);
    attr_dev = dev;
  }
  using ST = typename PL::template Stage1<BITS>;
  // The tensor maps (slab output, packed input) depend only on the pointers and sizes below;
  // the last four sets per instance are kept, so that steady streaming (one or a few
  // handles feeding equal chunks) encodes none of them again.
  struct MapKey {
    const void* scratch;
    long long slab_rows, hop_w;
    const void* base[2][kMaxIF];
    long long nsrc[2][kMaxIF];
  };
  struct MapSet {
    MapKey key;
    alignas(64) CUtensorMap slab;
    InMaps in;
    bool valid;
  };
  static thread_local MapSet cache[4];
  static thread_local int cache_next = 0;
  MapKey key;
  memset(&key, 0, sizeof key);
  key.scratch = a.scratch;
  key.slab_rows = (long long)a.nseg * a.n_fpair * PL::N1;
  key.hop_w = a.in.hop_w;
  const int seg_end = a.seg0 + a.nseg;  // segments [0, seg_end) of the feed are addressable
  for (int f = 0; f < a.n_fpair; ++f)
    for (int k = 0; k < 2; ++k) {
      const int ifx = k == 0 ? a.fa[f] : a.fb[f];
      if (ifx < 0) continue;
      key.base[0][ifx] = a.in.src0[ifx];
      key.base[1][ifx] = a.in.src1[ifx];
      key.nsrc[0][ifx] = a.in.n0;
      key.nsrc[1][ifx] = (long long)seg_end - a.in.n0;
    }
  MapSet* ms = nullptr;
  for (auto& c : cache)
    if (c.valid && memcmp(&c.key, &key, sizeof key) == 0) ms = &c;
  if (!ms) {
    ms = &cache[cache_next];
    cache_next = (cache_next + 1) % 4;
    ms->valid = false;
    memset(&ms->slab, 0, sizeof ms->slab);
    if constexpr (ST::TMA_OUT || ST::JOINT_OUT) {  // the kernel's TMA output paths
      if ((reinterpret_cast<uintptr_t>(a.scratch) & 15) != 0) return cudaErrorMisalignedAddress;
      const cudaError_t e =
          ST::TMA_OUT ? encode_slab_map(&ms->slab, a.scratch, key.slab_rows, PL::N2, PL::CW, PL::N1,
                                        CU_TENSOR_MAP_SWIZZLE_NONE)
                      : encode_slab_map(&ms->slab, a.scratch, key.slab_rows, PL::N2, ST::JC, ST::BOXR,
                                        ST::JSW == 7 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B);
      if (e != cudaSuccess) return e;
    }
    // input maps for TMA staging (else the kernel stages with cp.async)
    ms->in.use = 0;
    if constexpr (ST::TMA_IN) {
      const long long row_bytes = (long long)PL::N2 * BITS / 8, seg_bytes = a.in.hop_w * 4;
      bool ok = row_bytes % 16 == 0 && seg_bytes % 16 == 0;
      for (int f = 0; f < a.n_fpair && ok; ++f)
        for (int k = 0; k < 2 && ok; ++k) {
          const int ifx = k == 0 ? a.fa[f] : a.fb[f];
          if (ifx < 0) continue;
          for (int src = 0; src < 2 && ok; ++src) {
            const long long nseg_src = key.nsrc[src][ifx];
            if (nseg_src <= 0) continue;
            const uint32_t* base = src == 0 ? a.in.src0[ifx] : a.in.src1[ifx];
            ok = encode_input_map(&ms->in.m[src][ifx], base, PL::N2 * BITS / 32, PL::N1, ST::BOXR, nseg_src,
                                  row_bytes, seg_bytes, ST::WPR) == cudaSuccess;
          }
        }
      ms->in.use = ok ? 1 : 0;
    }
    ms->key = key;
    ms->valid = true;
  }
  const long long cols = (long long)a.nseg * a.n_fpair * PL::N2;
  // staged: one unit (a tile, or half of one in the last round) per CTA pass
  const long long ctas = ST::STAGED ? (cols / ST::TILE) * ST::IPT
                                     : ((cols + PL::CW - 1) / PL::CW + PL::WARPS - 1) / PL::WARPS;
  const int eff = (a.cap1 > 0 && a.cap1 < per_sm) ? a.cap1 : per_sm;
  const long long cap = (long long)eff * a.num_sms;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ctas < cap ? ctas : cap));
  cfg.blockDim = dim3(PL::THREADS);
  cfg.dynamicSmemBytes = ST::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_phase1<LOGN, BITS>, a, ms->slab, ms->in);
}

// phase 1 of one batch
template <int LOGN>
cudaError_t run_phase1(const BatchArgs& a, cudaStream_t st, bool pdl) {
  if (a.nseg <= 0) return cudaSuccess;
  switch (a.bits) {
    case 1: return launch_phase1<LOGN, 1>(a, st, pdl);
    case 2: return launch_phase1<LOGN, 2>(a, st, pdl);
    case 4: return launch_phase1<LOGN, 4>(a, st, pdl);
    case 8: return launch_phase1<LOGN, 8>(a, st, pdl);
    default: return cudaErrorInvalidValue;
  }
}

// phase 2 of one batch: items (pair, unit group, range of segments), about one per warp
template <int LOGN>
cudaError_t run_phase2(const BatchArgs& a, cudaStream_t st, bool pdl) {
  using PL = Plan<LOGN>;
  if (a.nseg <= 0) return cudaSuccess;
  static int attr_dev = -1, per_sm = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (attr_dev != dev) {
    cudaError_t e = cudaFuncSetAttribute(k_phase2<LOGN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::SMEM2);
    if (e != cudaSuccess) return e;
    per_sm = ctas_per_sm(k_phase2<LOGN>, PL::THREADS, PL::SMEM2, PL::TCOLS2);
    attr_dev = dev;
  }
  const int eff = (a.cap2 > 0 && a.cap2 < per_sm) ? a.cap2 : per_sm;
  const long long warps = (long long)eff * a.num_sms * PL::WARPS;
  const int R = (a.nseg + PL::SL - 1) / PL::SL;
  const long long groups = (long long)a.n_fpair * PL::UGW;
  // as many segment ranges per (pair, unit group) as leave every warp at most one item; the
  // ranges of one group go to consecutive warps (they share the group's twiddles and slab
  // columns)
  long long nrg = warps / groups;
  if (nrg < 1) nrg = 1;
  if (nrg > R) nrg = R;
  const long long range_len = (R + nrg - 1) / nrg;  // rounds per item
  const long long n_items = groups * ((R + range_len - 1) / range_len);
  const long long ctas = (n_items + PL::WARPS - 1) / PL::WARPS;
  const long long cap = (long long)eff * a.num_sms;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ctas < cap ? ctas : cap));
  cfg.blockDim = dim3(PL::THREADS);
  cfg.dynamicSmemBytes = PL::SMEM2;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k_phase2<LOGN>, a, (int)range_len);
}

}  // namespace polaris

#define POLARIS_INSTANTIATE(LOGN)                                                          \
  template cudaError_t polaris::run_phase1<LOGN>(const polaris::BatchArgs&, cudaStream_t, bool); \
  template cudaError_t polaris::run_phase2<LOGN>(const polaris::BatchArgs&, cudaStream_t, bool);
