// C ABI of the PolariS hot path (declared in include/polaris.h) and the two small
// kernels that sit around the FFT-correlator: the stand-alone data-translation kernel
// (bit-exact checks) and the readout kernel that turns the integration accumulators
// into autos, crosses and Stokes I, Q, U, V (Eq. 2).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/polaris.h"
#include "polaris_kernels.cuh"
#include "polaris_tuning.h"

namespace polaris {
// per-size phase runners, one translation unit each (polaris_n<LOGN>.cu)
#define POLARIS_DECLARE(LOGN)                                                    \
  extern template cudaError_t run_phase1<LOGN>(const BatchArgs&, cudaStream_t, bool); \
  extern template cudaError_t run_phase2<LOGN>(const BatchArgs&, cudaStream_t, bool);
POLARIS_DECLARE(4)
POLARIS_DECLARE(5)
POLARIS_DECLARE(6)
POLARIS_DECLARE(7)
POLARIS_DECLARE(8)
POLARIS_DECLARE(9)
POLARIS_DECLARE(10)
POLARIS_DECLARE(11)
POLARIS_DECLARE(12)
POLARIS_DECLARE(13)
POLARIS_DECLARE(14)
POLARIS_DECLARE(15)
POLARIS_DECLARE(16)
POLARIS_DECLARE(17)
POLARIS_DECLARE(18)
POLARIS_DECLARE(19)
POLARIS_DECLARE(20)
#undef POLARIS_DECLARE

// (args, stream, programmatic dependent launch on the predecessor in `stream`)
typedef cudaError_t (*phase_fn)(const BatchArgs&, cudaStream_t, bool);
// per-IF code histograms of segments [0, nseg) of `in` (polaris_stats.cu)
cudaError_t launch_code_hist(const SegSrc& in, int n_if, int bits, int nseg, int64_t n_fft,
                             unsigned long long* hist, int* err, int num_sms, cudaStream_t st);
// the staged data translation of phase 1 alone (polaris_debug.cu)
bool phase1_staged(int logn, int bits);
cudaError_t launch_unpack_staged(int logn, int bits, const uint32_t* pa, const uint32_t* pb, long long nseg, int dense,
                                 float* oa, float* ob, cudaStream_t st);
#define POLARIS_ROW(LOGN) {run_phase1<LOGN>, run_phase2<LOGN>}
static const phase_fn kPhases[21][2] = {
    {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr},
    POLARIS_ROW(4),  POLARIS_ROW(5),  POLARIS_ROW(6),  POLARIS_ROW(7),  POLARIS_ROW(8),  POLARIS_ROW(9),
    POLARIS_ROW(10), POLARIS_ROW(11), POLARIS_ROW(12), POLARIS_ROW(13), POLARIS_ROW(14), POLARIS_ROW(15),
    POLARIS_ROW(16), POLARIS_ROW(17), POLARIS_ROW(18), POLARIS_ROW(19), POLARIS_ROW(20)};
#undef POLARIS_ROW

// ---------------------------------------------------------------------------------------
// data translation alone
// ---------------------------------------------------------------------------------------
template <int BITS>
__global__ void k_unpack(const uint32_t* __restrict__ w, long long n, float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long bit = (unsigned long long)i * BITS;
  out[i] = decode_level<BITS>(w[bit >> 5], (uint32_t)(bit & 31u));
}

// ---------------------------------------------------------------------------------------
// readout + Stokes (Eq. 2).  One thread per output bin k and FFT pair f.
// Native accumulator order of FFT pair f (k = c + N1 d):
//   c = 0         : slot d              (d = 0 .. N2/2)
//   c = N1/2      : slot N2/2 + 1 + d   (d = 0 .. N2/2 - 2), d = N2/2 - 1 in slot UPS*N2
//   0 < c < N1/2  : slot c N2 + d       (d < N2/2)
//   c > N1/2      : slot (N1 - c) N2 + (N2 - 1 - d), cross conjugated
// Each slot holds sum |S|^2, |D|^2 and Re, Im of i S conj(D) with S = 2X, D = 2iY.
// ---------------------------------------------------------------------------------------
struct ReadoutArgs {
  void* acc;  // read, then cleared: [copies][FFT pair][native slot]
  int copies;             // accumulator copies summed per slot (0 or 1: one)
  long long copy_stride;  // slots per copy
  int fp64;
  int N1, N2, UPS, nbin, native;
  int fa[kMaxIF], fb[kMaxIF], fcorr[kMaxIF];
  float* autos;
  float* cross;
  float* stokes;
  int feed;
  float c2, s2;
  float inv_ga2[kMaxIF], inv_gb2[kMaxIF], ig_re[kMaxIF], ig_im[kMaxIF];  // 1/|Ga|^2, 1/|Gb|^2, 1/(Ga conj Gb)
  const int* err;  // nonzero: a phase kernel gave up a wait; every output is NaN
  long long acc_slots;  // accumulator slots over all copies (read by the checked build)
};

// Readout of one block: a tile of CT consecutive columns c times DT consecutive values of d,
// i.e. the natural bins k = c + N1 d of those (c, d).  Reads walk the native layout along d
// (runs of DT consecutive or reversed slots per c: 256 contiguous bytes), writes walk k (CT
// consecutive bins per d: 128-byte lines per output array); a padded shared tile turns one
// into the other.  The map k -> native slot is a bijection, so the block also clears the
// slots it read: the accumulators start the next integration at zero without a memset.
// Bins per block.  At 2^17 with three integrations in flight, 1024 and 2048 bins (4 and 8 per
// thread) ran at 613k and 601k Msample/s against 615k with 512; alone, the 2048-bin readout
// took 12.1 us instead of 8.2 (a quarter of the blocks) and one handle's rate fell 6%.
#ifndef POLARIS_READOUT_TILE
#define POLARIS_READOUT_TILE 512
#endif
constexpr int kReadoutTile = POLARIS_READOUT_TILE;
constexpr int kReadoutThreads = 256;
constexpr int readout_ct(int n1) { return n1 < 32 ? n1 : 32; }

template <int LN1>
__global__ void __launch_bounds__(kReadoutThreads) k_readout(ReadoutArgs a) {
  constexpr int N1 = 1 << LN1;
  constexpr int CT = readout_ct(N1), DT = kReadoutTile / CT;
  constexpr int PT = kReadoutTile / kReadoutThreads;  // entries per thread
  __shared__ float4 tile[DT * (CT + 1)];
  asm volatile("griddepcontrol.wait;\n" ::: "memory");  // accumulators complete (dependent launch)
  // the next feed's phase 1 may set up alongside (it waits for this grid before touching data)
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  const int f = blockIdx.y, N2 = a.N2;
  constexpr int CB = N1 / CT;  // column blocks
  const int c0 = (blockIdx.x % CB) * CT, d0 = (blockIdx.x / CB) * DT;
  const size_t fo = (size_t)f * a.native;
  int slot[PT], sidx[PT];
  float4 v[PT];
  // all loads first (several in flight per thread), then the clears and the shared stores;
  // consecutive threads take consecutive d of one column
#pragma unroll
  for (int i = 0; i < PT; ++i) {
    const int e = threadIdx.x + i * kReadoutThreads;
    slot[i] = -1;
    const int dd = e % DT, cc = e / DT, c = c0 + cc, d = d0 + dd;
    const int k = c + N1 * d;
    if (k >= a.nbin) continue;
    int idx;
    if (c == 0) idx = d;
    else if (c == N1 / 2) idx = (d <= N2 / 2 - 2) ? N2 / 2 + 1 + d : a.UPS * N2;
    else if (c < N1 / 2) idx = c * N2 + d;
    else idx = (N1 - c) * N2 + (N2 - 1 - d);
    // (checked build: a slot outside the accumulators of every copy is recorded and skipped)
    if (!in_bounds(const_cast<int*>(a.err), (long long)(a.copies > 1 ? a.copies - 1 : 0) * a.copy_stride + fo + idx,
                   a.acc_slots))
      continue;
    slot[i] = idx;
    sidx[i] = dd * (CT + 1) + cc;
    if (a.fp64) {
      double4 w = reinterpret_cast<const double4*>(a.acc)[fo + idx];
      for (int k = 1; k < a.copies; ++k) {
        const double4 x = reinterpret_cast<const double4*>(a.acc)[(size_t)k * a.copy_stride + fo + idx];
        w = make_double4(w.x + x.x, w.y + x.y, w.z + x.z, w.w + x.w);
      }
      v[i] = make_float4((float)(0.25 * w.x), (float)(0.25 * w.y), (float)(0.25 * w.z), (float)(0.25 * w.w));
    } else {
      float4 w = reinterpret_cast<const float4*>(a.acc)[fo + idx];
      for (int k = 1; k < a.copies; ++k) {
        const float4 x = reinterpret_cast<const float4*>(a.acc)[(size_t)k * a.copy_stride + fo + idx];
        w = make_float4(w.x + x.x, w.y + x.y, w.z + x.z, w.w + x.w);
      }
      v[i] = make_float4(0.25f * w.x, 0.25f * w.y, 0.25f * w.z, 0.25f * w.w);
    }
    if (c > N1 / 2) v[i].w = -v[i].w;  // mirror column: conjugate
  }
#pragma unroll
  for (int i = 0; i < PT; ++i) {
    if (slot[i] < 0) continue;
    for (int k = 0; k < (a.copies > 1 ? a.copies : 1); ++k) {
      const size_t o = (size_t)k * a.copy_stride + fo + slot[i];
      if (a.fp64) reinterpret_cast<double4*>(a.acc)[o] = make_double4(0.0, 0.0, 0.0, 0.0);
      else reinterpret_cast<float4*>(a.acc)[o] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    tile[sidx[i]] = v[i];
  }
  __syncthreads();
  const bool failed = a.err && *a.err != 0;
  const int p = a.fcorr[f];
  float* autos_a = a.autos ? a.autos + (size_t)a.fa[f] * a.nbin : nullptr;
  float* autos_b = (a.autos && a.fb[f] >= 0) ? a.autos + (size_t)a.fb[f] * a.nbin : nullptr;
  float2* cross = (a.cross && p >= 0) ? reinterpret_cast<float2*>(a.cross) + (size_t)p * a.nbin : nullptr;
  float* stokes = (a.stokes && p >= 0) ? a.stokes + (size_t)p * 4 * a.nbin : nullptr;
  float inv_ga2 = 0.f, inv_gb2 = 0.f, ig_re = 0.f, ig_im = 0.f;
  if (p >= 0) {
    inv_ga2 = a.inv_ga2[p];
    inv_gb2 = a.inv_gb2[p];
    ig_re = a.ig_re[p];
    ig_im = a.ig_im[p];
  }
  // consecutive threads take consecutive c of one d (consecutive bins)
  for (int e = threadIdx.x; e < kReadoutTile; e += kReadoutThreads) {
    const int cc = e % CT, dd = e / CT;
    const int k = c0 + cc + N1 * (d0 + dd);
    if (k >= a.nbin) continue;
    float4 v = tile[dd * (CT + 1) + cc];
    if (failed) {
      const float qnan = __int_as_float(0x7fc00000);
      v = make_float4(qnan, qnan, qnan, qnan);
    }
    const float xx = v.x, yy = v.y, xr = v.z, xi = v.w;
    if (autos_a) autos_a[k] = xx;
    if (autos_b) autos_b[k] = yy;
    if (cross) cross[k] = make_float2(xr, xi);
    if (stokes) {
      const float x = xx * inv_ga2, y = yy * inv_gb2;
      const float cr = xr * ig_re - xi * ig_im;
      const float ci = xr * ig_im + xi * ig_re;
      float I, Q, Uq, V;
      if (a.feed == POLARIS_FEED_LINEAR) {
        I = 0.5f * (x + y);
        Q = 0.5f * (a.c2 * (x - y) - a.s2 * 2.0f * cr);
        Uq = 0.5f * (a.s2 * (x - y) + a.c2 * 2.0f * cr);
        V = ci;
      } else {
        I = 0.5f * (x + y);
        V = 0.5f * (x - y);
        Q = a.c2 * cr - a.s2 * ci;
        Uq = a.s2 * cr + a.c2 * ci;
      }
      stokes[k] = I;
      stokes[a.nbin + k] = Q;
      stokes[2 * (size_t)a.nbin + k] = Uq;
      stokes[3 * (size_t)a.nbin + k] = V;
    }
  }
}

static dim3 readout_grid(int N1, int N2, int n_fpair) {
  const int ct = readout_ct(N1), dt = kReadoutTile / ct;
  return dim3((unsigned)((N1 / ct) * ((N2 / 2 + 1 + dt - 1) / dt)), (unsigned)n_fpair);
}

static cudaError_t launch_readout(const ReadoutArgs& r, int n_fpair, cudaStream_t st, bool pdl) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = readout_grid(r.N1, r.N2, n_fpair);
  cfg.blockDim = dim3(kReadoutThreads);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  switch (r.N1) {
#define POLARIS_RO(LN1)                                       \
  case 1 << LN1:                                              \
    return cudaLaunchKernelEx(&cfg, k_readout<LN1>, r);
    POLARIS_RO(1) POLARIS_RO(2) POLARIS_RO(3) POLARIS_RO(4) POLARIS_RO(5) POLARIS_RO(6) POLARIS_RO(7)
    POLARIS_RO(8) POLARIS_RO(9) POLARIS_RO(10) POLARIS_RO(11)
#undef POLARIS_RO
    default: return cudaErrorInvalidValue;
  }
}

static int host_plan_n2(int logn) { return 1 << plan_log_n2(logn); }

}  // namespace polaris

using namespace polaris;

// ---------------------------------------------------------------------------------------
// handle
// ---------------------------------------------------------------------------------------
struct polaris_spec {
  int n_if = 0, bits = 0, window = 0, accum_fp64 = 0, device = 0, num_sms = 0;
  int logn = 0;
  int64_t N = 0, hop = 0, nbin = 0, spw = 0;
  int N1 = 0, N2 = 0, UPS = 0, native = 0;
  int n_pair = 0, n_fpair = 0;
  int fa[kMaxIF], fb[kMaxIF], fcorr[kMaxIF];
  int max_batch = 0;
  int cap1 = 0, cap2 = 0;  // CTAs per SM of phase 1 / phase 2 at most (0: as many as fit)
  int acc_copies = 1;
  float* d_taps = nullptr;
  float2* d_tw = nullptr;
  void* d_acc = nullptr;
  float2* d_scratch = nullptr;
  uint32_t* d_carry[2] = {nullptr, nullptr};  // ping-pong, each n_if * carry_words_cap
  int carry_sel = 0;
  int64_t carry_len = 0;                      // carried samples per IF
  uint32_t* d_stage = nullptr;                // n_if * stage_words_cap
  uint32_t* d_in = nullptr;                   // n_if * in_words_cap (host-fed input)
  int64_t in_words_cap = 0;
  int64_t carry_words_cap = 0, stage_words_cap = 0;
  float* d_out_autos = nullptr;
  float* d_out_cross = nullptr;
  float* d_out_stokes = nullptr;
  int code_stats = 0;
  unsigned long long* d_hist = nullptr;  // [n_if][2^bits] code counts (code_stats only)
  int* d_err = nullptr;                  // device status word written by the phase kernels
  cudaEvent_t ev_h2d = nullptr;
  // two internal streams: phase 1 of batch b+1 runs beside phase 2 of batch b; the
  // slab is split into two halves used by alternate batches
  cudaStream_t st_p1 = nullptr, st_p2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_p1[2] = {nullptr, nullptr}, ev_p2[2] = {nullptr, nullptr};
  size_t slab_half = 0;  // float2 elements per slab half
  int64_t seg_acc = 0;  // segments accumulated in the open integration
  int64_t launches = 0; // kernels launched by this handle (all kinds)
  bool profiling = false;
  struct ProfRec {
    int kind;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof;      // bracketed launches not yet summed
  std::vector<cudaEvent_t> spare; // event pool
  bool broken = false;
  std::string err;
};

static thread_local std::string g_create_err;
static int64_t g_alloc_limit = -1;

static int set_err(polaris_spec* s, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s) {
    s->err = buf;
    if (code == POLARIS_ECUDA) s->broken = true;
  } else {
    g_create_err = buf;
  }
  return code;
}

#define CUDA_OR_FAIL(s, call)                                                                        \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return set_err((s), POLARIS_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// NVTX range over one public call, so that a timeline profiler shows feed and integrate
// (header-only NVTX 3: a no-op unless a tool is attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

static void drop_prof(polaris_spec* s) {
  for (auto& r : s->prof) {
    s->spare.push_back(r.a);
    s->spare.push_back(r.b);
  }
  s->prof.clear();
}

static cudaEvent_t take_event(polaris_spec* s) {
  if (!s->spare.empty()) {
    cudaEvent_t e = s->spare.back();
    s->spare.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Launch one kernel through `fn`, counting it and, when profiling, bracketing it with
// CUDA events on the launching stream.  kind: 0 phase 1, 1 phase 2, 2 readout.
template <typename F>
static cudaError_t counted_launch(polaris_spec* s, int kind, cudaStream_t st, F&& fn) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (s->profiling) {
    a = take_event(s);
    b = take_event(s);
    if (a) cudaEventRecord(a, st);
  }
  cudaError_t e = fn();
  if (e == cudaSuccess) ++s->launches;
  if (s->profiling) {
    if (a && b && e == cudaSuccess) {
      cudaEventRecord(b, st);
      s->prof.push_back({kind, a, b});
    } else {
      if (a) s->spare.push_back(a);
      if (b) s->spare.push_back(b);
    }
  }
  return e;
}

static void free_all(polaris_spec* s) {
  if (s->st_p1) cudaStreamDestroy(s->st_p1);
  if (s->st_p2) cudaStreamDestroy(s->st_p2);
  for (cudaEvent_t e : {s->ev_fork, s->ev_join, s->ev_p1[0], s->ev_p1[1], s->ev_p2[0], s->ev_p2[1]})
    if (e) cudaEventDestroy(e);
  drop_prof(s);
  for (cudaEvent_t e : s->spare) cudaEventDestroy(e);
  s->spare.clear();
  cudaFree(s->d_taps);
  cudaFree(s->d_tw);
  cudaFree(s->d_acc);
  cudaFree(s->d_scratch);
  cudaFree(s->d_carry[0]);
  cudaFree(s->d_carry[1]);
  cudaFree(s->d_stage);
  cudaFree(s->d_in);
  cudaFree(s->d_out_autos);
  cudaFree(s->d_out_cross);
  cudaFree(s->d_out_stokes);
  cudaFree(s->d_hist);
  cudaFree(s->d_err);
  if (s->ev_h2d) cudaEventDestroy(s->ev_h2d);
}

extern "C" void polaris_set_alloc_limit(int64_t bytes) { g_alloc_limit = bytes; }

// test hook of the bounds-checked build: later feeds tell the kernels half the slab each pass uses
static bool g_check_understate = false;
extern "C" int polaris_set_check_understate(int on) {
#ifdef POLARIS_CHECK
  g_check_understate = on != 0;
  return POLARIS_OK;
#else
  (void)on;
  return POLARIS_EINVAL;
#endif
}
extern "C" int polaris_checked_build(void) {
#ifdef POLARIS_CHECK
  return 1;
#else
  return 0;
#endif
}

// polls of a bounded device-side wait before it counts as timed out (test hook below)
static constexpr unsigned kDefaultWaitLimit = 1u << 20;
static unsigned g_wait_limit = kDefaultWaitLimit;
extern "C" void polaris_set_wait_limit(int64_t polls) {
  g_wait_limit = polls < 0 ? kDefaultWaitLimit : (polls > 0x7fffffff ? 0x7fffffffu : (unsigned)polls);
}

extern "C" int spectrometer_create(const polaris_config* cfg, polaris_spec** out) {
  if (!cfg || !out) return set_err(nullptr, POLARIS_EINVAL, "null config or output pointer");
  const polaris_config& c = *cfg;
  if (c.n_if < 1 || c.n_if > kMaxIF) return set_err(nullptr, POLARIS_EINVAL, "n_if must be in [1, %d]", kMaxIF);
  if (!(c.bits == 1 || c.bits == 2 || c.bits == 4 || c.bits == 8))
    return set_err(nullptr, POLARIS_EINVAL, "bits must be 1, 2, 4 or 8");
  const int64_t N = c.n_fft;
  if (N < 16 || N > (1 << 20) || (N & (N - 1)))
    return set_err(nullptr, POLARIS_EINVAL, "n_fft must be a power of two in [16, 1048576]");
  const int64_t spw = 32 / c.bits;
  if (N < spw) return set_err(nullptr, POLARIS_EINVAL, "n_fft must be at least 32/bits samples");
  const int64_t hop = c.hop == 0 ? N : c.hop;
  if (hop < 1 || hop > N || hop % spw)
    return set_err(nullptr, POLARIS_EINVAL, "hop must be in (0, n_fft] and a multiple of 32/bits");
  if (c.window < POLARIS_WIN_RECT || c.window > POLARIS_WIN_CUSTOM)
    return set_err(nullptr, POLARIS_EINVAL, "unknown window kind");
  if (c.window == POLARIS_WIN_CUSTOM && !c.taps) return set_err(nullptr, POLARIS_EINVAL, "custom window needs taps");
  if (c.max_batch_segments < 0) return set_err(nullptr, POLARIS_EINVAL, "max_batch_segments must be >= 0");
  if (c.code_stats != 0 && c.code_stats != 1) return set_err(nullptr, POLARIS_EINVAL, "code_stats must be 0 or 1");
  // correlation pairs
  int pairs[2 * kMaxIF];
  int n_pair = 0;
  if (c.pairs) {
    if (c.n_pair < 0 || 2 * c.n_pair > c.n_if) return set_err(nullptr, POLARIS_EINVAL, "bad n_pair");
    n_pair = c.n_pair;
    for (int i = 0; i < 2 * n_pair; ++i) pairs[i] = c.pairs[i];
  } else {
    if (c.n_pair != 0) return set_err(nullptr, POLARIS_EINVAL, "n_pair given without pairs");
    if (c.n_if % 2 == 0) {
      n_pair = c.n_if / 2;
      for (int i = 0; i < n_pair; ++i) {
        pairs[2 * i] = i;
        pairs[2 * i + 1] = i + n_pair;
      }
    }
  }
  int used[kMaxIF] = {0};
  for (int i = 0; i < 2 * n_pair; ++i) {
    if (pairs[i] < 0 || pairs[i] >= c.n_if) return set_err(nullptr, POLARIS_EINVAL, "pair index out of range");
    if (used[pairs[i]]++) return set_err(nullptr, POLARIS_EINVAL, "an IF appears in more than one pair");
  }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) {
    cudaGetLastError();
    return set_err(nullptr, POLARIS_ECUDA, "no CUDA device available");
  }
  if (c.device < 0 || c.device >= ndev) return set_err(nullptr, POLARIS_EINVAL, "device ordinal out of range");

  polaris_spec* s = new polaris_spec();
  s->n_if = c.n_if;
  s->bits = c.bits;
  s->window = c.window;
  s->accum_fp64 = c.accum_fp64 ? 1 : 0;
  s->device = c.device;
  s->N = N;
  s->hop = hop;
  s->spw = spw;
  s->nbin = N / 2 + 1;
  int logn = 0;
  while ((1LL << logn) < N) ++logn;
  s->logn = logn;
  s->N2 = host_plan_n2(logn);
  s->N1 = (int)(N / s->N2);
  s->UPS = s->N1 / 2;
  s->native = s->UPS * s->N2 + 1;
  s->n_pair = n_pair;
  // FFT pairs: correlation pairs first, then the remaining IFs two at a time
  int nf = 0;
  for (int p = 0; p < n_pair; ++p) {
    s->fa[nf] = pairs[2 * p];
    s->fb[nf] = pairs[2 * p + 1];
    s->fcorr[nf] = p;
    ++nf;
  }
  int pending = -1;
  for (int i = 0; i < c.n_if; ++i) {
    if (used[i]) continue;
    if (pending < 0) pending = i;
    else {
      s->fa[nf] = pending;
      s->fb[nf] = i;
      s->fcorr[nf] = -1;
      ++nf;
      pending = -1;
    }
  }
  if (pending >= 0) {
    s->fa[nf] = pending;
    s->fb[nf] = -1;
    s->fcorr[nf] = -1;
    ++nf;
  }
  s->n_fpair = nf;
  for (int f = nf; f < kMaxIF; ++f) s->fa[f] = s->fb[f] = s->fcorr[f] = -1;

  DeviceGuard dg(c.device);
  cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, c.device);
  // batch size: segments per kernel pass.  Each pass pays a ramp and a tail on every SM, so
  // the default takes large passes (each slab half up to ~256 MB, at least 64 segments);
  // the slab then streams through HBM, which has bandwidth to spare for this path.
  // (the tuned table, when it has an entry for this size and width, replaces the rule)
  const TuneEntry* tuned = nullptr;
  for (const TuneEntry& t : kTuned)
    if (t.logn == logn && t.bits == c.bits) tuned = &t;
  if (c.max_batch_segments > 0) s->max_batch = c.max_batch_segments;
  else if (tuned && tuned->max_batch > 0) s->max_batch = tuned->max_batch;
  else {
    const int64_t per_seg = (int64_t)nf * N * 8;
    int64_t mb = (256LL << 20) / per_seg;
    if (mb < 64) mb = 64;
    s->max_batch = (int)(mb > 4096 ? 4096 : mb);
  }
  if (c.max_batch_segments == 0 && tuned) {
    s->cap1 = tuned->cap1;
    s->cap2 = tuned->cap2;
  }
  s->slab_half = (size_t)s->max_batch * nf * N;
  s->carry_words_cap = N / spw;               // carried samples < N
  s->stage_words_cap = 2 * N / spw;           // staging < carry + N samples
  // Accumulator copies.  Phase 2 gives each warp one range of segments of one (pair, unit
  // group) and adds the range's sums into every slot of the group once; at small N (few
  // groups, ranges of a few segments) a slot would take ~1200 atomic adds per pass, which
  // serialise per address.  Range r adds into copy r % K (about 64 adds per copy); the
  // readout sums the copies.
  {
    const int P = plan_p(logn), Q2 = s->N2 / P, UPW = 16 / Q2;
    const int UGW = UPW > s->UPS ? 1 : s->UPS / UPW;
    const long long warps = (s->cap2 == 1 ? 1LL : 2LL) * s->num_sms * 8;  // phase-2 warps resident (8-warp CTAs)
    const long long nrg = warps / ((long long)nf * UGW);
    s->acc_copies = (int)(nrg / 64 < 1 ? 1 : (nrg / 64 > 16 ? 16 : nrg / 64));
  }
  const size_t acc_bytes = (size_t)s->acc_copies * nf * s->native * 4 * (s->accum_fp64 ? 8 : 4);
  const size_t bytes_tw = (size_t)s->N2 * (s->UPS + 1) * sizeof(float2);
  const size_t bytes_scratch = 2 * (size_t)s->max_batch * nf * N * sizeof(float2);
  const size_t bytes_carry = (size_t)c.n_if * s->carry_words_cap * 4;
  const size_t bytes_stage = (size_t)c.n_if * s->stage_words_cap * 4;
  const size_t bytes_out = (size_t)s->nbin * 4 * (c.n_if + 2 * n_pair + 4 * n_pair);
  const size_t bytes_hist = c.code_stats ? (size_t)c.n_if * ((size_t)1 << c.bits) * 8 : 0;
  const size_t total = acc_bytes + bytes_tw + bytes_scratch + 2 * bytes_carry + bytes_stage + bytes_out +
                       bytes_hist + (c.window != POLARIS_WIN_RECT ? N * 4 : 0);
  if (g_alloc_limit >= 0 && (int64_t)total > g_alloc_limit) {
    delete s;
    return set_err(nullptr, POLARIS_ENOMEM, "device allocation of %zu bytes exceeds the limit %lld", total,
                   (long long)g_alloc_limit);
  }
  auto alloc = [&](void** p, size_t bytes) -> bool {
    if (bytes == 0) bytes = 16;
    return cudaMalloc(p, bytes) == cudaSuccess;
  };
  bool ok = alloc((void**)&s->d_acc, acc_bytes) && alloc((void**)&s->d_tw, bytes_tw) &&
            alloc((void**)&s->d_scratch, bytes_scratch) && alloc((void**)&s->d_carry[0], bytes_carry) &&
            alloc((void**)&s->d_carry[1], bytes_carry) && alloc((void**)&s->d_stage, bytes_stage) &&
            alloc((void**)&s->d_out_autos, (size_t)s->nbin * 4 * c.n_if) &&
            alloc((void**)&s->d_out_cross, (size_t)s->nbin * 8 * (n_pair ? n_pair : 1)) &&
            alloc((void**)&s->d_out_stokes, (size_t)s->nbin * 16 * (n_pair ? n_pair : 1));
  if (ok && c.window != POLARIS_WIN_RECT) ok = alloc((void**)&s->d_taps, N * 4);
  if (ok && c.code_stats) ok = alloc((void**)&s->d_hist, bytes_hist);
  if (ok) ok = alloc((void**)&s->d_err, 256);
  if (!ok) {
    cudaGetLastError();
    free_all(s);
    delete s;
    return set_err(nullptr, POLARIS_ENOMEM, "cudaMalloc failed");
  }
  // twiddles W_N^{b u} for b < N2, u <= N1/2, in FP64 then rounded; unit-major ([u][b]), so
  // that the lanes of a phase-2 item (consecutive b of one unit) read one contiguous run
  std::vector<float2> tw((size_t)s->N2 * (s->UPS + 1));
  for (int b = 0; b < s->N2; ++b)
    for (int u = 0; u <= s->UPS; ++u) {
      const int64_t e = ((int64_t)b * u) % N;
      const double ang = -2.0 * M_PI * (double)e / (double)N;
      tw[(size_t)u * s->N2 + b] = make_float2((float)std::cos(ang), (float)std::sin(ang));
    }
  cudaError_t e = cudaMemcpy(s->d_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && c.window != POLARIS_WIN_RECT) {
    std::vector<float> taps(N);
    for (int64_t n = 0; n < N; ++n)
      taps[n] = c.window == POLARIS_WIN_HANN ? (float)(0.5 - 0.5 * std::cos(2.0 * M_PI * (double)n / (double)N))
                                             : c.taps[n];
    e = cudaMemcpy(s->d_taps, taps.data(), N * 4, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(s->d_acc, 0, acc_bytes);
  if (e == cudaSuccess && c.code_stats) e = cudaMemset(s->d_hist, 0, bytes_hist);
  if (e == cudaSuccess) e = cudaMemset(s->d_err, 0, 256);
  s->code_stats = c.code_stats;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_h2d, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st_p1, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->st_p2, cudaStreamNonBlocking);
  for (cudaEvent_t* ev : {&s->ev_fork, &s->ev_join, &s->ev_p1[0], &s->ev_p1[1], &s->ev_p2[0], &s->ev_p2[1]})
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_all(s);
    delete s;
    return set_err(nullptr, POLARIS_ECUDA, "create: %s", cudaGetErrorString(e));
  }
  *out = s;
  return POLARIS_OK;
}

extern "C" void spectrometer_destroy(polaris_spec* s) {
  if (!s) return;
  {
    DeviceGuard dg(s->device);
    cudaDeviceSynchronize();
    free_all(s);
  }
  delete s;
}

extern "C" const char* spectrometer_last_error(const polaris_spec* s) {
  return s ? s->err.c_str() : g_create_err.c_str();
}

extern "C" int64_t spectrometer_n_bins(const polaris_spec* s) { return s ? s->nbin : -1; }

extern "C" int spectrometer_n_pairs(const polaris_spec* s) { return s ? s->n_pair : -1; }

static int check_usable(polaris_spec* s) {
  if (!s) return POLARIS_EINVAL;
  if (s->broken) return set_err(s, POLARIS_ESTATE, "handle unusable after an earlier CUDA error: %s", s->err.c_str());
  return POLARIS_OK;
}

// After a synchronisation: a phase kernel that gave up a bounded wait has set the status
// word (its outputs are NaN); the handle becomes unusable.
static int check_device_status(polaris_spec* s) {
  int st = 0;
  const cudaError_t e = cudaMemcpy(&st, s->d_err, sizeof st, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    s->broken = true;
    return set_err(s, POLARIS_ECUDA, "status read: %s", cudaGetErrorString(e));
  }
  if (st == kErrBounds) {
    set_err(s, POLARIS_EBOUNDS, "an index check of the bounds-checked build failed; outputs are NaN");
    s->broken = true;
    return POLARIS_EBOUNDS;
  }
  if (st) {
    set_err(s, POLARIS_ETIMEOUT, "a device-side wait ran out of its bound; outputs are NaN");
    s->broken = true;
    return POLARIS_ETIMEOUT;
  }
  return POLARIS_OK;
}

extern "C" int spectrometer_feed(polaris_spec* s, const void* const* packed, int64_t n, int on_device,
                                 void* cuda_stream) {
  NvtxRange nvtx("polaris.feed");
  int rc = check_usable(s);
  if (rc) return rc;
  if (!packed) return set_err(s, POLARIS_EINVAL, "packed is NULL");
  if (n < 0 || n % s->spw) return set_err(s, POLARIS_EINVAL, "n_samples_per_if must be >= 0 and a multiple of %lld",
                                          (long long)s->spw);
  for (int i = 0; i < s->n_if; ++i) {
    if (!packed[i]) return set_err(s, POLARIS_EINVAL, "packed[%d] is NULL", i);
    if (reinterpret_cast<uintptr_t>(packed[i]) & 3) return set_err(s, POLARIS_EINVAL, "packed[%d] is not 4-byte aligned", i);
  }
  if (on_device != POLARIS_INPUT_HOST && on_device != POLARIS_INPUT_DEVICE && on_device != POLARIS_INPUT_HOST_ASYNC)
    return set_err(s, POLARIS_EINVAL, "on_device must be POLARIS_INPUT_HOST, _DEVICE or _HOST_ASYNC");
  if (n == 0) return POLARIS_OK;
  const bool host_in = on_device != POLARIS_INPUT_DEVICE;
  DeviceGuard dg(s->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  const int64_t nw = n / s->spw;
  const uint32_t* src[kMaxIF] = {nullptr};
  if (host_in) {
    if (nw > s->in_words_cap) {
      CUDA_OR_FAIL(s, cudaStreamSynchronize(st));
      cudaFree(s->d_in);
      s->d_in = nullptr;
      s->in_words_cap = 0;
      if (cudaMalloc((void**)&s->d_in, (size_t)nw * 4 * s->n_if) != cudaSuccess) {
        cudaGetLastError();
        return set_err(s, POLARIS_ENOMEM, "cannot allocate %lld bytes of device input staging",
                       (long long)(nw * 4 * s->n_if));
      }
      s->in_words_cap = nw;
    }
    // IF streams at one constant stride (rows of one host array, say) go over in one
    // pitched copy: one API call instead of one per IF (each costs host time).  The CUDA driver
    // refuses (at the call, queueing nothing) a pitched copy whose rows lie in different
    // pinned allocations; then the streams go one by one.
    const long long stride = s->n_if > 1 ? (long long)((const char*)packed[1] - (const char*)packed[0]) : 0;
    bool uniform = s->n_if > 1 && stride >= nw * 4;
    for (int i = 2; i < s->n_if && uniform; ++i)
      uniform = (long long)((const char*)packed[i] - (const char*)packed[i - 1]) == stride;
    if (uniform) {
      // contiguous on both sides (no gap between rows): one linear copy, the cheapest call
      const bool linear = stride == nw * 4 && s->in_words_cap == nw;
      const cudaError_t ec =
          linear ? cudaMemcpyAsync(s->d_in, packed[0], (size_t)nw * 4 * s->n_if, cudaMemcpyHostToDevice, st)
                 : cudaMemcpy2DAsync(s->d_in, (size_t)s->in_words_cap * 4, packed[0], (size_t)stride, (size_t)nw * 4,
                                     (size_t)s->n_if, cudaMemcpyHostToDevice, st);
      if (ec != cudaSuccess) {
        cudaGetLastError();
        uniform = false;
      }
    }
    if (!uniform) {
      for (int i = 0; i < s->n_if; ++i)
        CUDA_OR_FAIL(s, cudaMemcpyAsync(s->d_in + (size_t)i * s->in_words_cap, packed[i], (size_t)nw * 4,
                                        cudaMemcpyHostToDevice, st));
    }
    for (int i = 0; i < s->n_if; ++i) src[i] = s->d_in + (size_t)i * s->in_words_cap;
    CUDA_OR_FAIL(s, cudaEventRecord(s->ev_h2d, st));
  } else {
    for (int i = 0; i < s->n_if; ++i) src[i] = static_cast<const uint32_t*>(packed[i]);
  }
  const int64_t N = s->N, hop = s->hop, spw = s->spw;
  const int64_t carry = s->carry_len;
  const int64_t total = carry + n;
  const int64_t nseg = total >= N ? (total - N) / hop + 1 : 0;
  const int64_t n0 = nseg < (carry + hop - 1) / hop ? nseg : (carry + hop - 1) / hop;
  uint32_t* cur_carry = s->d_carry[s->carry_sel];
  if (n0 > 0) {
    const int64_t stage_len = (n0 - 1) * hop + N;  // samples: carry + (stage_len - carry) new ones
    for (int i = 0; i < s->n_if; ++i) {
      uint32_t* dst = s->d_stage + (size_t)i * s->stage_words_cap;
      if (carry)
        CUDA_OR_FAIL(s, cudaMemcpyAsync(dst, cur_carry + (size_t)i * s->carry_words_cap, (size_t)(carry / spw) * 4,
                                        cudaMemcpyDeviceToDevice, st));
      CUDA_OR_FAIL(s, cudaMemcpyAsync(dst + carry / spw, src[i], (size_t)((stage_len - carry) / spw) * 4,
                                      cudaMemcpyDeviceToDevice, st));
    }
  }
  BatchArgs a;
  memset(&a, 0, sizeof a);
  for (int i = 0; i < s->n_if; ++i) {
    a.in.src0[i] = s->d_stage + (size_t)i * s->stage_words_cap;
    a.in.src1[i] = src[i] + (n0 * hop - carry) / spw;
  }
  a.in.hop_w = hop / spw;
  a.in.n0 = (int)n0;
  a.in.in_words0 = s->stage_words_cap;
  a.in.in_words1 = nw - (n0 * hop - carry) / spw;
  for (int f = 0; f < kMaxIF; ++f) {
    a.fa[f] = s->fa[f];
    a.fb[f] = s->fb[f];
  }
  a.n_fpair = s->n_fpair;
  a.taps = s->d_taps;
  a.scratch = s->d_scratch;
  a.tw = s->d_tw;
  a.acc = s->d_acc;
  a.acc_copies = s->acc_copies;
  a.cap1 = s->cap1;
  a.cap2 = s->cap2;
  a.fp64 = s->accum_fp64;
  a.bits = s->bits;
  a.num_sms = s->num_sms;
  a.err = s->d_err;
  a.wait_limit = g_wait_limit;
  a.slab_elems = (long long)s->slab_half;
  // (test hook: half of what the pass writes and reads)
  auto understate = [&](BatchArgs& x) {
    if (g_check_understate) x.slab_elems = (long long)x.nseg * s->n_fpair * s->N / 2;
  };
  a.acc_slots = (long long)s->acc_copies * s->n_fpair * s->native;
  const phase_fn f1 = kPhases[s->logn][0], f2 = kPhases[s->logn][1];
  if (nseg > 0 && s->code_stats) {
    cudaError_t e = counted_launch(s, 3, st, [&]() {
      return launch_code_hist(a.in, s->n_if, s->bits, (int)nseg, N, s->d_hist, s->d_err, s->num_sms, st);
    });
    if (e != cudaSuccess) return set_err(s, POLARIS_ECUDA, "code-histogram launch: %s", cudaGetErrorString(e));
  }
  if (nseg > 0 && nseg <= s->max_batch) {
    // one pass: both phases on the caller's stream, each a programmatic dependent launch
    // (its CTAs set up while the previous kernel drains, then wait for it) unless launches
    // are being timed
    a.seg0 = 0;
    a.nseg = (int)nseg;
    a.scratch = s->d_scratch;
    understate(a);
    const bool pdl = st != nullptr && !s->profiling;
    cudaError_t e = counted_launch(s, 0, st, [&]() { return f1(a, st, pdl); });
    if (e != cudaSuccess) return set_err(s, POLARIS_ECUDA, "phase-1 launch: %s", cudaGetErrorString(e));
    e = counted_launch(s, 1, st, [&]() { return f2(a, st, pdl); });
    if (e != cudaSuccess) return set_err(s, POLARIS_ECUDA, "phase-2 launch: %s", cudaGetErrorString(e));
  } else if (nseg > 0) {
    // several passes: phase 1 and phase 2 on two internal streams, pass b + 1's phase 1
    // overlapping pass b's phase 2 (alternate slab halves).
    // fork: both internal streams start after everything queued so far on the caller's stream
    CUDA_OR_FAIL(s, cudaEventRecord(s->ev_fork, st));
    CUDA_OR_FAIL(s, cudaStreamWaitEvent(s->st_p1, s->ev_fork, 0));
    CUDA_OR_FAIL(s, cudaStreamWaitEvent(s->st_p2, s->ev_fork, 0));
    int b = 0;
    for (int64_t s0 = 0; s0 < nseg; s0 += s->max_batch, ++b) {
      a.seg0 = (int)s0;
      a.nseg = (int)(nseg - s0 < s->max_batch ? nseg - s0 : s->max_batch);
      a.scratch = s->d_scratch + (size_t)(b & 1) * s->slab_half;
      understate(a);
      // phase 1 of batch b may overwrite its slab half once phase 2 of batch b-2 has read it
      if (b >= 2) CUDA_OR_FAIL(s, cudaStreamWaitEvent(s->st_p1, s->ev_p2[b & 1], 0));
      cudaError_t e = counted_launch(s, 0, s->st_p1, [&]() { return f1(a, s->st_p1, false); });
      if (e != cudaSuccess) return set_err(s, POLARIS_ECUDA, "phase-1 launch: %s", cudaGetErrorString(e));
      CUDA_OR_FAIL(s, cudaEventRecord(s->ev_p1[b & 1], s->st_p1));
      CUDA_OR_FAIL(s, cudaStreamWaitEvent(s->st_p2, s->ev_p1[b & 1], 0));
      e = counted_launch(s, 1, s->st_p2, [&]() { return f2(a, s->st_p2, false); });
      if (e != cudaSuccess) return set_err(s, POLARIS_ECUDA, "phase-2 launch: %s", cudaGetErrorString(e));
      CUDA_OR_FAIL(s, cudaEventRecord(s->ev_p2[b & 1], s->st_p2));
    }
    // join: phase 2 of the last batch follows every phase 1, so waiting on st_p2 suffices
    CUDA_OR_FAIL(s, cudaEventRecord(s->ev_join, s->st_p2));
    CUDA_OR_FAIL(s, cudaStreamWaitEvent(st, s->ev_join, 0));
  }
  // carry the samples after the last whole segment: stream positions [nseg*hop, total)
  const int64_t keep0 = nseg * hop, keep = total - keep0;
  uint32_t* nxt = s->d_carry[s->carry_sel ^ 1];
  for (int i = 0; i < s->n_if && keep > 0; ++i) {
    uint32_t* dst = nxt + (size_t)i * s->carry_words_cap;
    if (keep0 >= carry) {
      CUDA_OR_FAIL(s, cudaMemcpyAsync(dst, src[i] + (keep0 - carry) / spw, (size_t)(keep / spw) * 4,
                                      cudaMemcpyDeviceToDevice, st));
    } else {
      const int64_t from_old = carry - keep0;
      CUDA_OR_FAIL(s, cudaMemcpyAsync(dst, cur_carry + (size_t)i * s->carry_words_cap + keep0 / spw,
                                      (size_t)(from_old / spw) * 4, cudaMemcpyDeviceToDevice, st));
      CUDA_OR_FAIL(s, cudaMemcpyAsync(dst + from_old / spw, src[i], (size_t)(n / spw) * 4, cudaMemcpyDeviceToDevice, st));
    }
  }
  s->carry_sel ^= 1;
  s->carry_len = keep;
  s->seg_acc += nseg;
  if (on_device == POLARIS_INPUT_HOST) CUDA_OR_FAIL(s, cudaEventSynchronize(s->ev_h2d));  // host input has been read
  return POLARIS_OK;
}

static int fill_readout(polaris_spec* s, const polaris_stokes_params* prm, ReadoutArgs& r) {
  memset(&r, 0, sizeof r);
  r.acc = s->d_acc;
  r.copies = s->acc_copies;
  r.copy_stride = (long long)s->n_fpair * s->native;
  r.err = s->d_err;
  r.acc_slots = (long long)s->acc_copies * s->n_fpair * s->native;
  r.fp64 = s->accum_fp64;
  r.N1 = s->N1;
  r.N2 = s->N2;
  r.UPS = s->UPS;
  r.nbin = (int)s->nbin;
  r.native = s->native;
  for (int f = 0; f < kMaxIF; ++f) {
    r.fa[f] = s->fa[f];
    r.fb[f] = s->fb[f];
    r.fcorr[f] = s->fcorr[f];
  }
  const int feed = prm ? prm->feed : POLARIS_FEED_LINEAR;
  if (feed != POLARIS_FEED_LINEAR && feed != POLARIS_FEED_CIRCULAR) return set_err(s, POLARIS_EINVAL, "unknown feed type");
  const double psi = prm ? prm->psi_m : 0.0;
  r.feed = feed;
  r.c2 = (float)std::cos(2.0 * psi);
  r.s2 = (float)std::sin(2.0 * psi);
  for (int p = 0; p < s->n_pair; ++p) {
    double gar = 1, gai = 0, gbr = 1, gbi = 0;
    if (prm && prm->gains) {
      gar = prm->gains[4 * p + 0];
      gai = prm->gains[4 * p + 1];
      gbr = prm->gains[4 * p + 2];
      gbi = prm->gains[4 * p + 3];
    }
    const double gaa = gar * gar + gai * gai, gbb = gbr * gbr + gbi * gbi;
    if (gaa == 0.0 || gbb == 0.0) return set_err(s, POLARIS_EINVAL, "zero gain for pair %d", p);
    // g = Ga conj(Gb); 1/g = conj(g)/|g|^2
    const double gr = gar * gbr + gai * gbi, gi = gai * gbr - gar * gbi, g2 = gr * gr + gi * gi;
    r.inv_ga2[p] = (float)(1.0 / gaa);
    r.inv_gb2[p] = (float)(1.0 / gbb);
    r.ig_re[p] = (float)(gr / g2);
    r.ig_im[p] = (float)(-gi / g2);
  }
  return POLARIS_OK;
}

extern "C" int spectrometer_integrate_device(polaris_spec* s, const polaris_stokes_params* prm, float* d_autos,
                                             float* d_cross, float* d_stokes, int64_t* n_segments_out,
                                             void* cuda_stream) {
  NvtxRange nvtx("polaris.integrate");
  int rc = check_usable(s);
  if (rc) return rc;
  if (s->seg_acc == 0) return set_err(s, POLARIS_ESTATE, "no segment accumulated since the last integrate");
  ReadoutArgs r;
  rc = fill_readout(s, prm, r);
  if (rc) return rc;
  DeviceGuard dg(s->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  r.autos = d_autos;
  r.cross = d_cross;
  r.stokes = d_stokes;
  const bool pdl = st != nullptr && !s->profiling;  // dependent launch on the last phase 2
  CUDA_OR_FAIL(s, counted_launch(s, 2, st, [&]() { return launch_readout(r, s->n_fpair, st, pdl); }));
  // (the readout has cleared the accumulators it read)
  if (n_segments_out) *n_segments_out = s->seg_acc;
  s->seg_acc = 0;
  return POLARIS_OK;
}

extern "C" int spectrometer_integrate_async(polaris_spec* s, const polaris_stokes_params* prm, float* autos,
                                            float* cross, float* stokes, int64_t* n_segments_out, void* cuda_stream) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (s->seg_acc == 0) return set_err(s, POLARIS_ESTATE, "no segment accumulated since the last integrate");
  DeviceGuard dg(s->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  rc = spectrometer_integrate_device(s, prm, s->d_out_autos, s->n_pair ? s->d_out_cross : nullptr,
                                     s->n_pair ? s->d_out_stokes : nullptr, n_segments_out, cuda_stream);
  if (rc) return rc;
  if (autos)
    CUDA_OR_FAIL(s, cudaMemcpyAsync(autos, s->d_out_autos, (size_t)s->nbin * 4 * s->n_if, cudaMemcpyDeviceToHost, st));
  if (cross && s->n_pair)
    CUDA_OR_FAIL(s, cudaMemcpyAsync(cross, s->d_out_cross, (size_t)s->nbin * 8 * s->n_pair, cudaMemcpyDeviceToHost, st));
  if (stokes && s->n_pair)
    CUDA_OR_FAIL(s, cudaMemcpyAsync(stokes, s->d_out_stokes, (size_t)s->nbin * 16 * s->n_pair, cudaMemcpyDeviceToHost,
                                    st));
  return POLARIS_OK;
}

extern "C" int spectrometer_integrate(polaris_spec* s, const polaris_stokes_params* prm, float* autos, float* cross,
                                      float* stokes, int64_t* n_segments_out) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (s->seg_acc == 0) return set_err(s, POLARIS_ESTATE, "no segment accumulated since the last integrate");
  DeviceGuard dg(s->device);
  rc = spectrometer_integrate_device(s, prm, s->d_out_autos, s->n_pair ? s->d_out_cross : nullptr,
                                     s->n_pair ? s->d_out_stokes : nullptr, n_segments_out, nullptr);
  if (rc) return rc;
  // stream-ordered after the readout; one synchronisation for all three (direct copies when
  // the caller's buffers are pinned)
  if (autos)
    CUDA_OR_FAIL(s, cudaMemcpyAsync(autos, s->d_out_autos, (size_t)s->nbin * 4 * s->n_if, cudaMemcpyDeviceToHost,
                                    nullptr));
  if (cross && s->n_pair)
    CUDA_OR_FAIL(s, cudaMemcpyAsync(cross, s->d_out_cross, (size_t)s->nbin * 8 * s->n_pair, cudaMemcpyDeviceToHost,
                                    nullptr));
  if (stokes && s->n_pair)
    CUDA_OR_FAIL(s, cudaMemcpyAsync(stokes, s->d_out_stokes, (size_t)s->nbin * 16 * s->n_pair,
                                    cudaMemcpyDeviceToHost, nullptr));
  CUDA_OR_FAIL(s, cudaStreamSynchronize(nullptr));
  return check_device_status(s);
}

extern "C" int spectrometer_debug_unpack(polaris_spec* s, const void* packed, int64_t n, float* out) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (!packed || !out) return set_err(s, POLARIS_EINVAL, "null pointer");
  if (n < 0 || n % s->spw) return set_err(s, POLARIS_EINVAL, "n must be >= 0 and a multiple of %lld", (long long)s->spw);
  if (n == 0) return POLARIS_OK;
  DeviceGuard dg(s->device);
  uint32_t* dw = nullptr;
  float* df = nullptr;
  const size_t nw = (size_t)(n / s->spw);
  if (cudaMalloc((void**)&dw, nw * 4) != cudaSuccess || cudaMalloc((void**)&df, (size_t)n * 4) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dw);
    cudaFree(df);
    return set_err(s, POLARIS_ENOMEM, "debug_unpack allocation failed");
  }
  cudaError_t e = cudaMemcpy(dw, packed, nw * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const unsigned grid = (unsigned)((n + 255) / 256);
    switch (s->bits) {
      case 1: k_unpack<1><<<grid, 256>>>(dw, n, df); break;
      case 2: k_unpack<2><<<grid, 256>>>(dw, n, df); break;
      case 4: k_unpack<4><<<grid, 256>>>(dw, n, df); break;
      default: k_unpack<8><<<grid, 256>>>(dw, n, df); break;
    }
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, df, (size_t)n * 4, cudaMemcpyDeviceToHost);
  cudaFree(dw);
  cudaFree(df);
  if (e != cudaSuccess) return set_err(s, POLARIS_ECUDA, "debug_unpack: %s", cudaGetErrorString(e));
  return POLARIS_OK;
}

extern "C" int spectrometer_debug_unpack_staged(polaris_spec* s, const void* packed_a, const void* packed_b, int64_t n,
                                                int layout, float* out_a, float* out_b) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (!packed_a || !out_a || (packed_b && !out_b)) return set_err(s, POLARIS_EINVAL, "null pointer");
  if (n <= 0 || n % s->N) return set_err(s, POLARIS_EINVAL, "n must be a positive multiple of n_fft");
  if (layout != 0 && layout != 1) return set_err(s, POLARIS_EINVAL, "layout must be 0 (interleaved) or 1 (dense)");
  if (!phase1_staged(s->logn, s->bits))
    return set_err(s, POLARIS_EINVAL, "phase 1 does not stage its input at this size and width");
  DeviceGuard dg(s->device);
  const size_t nw = (size_t)(n / s->spw);
  const int nif = packed_b ? 2 : 1;
  uint32_t* dw = nullptr;
  float* df = nullptr;
  if (cudaMalloc((void**)&dw, nw * 4 * nif) != cudaSuccess || cudaMalloc((void**)&df, (size_t)n * 4 * nif) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(dw);
    cudaFree(df);
    return set_err(s, POLARIS_ENOMEM, "debug_unpack_staged allocation failed");
  }
  cudaError_t e = cudaMemcpy(dw, packed_a, nw * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && packed_b) e = cudaMemcpy(dw + nw, packed_b, nw * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = launch_unpack_staged(s->logn, s->bits, dw, packed_b ? dw + nw : nullptr, (long long)(n / s->N), layout, df,
                             packed_b ? df + n : nullptr, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out_a, df, (size_t)n * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && packed_b) e = cudaMemcpy(out_b, df + n, (size_t)n * 4, cudaMemcpyDeviceToHost);
  cudaFree(dw);
  cudaFree(df);
  if (e != cudaSuccess) return set_err(s, POLARIS_ECUDA, "debug_unpack_staged: %s", cudaGetErrorString(e));
  return POLARIS_OK;
}

extern "C" int64_t spectrometer_kernel_launches(const polaris_spec* s) { return s ? s->launches : -1; }

extern "C" int spectrometer_set_launch_caps(polaris_spec* s, int phase1_ctas_per_sm, int phase2_ctas_per_sm) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (phase1_ctas_per_sm < 0 || phase2_ctas_per_sm < 0)
    return set_err(s, POLARIS_EINVAL, "CTA caps must be >= 0 (0: as many as fit)");
  s->cap1 = phase1_ctas_per_sm;
  s->cap2 = phase2_ctas_per_sm;
  return POLARIS_OK;
}

extern "C" int spectrometer_get_launch(const polaris_spec* s, int* max_batch_segments, int* phase1_ctas_per_sm,
                                       int* phase2_ctas_per_sm) {
  if (!s) return POLARIS_EINVAL;
  if (max_batch_segments) *max_batch_segments = s->max_batch;
  if (phase1_ctas_per_sm) *phase1_ctas_per_sm = s->cap1;
  if (phase2_ctas_per_sm) *phase2_ctas_per_sm = s->cap2;
  return POLARIS_OK;
}


extern "C" int spectrometer_set_profiling(polaris_spec* s, int on) {
  if (!s) return POLARIS_EINVAL;
  DeviceGuard dg(s->device);
  s->profiling = on != 0;
  if (!s->profiling) drop_prof(s);
  return POLARIS_OK;
}

extern "C" int spectrometer_kernel_times(polaris_spec* s, double* ms, int64_t* launches, int n) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (!ms || !launches || n < 3) return set_err(s, POLARIS_EINVAL, "need arrays of at least 3 entries");
  DeviceGuard dg(s->device);
  for (int k = 0; k < n; ++k) {
    ms[k] = 0.0;
    launches[k] = 0;
  }
  for (auto& r : s->prof) {
    CUDA_OR_FAIL(s, cudaEventSynchronize(r.b));
    float t = 0.f;
    CUDA_OR_FAIL(s, cudaEventElapsedTime(&t, r.a, r.b));
    if (r.kind < n) {
      ms[r.kind] += t;
      launches[r.kind] += 1;
    }
  }
  drop_prof(s);
  return POLARIS_OK;
}

extern "C" int spectrometer_code_histogram(polaris_spec* s, uint64_t* counts, int reset) {
  int rc = check_usable(s);
  if (rc) return rc;
  if (!counts) return set_err(s, POLARIS_EINVAL, "null counts");
  if (!s->code_stats) return set_err(s, POLARIS_ESTATE, "spectrometer created with code_stats = 0");
  DeviceGuard dg(s->device);
  const size_t bytes = (size_t)s->n_if * ((size_t)1 << s->bits) * 8;
  CUDA_OR_FAIL(s, cudaDeviceSynchronize());  // the counts of everything queued so far
  rc = check_device_status(s);
  if (rc) return rc;
  CUDA_OR_FAIL(s, cudaMemcpy(counts, s->d_hist, bytes, cudaMemcpyDeviceToHost));
  if (reset) CUDA_OR_FAIL(s, cudaMemset(s->d_hist, 0, bytes));
  return POLARIS_OK;
}

// =======================================================================================
// Allocation-free one-shot variant.
//
// Some callers cannot allocate device memory at the point where they need a spectrum:
// real-time loops in which cudaMalloc/cudaFree would synchronise the device and miss a
// sampler deadline, and host frameworks that own all device memory through their own
// pool and forbid other allocators.  For them spectrometer_run_noalloc computes one
// integration without a handle: its scratch slab, accumulators, twiddle table and
// window taps live in the file-scope array below, which every GPU that loads this
// library holds until the process exits.  Every argument is checked before the first
// operation is queued.  The call never synchronises, so a bounded device-side wait that
// ran out is not reported as a status: it shows as NaN in every output.
// =======================================================================================
#define POLARIS_NOALLOC_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[POLARIS_NOALLOC_BYTES];

static const int kNoallocMaxDevices = 64;
static void* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};
static std::mutex g_noalloc_mu;

// twiddles W_N^{b u} (b < N2, u <= N1/2) in FP64, rounded once to f32, unit-major ([u][b])
__global__ void k_noalloc_twiddles(float2* tw, int N2, int UPS, long long N) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)N2 * (UPS + 1);
  if (i >= total) return;
  const long long u = i / N2, b = i % N2;
  const long long e = (b * u) % N;
  double s, c;
  sincospi(-2.0 * (double)e / (double)N, &s, &c);
  tw[i] = make_float2((float)c, (float)s);
}

// periodic Hann taps 0.5 - 0.5 cos(2 pi n / N)
__global__ void k_noalloc_hann(float* taps, long long N) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  taps[n] = (float)(0.5 - 0.5 * cospi(2.0 * (double)n / (double)N));
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

extern "C" int spectrometer_run_noalloc(const polaris_config* cfg, const void* const* d_packed,
                                        int64_t n_samples_per_if, const polaris_stokes_params* prm, float* d_autos,
                                        float* d_cross, float* d_stokes, int64_t* n_segments_out,
                                        void* cuda_stream) {
  NvtxRange nvtx("polaris.run_noalloc");
  if (!cfg || !d_packed) return set_err(nullptr, POLARIS_EINVAL, "null config or input");
  const polaris_config& c = *cfg;
  if (c.n_if < 1 || c.n_if > kMaxIF) return set_err(nullptr, POLARIS_EINVAL, "n_if must be in [1, %d]", kMaxIF);
  if (!(c.bits == 1 || c.bits == 2 || c.bits == 4 || c.bits == 8))
    return set_err(nullptr, POLARIS_EINVAL, "bits must be 1, 2, 4 or 8");
  const int64_t N = c.n_fft;
  if (N < 16 || N > (1 << 20) || (N & (N - 1)))
    return set_err(nullptr, POLARIS_EINVAL, "n_fft must be a power of two in [16, 1048576]");
  const int64_t spw = 32 / c.bits;
  const int64_t hop = c.hop == 0 ? N : c.hop;
  if (N < spw || hop < 1 || hop > N || hop % spw)
    return set_err(nullptr, POLARIS_EINVAL, "bad n_fft/hop for %d-bit samples", c.bits);
  if (c.window < POLARIS_WIN_RECT || c.window > POLARIS_WIN_CUSTOM || (c.window == POLARIS_WIN_CUSTOM && !c.taps))
    return set_err(nullptr, POLARIS_EINVAL, "bad window");
  if (n_samples_per_if < N || n_samples_per_if % spw)
    return set_err(nullptr, POLARIS_EINVAL, "need at least one whole segment and a multiple of 32/bits samples");
  for (int i = 0; i < c.n_if; ++i)
    if (!d_packed[i] || (reinterpret_cast<uintptr_t>(d_packed[i]) & 3))
      return set_err(nullptr, POLARIS_EINVAL, "input %d is NULL or not 4-byte aligned", i);
  // pairs (same rules as spectrometer_create)
  int pairs[2 * kMaxIF];
  int n_pair = 0;
  if (c.pairs) {
    if (c.n_pair < 0 || 2 * c.n_pair > c.n_if) return set_err(nullptr, POLARIS_EINVAL, "bad n_pair");
    n_pair = c.n_pair;
    for (int i = 0; i < 2 * n_pair; ++i) pairs[i] = c.pairs[i];
  } else if (c.n_if % 2 == 0) {
    n_pair = c.n_if / 2;
    for (int i = 0; i < n_pair; ++i) {
      pairs[2 * i] = i;
      pairs[2 * i + 1] = i + n_pair;
    }
  }
  int used[kMaxIF] = {0};
  for (int i = 0; i < 2 * n_pair; ++i) {
    if (pairs[i] < 0 || pairs[i] >= c.n_if || used[pairs[i]]++)
      return set_err(nullptr, POLARIS_EINVAL, "bad or repeated pair index");
  }
  int fa[kMaxIF], fb[kMaxIF], fcorr[kMaxIF];
  int nf = 0, pending = -1;
  for (int p = 0; p < n_pair; ++p, ++nf) {
    fa[nf] = pairs[2 * p];
    fb[nf] = pairs[2 * p + 1];
    fcorr[nf] = p;
  }
  for (int i = 0; i < c.n_if; ++i) {
    if (used[i]) continue;
    if (pending < 0) pending = i;
    else {
      fa[nf] = pending;
      fb[nf] = i;
      fcorr[nf++] = -1;
      pending = -1;
    }
  }
  if (pending >= 0) {
    fa[nf] = pending;
    fb[nf] = -1;
    fcorr[nf++] = -1;
  }
  for (int f = nf; f < kMaxIF; ++f) fa[f] = fb[f] = fcorr[f] = -1;
  // Stokes parameters (checked here, before anything is queued: a rejected call leaves the
  // static array and the outputs untouched)
  const int feed = prm ? prm->feed : POLARIS_FEED_LINEAR;
  if (feed != POLARIS_FEED_LINEAR && feed != POLARIS_FEED_CIRCULAR) return set_err(nullptr, POLARIS_EINVAL, "bad feed");
  const double psi = prm ? prm->psi_m : 0.0;
  const float c2 = (float)std::cos(2.0 * psi), s2 = (float)std::sin(2.0 * psi);
  float inv_ga2[kMaxIF], inv_gb2[kMaxIF], ig_re[kMaxIF], ig_im[kMaxIF];
  for (int p = 0; p < n_pair; ++p) {
    double gar = 1, gai = 0, gbr = 1, gbi = 0;
    if (prm && prm->gains) {
      gar = prm->gains[4 * p + 0];
      gai = prm->gains[4 * p + 1];
      gbr = prm->gains[4 * p + 2];
      gbi = prm->gains[4 * p + 3];
    }
    const double gaa = gar * gar + gai * gai, gbb = gbr * gbr + gbi * gbi;
    if (gaa == 0.0 || gbb == 0.0) return set_err(nullptr, POLARIS_EINVAL, "zero gain for pair %d", p);
    const double gr = gar * gbr + gai * gbi, gi = gai * gbr - gar * gbi, g2 = gr * gr + gi * gi;
    inv_ga2[p] = (float)(1.0 / gaa);
    inv_gb2[p] = (float)(1.0 / gbb);
    ig_re[p] = (float)(gr / g2);
    ig_im[p] = (float)(-gi / g2);
  }
  int logn = 0;
  while ((1LL << logn) < N) ++logn;
  const int N2 = host_plan_n2(logn), N1 = (int)(N / N2), UPS = N1 / 2, native = UPS * N2 + 1;
  // carve the static array: accumulators | twiddles | taps | slab
  const size_t acc_bytes = align256((size_t)nf * native * 4 * (c.accum_fp64 ? 8 : 4));
  const size_t tw_bytes = align256((size_t)N2 * (UPS + 1) * sizeof(float2));
  const size_t taps_bytes = c.window == POLARIS_WIN_RECT ? 0 : align256((size_t)N * 4);
  const size_t err_bytes = 256;  // the phase kernels' status word
  const size_t per_seg = (size_t)nf * N * sizeof(float2);
  const size_t fixed = acc_bytes + tw_bytes + taps_bytes + err_bytes;
  if (fixed + per_seg > POLARIS_NOALLOC_BYTES)
    return set_err(nullptr, POLARIS_EINVAL,
                   "configuration needs %zu bytes of scratch for one segment, above the %u-byte static limit",
                   fixed + per_seg, (unsigned)POLARIS_NOALLOC_BYTES);
  const int batch = (int)((POLARIS_NOALLOC_BYTES - fixed) / per_seg);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device < 0 || c.device >= ndev || c.device >= kNoallocMaxDevices) {
    cudaGetLastError();
    return set_err(nullptr, POLARIS_EINVAL, "device ordinal out of range");
  }
  DeviceGuard dg(c.device);
  // set-up, once per device: the device address of the static array
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[c.device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return set_err(nullptr, POLARIS_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_noalloc_ptr[c.device] = p;
    }
    base = static_cast<unsigned char*>(g_noalloc_ptr[c.device]);
  }
  void* acc = base;
  float2* tw = reinterpret_cast<float2*>(base + acc_bytes);
  float* taps = c.window == POLARIS_WIN_RECT ? nullptr : reinterpret_cast<float*>(base + acc_bytes + tw_bytes);
  int* d_err = reinterpret_cast<int*>(base + acc_bytes + tw_bytes + taps_bytes);
  float2* slab = reinterpret_cast<float2*>(base + fixed);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  int num_sms = 0;
  cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, c.device);
  cudaError_t e = cudaMemsetAsync(acc, 0, acc_bytes, st);  // accumulators start at zero
  if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    const long long ntw = (long long)N2 * (UPS + 1);
    k_noalloc_twiddles<<<(unsigned)((ntw + 255) / 256), 256, 0, st>>>(tw, N2, UPS, N);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && c.window == POLARIS_WIN_HANN) {
    k_noalloc_hann<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(taps, N);
    e = cudaGetLastError();
  } else if (e == cudaSuccess && c.window == POLARIS_WIN_CUSTOM) {
    e = cudaMemcpyAsync(taps, c.taps, (size_t)N * 4, cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return set_err(nullptr, POLARIS_ECUDA, "no-alloc set-up: %s", cudaGetErrorString(e));
  const int64_t nseg = (n_samples_per_if - N) / hop + 1;
  BatchArgs a;
  memset(&a, 0, sizeof a);
  for (int i = 0; i < c.n_if; ++i) {
    a.in.src0[i] = static_cast<const uint32_t*>(d_packed[i]);
    a.in.src1[i] = static_cast<const uint32_t*>(d_packed[i]);
  }
  a.in.hop_w = hop / spw;
  a.in.n0 = 0;
  a.in.in_words0 = a.in.in_words1 = n_samples_per_if / spw;
  for (int f = 0; f < kMaxIF; ++f) {
    a.fa[f] = fa[f];
    a.fb[f] = fb[f];
  }
  a.n_fpair = nf;
  a.taps = taps;
  a.scratch = slab;
  a.err = d_err;
  a.wait_limit = g_wait_limit;
  a.tw = tw;
  a.acc = acc;
  a.acc_copies = 1;
  a.slab_elems = (long long)batch * nf * N;
  a.acc_slots = (long long)nf * native;
  a.fp64 = c.accum_fp64 ? 1 : 0;
  a.bits = c.bits;
  a.num_sms = num_sms;
  for (int64_t s0 = 0; s0 < nseg; s0 += batch) {
    a.seg0 = (int)s0;
    a.nseg = (int)(nseg - s0 < batch ? nseg - s0 : batch);
    for (int ph = 0; ph < 2 && e == cudaSuccess; ++ph) e = kPhases[logn][ph](a, st, st != nullptr);
    if (e != cudaSuccess) return set_err(nullptr, POLARIS_ECUDA, "no-alloc FFT-correlator: %s", cudaGetErrorString(e));
  }
  // readout (same kernel as spectrometer_integrate_device)
  ReadoutArgs r;
  memset(&r, 0, sizeof r);
  r.acc = acc;
  r.copies = 1;
  r.copy_stride = (long long)nf * native;
  r.err = d_err;
  r.acc_slots = (long long)nf * native;
  r.fp64 = a.fp64;
  r.N1 = N1;
  r.N2 = N2;
  r.UPS = UPS;
  r.nbin = (int)(N / 2 + 1);
  r.native = native;
  for (int f = 0; f < kMaxIF; ++f) {
    r.fa[f] = fa[f];
    r.fb[f] = fb[f];
    r.fcorr[f] = fcorr[f];
  }
  r.feed = feed;
  r.c2 = c2;
  r.s2 = s2;
  for (int p = 0; p < n_pair; ++p) {
    r.inv_ga2[p] = inv_ga2[p];
    r.inv_gb2[p] = inv_gb2[p];
    r.ig_re[p] = ig_re[p];
    r.ig_im[p] = ig_im[p];
  }
  r.autos = d_autos;
  r.cross = n_pair ? d_cross : nullptr;
  r.stokes = n_pair ? d_stokes : nullptr;
  e = launch_readout(r, nf, st, st != nullptr);
  if (e != cudaSuccess) return set_err(nullptr, POLARIS_ECUDA, "no-alloc readout: %s", cudaGetErrorString(e));
  if (n_segments_out) *n_segments_out = nseg;
  return POLARIS_OK;
}
