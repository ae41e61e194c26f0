/*
 * polaris.h — C ABI of the GB300-native PolariS spectrometer hot path.
 *
 * The operation (arXiv:1412.1256, Sec. 2 and the Fig. 2 caption): the GPU takes
 * the quantised voltage samples of each IF stream, translates the integer codes
 * to floats, cuts the stream into segments, transforms each segment with an FFT,
 * forms the power spectra <XX*>, <YY*> and the cross power spectrum <XY*>
 * (Fig. 1 caption; Table 1: 4 real autocorrelations, 2 complex cross
 * correlations) and integrates them; the full-Stokes spectra I, Q, U, V follow
 * from Eq. (2) (Sec. 2.1).  Every step runs in hand-written CUDA kernels for
 * sm_103a; this header has no CUDA or PyTorch types.
 *
 * Conventions (readings where the paper is silent):
 *   - Input: one planar stream of little-endian uint32 words per IF; sample j of
 *     a word sits in bits [j*bits, (j+1)*bits).  bits < 8: code c has level
 *     2c - (2^bits - 1) (2-bit: -3, -1, +1, +3); bits = 8: two's-complement int8.
 *   - Segment s covers stream samples [s*hop, s*hop + n_fft); only whole segments
 *     are transformed; the remainder is carried to the next feed.
 *   - Transform: unnormalised forward DFT, X_k = sum_n w[n] y[n] e^{-2 pi i n k/N},
 *     bins k = 0 .. N/2 (N/2 + 1 bins; DC and Nyquist included).
 *   - Integration: sums over segments (not means); autos A_i[k] = sum |X_i,k|^2,
 *     cross C_p[k] = sum X_a,k conj(X_b,k) for pair p = (a, b).
 *   - Stokes, linear feeds: Eq. (2) with x = XX/|Ga|^2, c = XY/(Ga conj(Gb)),
 *     y = YY/|Gb|^2, i.e. I = (x+y)/2, Q = [cos2psi (x-y) - sin2psi 2Re c]/2,
 *     U = [sin2psi (x-y) + cos2psi 2Re c]/2, V = Im c.
 *     Circular feeds (R, L): I = (RR+LL)/2, V = (RR-LL)/2, Q + iU = e^{2i psi} R conj(L).
 *
 * Threading: a handle is not thread-safe.  Errors never cross the ABI as
 * exceptions: every call returns a status; spectrometer_last_error() gives text.
 * A CUDA error inside a call is sticky: the handle answers POLARIS_ESTATE to
 * every later call except destroy and last_error.
 */
#ifndef POLARIS_H
#define POLARIS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
enum {
  POLARIS_OK = 0,
  POLARIS_EINVAL = -1,   /* bad argument; the call had no effect            */
  POLARIS_ENOMEM = -2,   /* device or pinned-host allocation failed          */
  POLARIS_ECUDA = -3,    /* a CUDA call failed; the handle is now unusable   */
  POLARIS_ESTATE = -4,   /* wrong state (e.g. integrate with zero segments,
                            or a handle after a CUDA error)                  */
  POLARIS_ETIMEOUT = -5, /* a bounded device-side wait ran out (see below)   */
  POLARIS_EBOUNDS = -6   /* bounds-checked build only (compiled with
                            -DPOLARIS_CHECK): a kernel found an index outside
                            its buffer, skipped that access and recorded it;
                            outputs are NaN and the handle is unusable       */
};

/* window kinds (Sec. 3.1: rectangular online; Sec. 5: others possible) */
enum { POLARIS_WIN_RECT = 0, POLARIS_WIN_HANN = 1, POLARIS_WIN_CUSTOM = 2 };

/* feed types for Stokes */
enum { POLARIS_FEED_LINEAR = 0, POLARIS_FEED_CIRCULAR = 1 };

typedef struct polaris_spec polaris_spec; /* opaque, library-owned */

/* Spectrometer configuration (Table 1: number of IFs, quantisation, channels).
 *   n_if        1..8 IF streams.
 *   bits        1, 2, 4 or 8 bits per sample.
 *   n_fft       segment length N, a power of two in [16, 1048576]; N/2+1 bins.
 *   hop         segment spacing in samples, 0 < hop <= n_fft, a multiple of
 *               32/bits (0 means hop = n_fft; hop = n_fft/2 is the 50% overlap
 *               of Sec. 3.1).
 *   window      POLARIS_WIN_*; taps: n_fft float taps for POLARIS_WIN_CUSTOM
 *               (copied at create; ignored otherwise).  Hann is periodic:
 *               0.5 - 0.5 cos(2 pi n / N).
 *   n_pair      number of (X, Y) correlation pairs; pairs: 2*n_pair IF indices
 *               (a, b), each IF in at most one pair.  pairs == NULL selects the
 *               default: IF i with IF i + n_if/2 for even n_if (Table 1 order
 *               X0, X1, Y0, Y1 gives (X0, Y0), (X1, Y1)); none for odd n_if.
 *   accum_fp64  1: integration accumulators in FP64 (per-launch partial sums in
 *               FP32); 0: FP32.
 *   device      CUDA device ordinal.
 *   max_batch_segments  segments processed per kernel pass (bounds the device
 *               scratch: 2 * max_batch_segments * n_fft * 8 bytes per pair);
 *               0 selects the default (passes of at least 64 segments).
 *   code_stats  1: also count, per IF, how often each b-bit code occurs in the
 *               segments that feed() integrates (the bit distribution used for
 *               total-power measurement, Sec. 2 and Sec. 3.2.2); read with
 *               spectrometer_code_histogram.  0: no counting (no extra work). */
typedef struct {
  int n_if;
  int bits;
  int64_t n_fft;
  int64_t hop;
  int window;
  const float* taps;
  int n_pair;
  const int* pairs;
  int accum_fp64;
  int device;
  int max_batch_segments;
  int code_stats;
} polaris_config;

/* Stokes parameters for integrate (Eq. 2): feed type, parallactic angle psi_m
 * (radians, used as written in Eq. 2), and per-pair complex voltage gains
 * gains[4*p + 0..3] = (Ga re, Ga im, Gb re, Gb im); gains == NULL means G = 1. */
typedef struct {
  int feed;
  double psi_m;
  const float* gains;
} polaris_stokes_params;

/* Create a spectrometer.  Allocates all device state (accumulators, twiddle and
 * window tables, scratch).  Returns POLARIS_EINVAL for invalid config (out is
 * untouched), POLARIS_ENOMEM / POLARIS_ECUDA on allocation / CUDA failure.
 * A handle runs its integrations one after another in stream order.  Independent
 * integrations (consecutive seconds of a stream, other IF sets) kept in flight on
 * separate handles and CUDA streams overlap on the GPU: one integration's transform
 * runs beside another's correlation (three handles: about 1.3x one handle's rate at
 * N = 2^17). */
int spectrometer_create(const polaris_config* cfg, polaris_spec** out);

/* Feed n_samples_per_if new samples of every IF stream and accumulate all whole
 * segments they complete into the current integration.  This is the GPU side of the
 * paper's data path (Sec. 2, Fig. 2 caption): the sampler's quantised IF streams
 * (Table 1: four IFs, 4- or 8-bit samples at 8 or 16 Msps) are translated to floats, cut
 * into segments, transformed, multiplied into power and cross-power spectra, and added to
 * the running integration (function (4) of Sec. 2: integration over the 1-s time
 * resolution of Table 1, closed by spectrometer_integrate).
 *   packed[i]   pointer to IF i's words (n_samples_per_if * bits / 32 words), 4-byte
 *               aligned, in the memory that on_device names:
 *   on_device   POLARIS_INPUT_HOST (0): host memory, read when the call returns;
 *               POLARIS_INPUT_DEVICE (1): device memory, read in stream order (keep it
 *               alive until the stream reaches this point);
 *               POLARIS_INPUT_HOST_ASYNC (2): host memory (pinned, for the copy to be
 *               asynchronous), copied in stream order: the call returns at once and the
 *               buffers must stay unchanged until the stream reaches this point.
 *   n_samples_per_if  >= 0, a multiple of 32/bits.
 *   cuda_stream cudaStream_t to order the work on (NULL = legacy default stream); feeds
 *               and integrations of one handle go on one stream.
 * IF streams that are rows of one host array (a constant stride) go over in one copy.
 * Work is asynchronous with respect to the host except for the wait of mode 0. */
enum { POLARIS_INPUT_HOST = 0, POLARIS_INPUT_DEVICE = 1, POLARIS_INPUT_HOST_ASYNC = 2 };
int spectrometer_feed(polaris_spec* s, const void* const* packed, int64_t n_samples_per_if, int on_device,
                      void* cuda_stream);

/* Close the current integration: form autos, crosses and Stokes from the
 * accumulated sums, copy them to the HOST buffers given (NULL skips an output),
 * and reset the accumulators (carried samples persist).  Synchronous.
 *   autos   [n_if][N/2+1] float
 *   cross   [n_pair][N/2+1][2] float (re, im) = sum X_a conj(X_b)
 *   stokes  [n_pair][4][N/2+1] float (I, Q, U, V)
 *   n_segments_out  segments per IF in this integration (may be NULL)
 * params == NULL means linear feeds, psi_m = 0, unit gains.
 * Returns POLARIS_ESTATE when no segment has been accumulated. */
int spectrometer_integrate(polaris_spec* s, const polaris_stokes_params* params, float* autos, float* cross,
                           float* stokes, int64_t* n_segments_out);

/* As spectrometer_integrate, but asynchronous: the readout and the copies into the
 * caller's HOST buffers (pinned memory, for the copies to be asynchronous) are queued on
 * cuda_stream and the call returns without synchronising.  The outputs are valid once the
 * stream has passed this point (cudaStreamSynchronize, or an event recorded after the
 * call).  The results are staged in the handle's device output buffers, so successive
 * calls on one handle must be ordered (one stream).  A device-side wait that ran out
 * shows as NaN outputs; spectrometer_integrate (synchronous) reports POLARIS_ETIMEOUT. */
int spectrometer_integrate_async(polaris_spec* s, const polaris_stokes_params* params, float* autos, float* cross,
                                 float* stokes, int64_t* n_segments_out, void* cuda_stream);

/* As spectrometer_integrate, but the outputs are DEVICE buffers of the same
 * layouts, written in stream order on cuda_stream (no host synchronisation). */
int spectrometer_integrate_device(polaris_spec* s, const polaris_stokes_params* params, float* d_autos, float* d_cross,
                                  float* d_stokes, int64_t* n_segments_out, void* cuda_stream);

/* Launch choices of a handle (not in the paper: how the transform is cut into kernel passes
 * on this GPU).  spectrometer_get_launch reports the segments per kernel pass and the caps
 * on CTAs per SM of the two FFT kernels (0: as many as fit); a handle created with
 * max_batch_segments = 0 takes them from the library's tuned table (written by
 * paper_1412_1256_gb300/tune.py from timings per N and width) or, for sizes without an
 * entry, from the built-in rule.  spectrometer_set_launch_caps changes the two caps for
 * later feeds (results do not depend on them).  A caller that keeps several integrations in
 * flight on separate handles and streams gains by capping phase 1 at one CTA per SM: every SM
 * then keeps room for another integration's phase 2 (about 3% at N = 2^17 with three
 * handles, while one handle alone is about 6% slower with that cap).  Either output pointer
 * may be NULL; POLARIS_EINVAL for a NULL handle or negative caps. */
int spectrometer_get_launch(const polaris_spec* s, int* max_batch_segments, int* phase1_ctas_per_sm,
                            int* phase2_ctas_per_sm);
int spectrometer_set_launch_caps(polaris_spec* s, int phase1_ctas_per_sm, int phase2_ctas_per_sm);

/* Number of output bins (N/2 + 1), IFs and pairs of a handle. */
int64_t spectrometer_n_bins(const polaris_spec* s);
int spectrometer_n_pairs(const polaris_spec* s);

/* The data-translation step alone (Fig. 2 caption: integer codes to floats),
 * for bit-exact checks: decode n samples of one packed stream (host words) into
 * host floats `out`, on the GPU.  n must be a multiple of 32/bits. */
int spectrometer_debug_unpack(polaris_spec* s, const void* packed, int64_t n, float* out);

/* The data-translation step as the FFT kernel runs it from N = 2^13 up (Fig. 2 caption:
 * integer codes to floats; Sec. 2: two IF streams enter one transform): that kernel stages
 * each tile's packed words in shared memory and decodes every column at a per-column
 * rotation, both IFs of a pair in one packed subtraction.  This call stages and decodes
 * through that same device code, for bit-exact checks of the levels the transform sees.
 *   packed_a, packed_b  host words of IF a and IF b of one FFT pair (packed_b NULL: a pair
 *               without an IF b, decoded by the single-IF variant), n samples each;
 *   n           a positive multiple of n_fft (whole segments, hop = n_fft);
 *   layout      0: the interleaved stage of cp.async staging; 1: the dense [IF][row][word]
 *               stage of TMA staging;
 *   out_a, out_b  host floats, n each (out_b unused when packed_b is NULL).
 * POLARIS_EINVAL when the FFT kernel does not stage at this handle's size and width (below
 * 2^13, and 1-bit samples at 2^19 and 2^20: there it decodes as spectrometer_debug_unpack). */
int spectrometer_debug_unpack_staged(polaris_spec* s, const void* packed_a, const void* packed_b, int64_t n,
                                     int layout, float* out_a, float* out_b);

/* Free all resources.  NULL is ignored. */
void spectrometer_destroy(polaris_spec* s);

/* Text of the last error on this handle ("" if none); for s == NULL, the last
 * error of a failed spectrometer_create in this thread. */
const char* spectrometer_last_error(const polaris_spec* s);

/* Kernel accounting (for benchmarks).  spectrometer_kernel_launches: kernels this
 * handle has launched so far, all kinds.  spectrometer_set_profiling(s, 1) brackets
 * every later launch with CUDA events on its stream; spectrometer_kernel_times then
 * waits for those events and returns, per kind, the summed device time in ms and the
 * launch count since profiling began or since the previous query (kinds: 0 = phase 1,
 * decode/window/row DFT; 1 = phase 2, column DFT/correlate/accumulate; 2 = readout and
 * Stokes; 3 = code histogram).  n is the length of both arrays and must be >= 3; kinds
 * >= n are not reported. */
int64_t spectrometer_kernel_launches(const polaris_spec* s);
int spectrometer_set_profiling(polaris_spec* s, int on);
int spectrometer_kernel_times(polaris_spec* s, double* ms, int64_t* launches, int n);

/* One integration without any device allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they need a
 * spectrum -- real-time loops in which cudaMalloc/cudaFree would synchronise the device
 * and miss the sampler's deadline, and host frameworks that own all device memory
 * through their own pool and allow no other allocator.  It computes the same autos,
 * crosses and Stokes as create + feed + integrate_device for the whole segments of one
 * input block (samples after the last whole segment are ignored; nothing is carried),
 * but it keeps no handle: its scratch slab, accumulators, twiddles and window taps live
 * in one static device array of 32 MiB (POLARIS_NOALLOC_BYTES), which every GPU that
 * loads this library holds until the process exits.
 *   cfg         as for spectrometer_create (the max_batch_segments and code_stats fields
 *               are ignored).  Custom taps are host memory, copied in stream order:
 *               pageable memory has been read when the call returns, pinned memory must
 *               stay unchanged until the stream has passed this call.
 *   d_packed    n_if DEVICE pointers to the packed words; n_samples_per_if >= n_fft
 *               and a multiple of 32/bits.
 *   params      as for spectrometer_integrate (NULL: linear feeds, psi = 0, unit gains).
 *   d_autos, d_cross, d_stokes  DEVICE outputs in the layouts of
 *               spectrometer_integrate (NULL skips one).
 * Work is queued on cuda_stream (NULL = legacy default stream); nothing is allocated
 * and nothing synchronises the host.  Every argument is checked before anything is
 * queued: a call that returns POLARIS_EINVAL has queued no work and changed neither the
 * array nor the outputs.  A configuration whose accumulators, tables and one segment of
 * slab exceed 32 MiB is rejected that way, with a message.  The first call on a device
 * looks up the array's device address (once per device, with that device made current).
 * Every call reuses the same array, which keeps the previous call's contents (each call
 * zeroes the accumulators it needs): calls on the same device whose GPU work overlaps
 * (on different streams, say) race on the array and must be ordered by the caller.
 * Because the call does not synchronise, a bounded device-side wait that ran out (see
 * polaris_set_wait_limit) is not reported as a status: every output is then NaN. */
int spectrometer_run_noalloc(const polaris_config* cfg, const void* const* d_packed, int64_t n_samples_per_if,
                             const polaris_stokes_params* params, float* d_autos, float* d_cross, float* d_stokes,
                             int64_t* n_segments_out, void* cuda_stream);

/* Code histogram: the bit distribution of the digitised signal, from which PolariS
 * derives each IF's total power (Sec. 2; linearity of that measurement, Sec. 3.2.2).  counts: host array of n_if * 2^bits uint64, filled
 * with counts[i * 2^bits + c] = number of samples of IF i with code c, summed over
 * every segment integrated since the spectrometer was created or last reset (a
 * sample in two overlapping segments counts twice).  reset != 0 zeroes the counts
 * after reading them.  Synchronises with the work queued so far.  Returns
 * POLARIS_ESTATE if the spectrometer was created with code_stats = 0. */
int spectrometer_code_histogram(polaris_spec* s, uint64_t* counts, int reset);

/* Total power of one IF from its code histogram (counts: 2^bits entries; host-only
 * arithmetic in FP64).  Our reading of the bit-distribution method (the cited
 * scheme is not reproduced in the paper):
 *   moment2  = sum_c level(c)^2 counts[c] / sum_c counts[c], with the decoded levels
 *              (2c - (2^b - 1) for b < 8, int8 for b = 8): the power of the digitised
 *              signal in level units (a measure of input power for 4 and 8 bits);
 *   sigma_over_threshold (2-bit only) = 1 / (sqrt(2) erfcinv(p_outer)), p_outer the
 *              fraction of the two outer codes: the rms of a zero-mean Gaussian input
 *              in units of the sampler threshold; NaN for other widths or when
 *              p_outer is 0 or 1.
 * Either output pointer may be NULL.  Returns POLARIS_EINVAL for a bad width, NULL
 * counts or an empty histogram. */
int polaris_power_from_histogram(int bits, const uint64_t* counts, double* moment2, double* sigma_over_threshold);

/* ---- Differentiable leakage calibration ----
 * A model of our own (the paper calibrates the gains offline, Sec. 2.1, and does not
 * model polarisation leakage) with a hand-written adjoint, for fitting a window, the two
 * feeds' complex gains and per-channel leakage to target Stokes spectra.  Two IFs R and L
 * (circular feeds), segments of n_fft samples at hop n_fft, window w (n_fft taps):
 *   X_s[k] = sum_n w[n] x_s[n] e^{-2 pi i n k / N},  Y_s[k] likewise, k = 0..N/2
 *   Xt = gR (X + DR[k] Y),   Yt = gL (Y + DL[k] X)
 *   RR = sum_s |Xt|^2, LL = sum_s |Yt|^2, RL = sum_s Xt conj(Yt)
 *   I = (RR + LL)/2, Q = Re RL, U = Im RL, V = (RR - LL)/2     (circular feeds, psi = 0)
 *   loss = sum_k sum_{S = I, Q, U, V} (S[k] - T_S[k])^2
 * polaris_adj_create: n_fft a power of two in [32, 16384], bits 1/2/4/8; allocates a
 * handle with its twiddles and accumulators on `device`.
 * polaris_adj_run: all pointers are DEVICE pointers, fp32 unless stated, queued on
 * cuda_stream (NULL = legacy stream), nothing synchronises the host:
 *   packed[2]    the two IFs' packed codes (layout as spectrometer_feed), n_samples each,
 *                a positive multiple of n_fft
 *   window       n_fft taps;  gains  (gR re, gR im, gL re, gL im)
 *   leak         DR then DL, each n_fft/2+1 (re, im) pairs
 *   target       I, Q, U, V, each n_fft/2+1 (NULL: no loss, no gradients)
 *   stokes       out: I, Q, U, V of the model, each n_fft/2+1 (NULL skips)
 *   loss         out: one fp64 value (NULL skips)
 *   grad_window, grad_gains, grad_leak   out: d loss / d (each real parameter), in the
 *                layouts of the inputs; all three or none.  The adjoint transforms every
 *                segment again instead of storing the spectra.
 * Speed: for n_fft in [512, 16384] with packed[0], packed[1] and window 16-byte aligned
 * (as every cudaMalloc or torch allocation is), the segment passes run kernels specialised
 * per n_fft; other calls run kernels for any n_fft, with results equal within rounding.
 * A handle's work buffers serve one run at a time: runs on one handle whose GPU work
 * could overlap (on different streams) must be ordered by the caller.
 * Errors: POLARIS_EINVAL for bad arguments, POLARIS_ECUDA for a CUDA error (text from
 * polaris_adj_last_error; NULL handle: the last failed create in this thread). */
typedef struct polaris_adj polaris_adj;
int polaris_adj_create(int64_t n_fft, int bits, int device, polaris_adj** out);
int polaris_adj_run(polaris_adj* h, const void* const* packed, int64_t n_samples, const float* window,
                    const float* gains, const float* leak, const float* target, float* stokes, double* loss,
                    float* grad_window, float* grad_gains, float* grad_leak, void* cuda_stream);
void polaris_adj_destroy(polaris_adj* h);
const char* polaris_adj_last_error(const polaris_adj* h);

/* ---- Tensor-core DFT spectrometer (precision variant of the transform) ----
 * The spectrometer's transform (Sec. 2: FFT of each segment, auto and cross products,
 * accumulation; Stokes by Eq. 2) for one FFT pair of IFs, with the FFT taken as radix-64
 * Stockham passes whose 64-point DFTs run as GEMMs on the tensor cores (tcgen05.mma,
 * 16-bit operands, FP32 accumulation).  FP32 data are split into two 16-bit halves and
 * multiplied as three products (the lo x lo term dropped):
 *   POLARIS_TC_BF16X3  bf16 halves (about 17 significant bits)
 *   POLARIS_TC_FP16X3  fp16 halves (about 22 bits), each DFT vector scaled by an exact
 *                      power of two into fp16 range
 *   POLARIS_TC_BF16X1  one bf16 product (the plain 16-bit tensor-core result)
 * Twiddles and DFT matrices are FP64-computed; integration accumulators are FP64.
 * polaris_tc_create: n_fft 4096 (= 64^2) or 262144 (= 64^3); bits 1/2/4/8; window
 *   POLARIS_WIN_* (taps: n_fft floats for POLARIS_WIN_CUSTOM, copied); on `device`.
 *   Holds about 70 MB of device memory (two 32 MB pass buffers).
 * polaris_tc_feed: packed[2] are DEVICE pointers to the two IFs' packed streams (layout as
 *   spectrometer_feed), n_samples each, a multiple of n_fft (whole segments, hop = n_fft);
 *   queued on cuda_stream (NULL = legacy stream); accumulates.
 * polaris_tc_integrate: writes DEVICE fp64 outputs (each may be NULL): autos [2][nbin],
 *   cross [nbin][2] (X conj Y), stokes [4][nbin] (I, Q, U, V for linear feeds, psi = 0,
 *   unit gains); nbin = n_fft/2 + 1; *n_segments (host) = segments integrated; clears the
 *   accumulators; synchronises cuda_stream.  POLARIS_ETIMEOUT if a tensor-core completion
 *   wait ran out (bounded; polaris_tc_set_wait_limit lowers the bound for tests, -1
 *   restores it), after which the handle answers POLARIS_ESTATE.
 * Errors: POLARIS_EINVAL (bad argument), POLARIS_ENOMEM, POLARIS_ECUDA; text from
 * polaris_tc_last_error (NULL handle: the last failed create in this thread). */
enum { POLARIS_TC_BF16X3 = 0, POLARIS_TC_FP16X3 = 1, POLARIS_TC_BF16X1 = 2 };
typedef struct polaris_tc polaris_tc;
int polaris_tc_create(int64_t n_fft, int bits, int window, const float* taps, int precision, int device,
                      polaris_tc** out);
int polaris_tc_feed(polaris_tc* h, const void* const* packed, int64_t n_samples, void* cuda_stream);
int polaris_tc_integrate(polaris_tc* h, double* autos, double* cross, double* stokes, int64_t* n_segments,
                         void* cuda_stream);
int polaris_tc_set_wait_limit(polaris_tc* h, int64_t limit);
void polaris_tc_destroy(polaris_tc* h);
const char* polaris_tc_last_error(const polaris_tc* h);

/* Bounded device-side waits.  Phase 2 (N >= 2^17) prefetches its next columns with
 * asynchronous bulk copies and waits for them on a shared-memory barrier; every such wait
 * polls at most a fixed number of times.  If one runs out, the kernel records the fact in
 * the handle's device status word, waits (again bounded) for its own copies in flight,
 * releases its tensor memory and returns; the readout then writes NaN to every output,
 * and the next synchronising call on the handle (spectrometer_integrate,
 * spectrometer_code_histogram) returns POLARIS_ETIMEOUT, after which the handle is
 * unusable (POLARIS_ESTATE).  The GPU context stays usable.
 * Test hook: polls per wait for later launches (0 makes every such wait run out at once;
 * a negative value restores the default of 2^20). */
void polaris_set_wait_limit(int64_t polls);

/* Bounds-checked build.  Compiled with -DPOLARIS_CHECK, every kernel of the spectrometer
 * path (phase kernels, readout, code histogram) tests each global-memory index that the
 * hardware does not check (tensor-map copies are checked by the copy engine) against its
 * buffer's extent; an index outside skips that access and sets the handle's device status
 * word, and the next synchronising call returns POLARIS_EBOUNDS.  Nothing traps.
 * polaris_checked_build: 1 in such a build, 0 otherwise.
 * polaris_set_check_understate (test hook, checked build only): on != 0 makes later feeds
 * tell the kernels half the slab they have, so that the checks fire while every access
 * stays inside its buffer; POLARIS_EINVAL in a build without checks. */
int polaris_checked_build(void);
int polaris_set_check_understate(int on);

/* Test hook: cap the bytes of device memory that later spectrometer_create
 * calls may allocate (-1 = no cap), so that allocation failure can be tested
 * without exhausting the GPU. */
void polaris_set_alloc_limit(int64_t bytes);

#ifdef __cplusplus
}
#endif

#endif /* POLARIS_H */
