"""Thin ctypes binding over ``libpolaris.so`` (C ABI in ``include/polaris.h``).

Argument marshalling only: every step of the hot path (data translation,
windowing, FFT, correlation, accumulation, Stokes) runs in the library's CUDA
kernels.  Host inputs are numpy arrays; device inputs and outputs are torch CUDA
tensors (PyTorch provides device memory and streams, nothing else).  There is
no fallback: if the library is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# POLARIS_LIB selects another build of the library (e.g. a tuning variant)
LIB_PATH = os.environ.get("POLARIS_LIB") or os.path.join(HERE, "libpolaris.so")

OK, EINVAL, ENOMEM, ECUDA, ESTATE, ETIMEOUT, EBOUNDS = 0, -1, -2, -3, -4, -5, -6
WIN_RECT, WIN_HANN, WIN_CUSTOM = 0, 1, 2
FEED_LINEAR, FEED_CIRCULAR = 0, 1
TC_BF16X3, TC_FP16X3, TC_BF16X1 = 0, 1, 2
INPUT_HOST, INPUT_DEVICE, INPUT_HOST_ASYNC = 0, 1, 2
STATUS_NAMES = {EINVAL: "EINVAL", ENOMEM: "ENOMEM", ECUDA: "ECUDA", ESTATE: "ESTATE", ETIMEOUT: "ETIMEOUT",
                EBOUNDS: "EBOUNDS"}

EXPORTS = (
    "spectrometer_create", "spectrometer_feed", "spectrometer_integrate", "spectrometer_integrate_device",
    "spectrometer_n_bins", "spectrometer_n_pairs", "spectrometer_debug_unpack", "spectrometer_destroy",
    "spectrometer_last_error", "spectrometer_debug_unpack_staged", "polaris_set_alloc_limit", "spectrometer_kernel_launches",
    "spectrometer_set_profiling", "spectrometer_kernel_times", "spectrometer_run_noalloc",
    "spectrometer_code_histogram", "polaris_power_from_histogram", "polaris_set_wait_limit",
    "spectrometer_integrate_async", "polaris_checked_build", "polaris_set_check_understate",
    "spectrometer_get_launch", "spectrometer_set_launch_caps",
    "polaris_adj_create", "polaris_adj_run", "polaris_adj_destroy", "polaris_adj_last_error",
    "polaris_tc_create", "polaris_tc_feed", "polaris_tc_integrate", "polaris_tc_set_wait_limit",
    "polaris_tc_destroy", "polaris_tc_last_error",
)


class PolarisError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class polaris_config(ctypes.Structure):
    _fields_ = [
        ("n_if", ctypes.c_int), ("bits", ctypes.c_int), ("n_fft", ctypes.c_int64), ("hop", ctypes.c_int64),
        ("window", ctypes.c_int), ("taps", ctypes.POINTER(ctypes.c_float)), ("n_pair", ctypes.c_int),
        ("pairs", ctypes.POINTER(ctypes.c_int)), ("accum_fp64", ctypes.c_int), ("device", ctypes.c_int),
        ("max_batch_segments", ctypes.c_int), ("code_stats", ctypes.c_int),
    ]


class polaris_stokes_params(ctypes.Structure):
    _fields_ = [("feed", ctypes.c_int), ("psi_m", ctypes.c_double), ("gains", ctypes.POINTER(ctypes.c_float))]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Load libpolaris.so (raises if it is absent: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise FileNotFoundError(f"{path} not built; run __graft_entry__.build()")
            lib = ctypes.CDLL(path)
            vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            lib.spectrometer_create.argtypes = [ctypes.POINTER(polaris_config), ctypes.POINTER(vp)]
            lib.spectrometer_create.restype = ci
            lib.spectrometer_feed.argtypes = [vp, ctypes.POINTER(vp), i64, ci, vp]
            lib.spectrometer_feed.restype = ci
            lib.spectrometer_integrate.argtypes = [vp, ctypes.POINTER(polaris_stokes_params), vp, vp, vp,
                                                   ctypes.POINTER(i64)]
            lib.spectrometer_integrate.restype = ci
            lib.spectrometer_integrate_device.argtypes = [vp, ctypes.POINTER(polaris_stokes_params), vp, vp, vp,
                                                          ctypes.POINTER(i64), vp]
            lib.spectrometer_integrate_device.restype = ci
            lib.spectrometer_integrate_async.argtypes = [vp, ctypes.POINTER(polaris_stokes_params), vp, vp, vp,
                                                         ctypes.POINTER(i64), vp]
            lib.spectrometer_integrate_async.restype = ci
            lib.spectrometer_n_bins.argtypes = [vp]
            lib.spectrometer_n_bins.restype = i64
            lib.spectrometer_get_launch.argtypes = [vp] + [ctypes.POINTER(ci)] * 3
            lib.spectrometer_get_launch.restype = ci
            lib.spectrometer_set_launch_caps.argtypes = [vp, ci, ci]
            lib.spectrometer_set_launch_caps.restype = ci
            lib.spectrometer_n_pairs.argtypes = [vp]
            lib.spectrometer_n_pairs.restype = ci
            lib.spectrometer_debug_unpack.argtypes = [vp, vp, i64, vp]
            lib.spectrometer_debug_unpack.restype = ci
            lib.spectrometer_debug_unpack_staged.argtypes = [vp, vp, vp, i64, ci, vp, vp]
            lib.spectrometer_debug_unpack_staged.restype = ci
            lib.spectrometer_destroy.argtypes = [vp]
            lib.spectrometer_destroy.restype = None
            lib.spectrometer_last_error.argtypes = [vp]
            lib.spectrometer_last_error.restype = ctypes.c_char_p
            lib.spectrometer_kernel_launches.argtypes = [vp]
            lib.spectrometer_kernel_launches.restype = i64
            lib.spectrometer_set_profiling.argtypes = [vp, ci]
            lib.spectrometer_set_profiling.restype = ci
            lib.spectrometer_kernel_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64), ci]
            lib.spectrometer_kernel_times.restype = ci
            lib.spectrometer_run_noalloc.argtypes = [ctypes.POINTER(polaris_config), ctypes.POINTER(vp), i64,
                                                     ctypes.POINTER(polaris_stokes_params), vp, vp, vp,
                                                     ctypes.POINTER(i64), vp]
            lib.spectrometer_run_noalloc.restype = ci
            lib.polaris_set_alloc_limit.argtypes = [i64]
            lib.polaris_set_alloc_limit.restype = None
            lib.polaris_checked_build.argtypes = []
            lib.polaris_checked_build.restype = ci
            lib.polaris_set_check_understate.argtypes = [ci]
            lib.polaris_set_check_understate.restype = ci
            lib.polaris_adj_create.argtypes = [i64, ci, ci, ctypes.POINTER(vp)]
            lib.polaris_adj_create.restype = ci
            lib.polaris_adj_run.argtypes = [vp, ctypes.POINTER(vp), i64] + [vp] * 10
            lib.polaris_adj_run.restype = ci
            lib.polaris_adj_destroy.argtypes = [vp]
            lib.polaris_adj_destroy.restype = None
            lib.polaris_adj_last_error.argtypes = [vp]
            lib.polaris_adj_last_error.restype = ctypes.c_char_p
            lib.polaris_tc_create.argtypes = [i64, ci, ci, vp, ci, ci, ctypes.POINTER(vp)]
            lib.polaris_tc_create.restype = ci
            lib.polaris_tc_feed.argtypes = [vp, ctypes.POINTER(vp), i64, vp]
            lib.polaris_tc_feed.restype = ci
            lib.polaris_tc_integrate.argtypes = [vp, vp, vp, vp, ctypes.POINTER(i64), vp]
            lib.polaris_tc_integrate.restype = ci
            lib.polaris_tc_set_wait_limit.argtypes = [vp, i64]
            lib.polaris_tc_set_wait_limit.restype = ci
            lib.polaris_tc_destroy.argtypes = [vp]
            lib.polaris_tc_destroy.restype = None
            lib.polaris_tc_last_error.argtypes = [vp]
            lib.polaris_tc_last_error.restype = ctypes.c_char_p
            lib.polaris_set_wait_limit.argtypes = [i64]
            lib.polaris_set_wait_limit.restype = None
            lib.spectrometer_code_histogram.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ci]
            lib.spectrometer_code_histogram.restype = ci
            lib.polaris_power_from_histogram.argtypes = [ci, ctypes.POINTER(ctypes.c_uint64),
                                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
            lib.polaris_power_from_histogram.restype = ci
            _lib = lib
    return _lib


def set_alloc_limit(nbytes: int) -> None:
    load().polaris_set_alloc_limit(int(nbytes))


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


def _ptr(x):
    """Address of a numpy array or torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x.data_ptr())


def set_wait_limit(polls: int) -> None:
    """Test hook: polls per bounded device-side wait for later launches (0: every such wait
    runs out at once; negative: the default)."""
    load().polaris_set_wait_limit(int(polls))


def power_from_histogram(bits: int, counts) -> tuple[float, float]:
    """(moment2, sigma_over_threshold) of one IF's code histogram (polaris_power_from_histogram)."""
    c = np.ascontiguousarray(np.asarray(counts, dtype=np.uint64).reshape(-1))
    m2, sg = ctypes.c_double(), ctypes.c_double()
    rc = load().polaris_power_from_histogram(int(bits), c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                             ctypes.byref(m2), ctypes.byref(sg))
    if rc != OK:
        raise PolarisError(rc, "invalid histogram")
    return m2.value, sg.value


class Spectrometer:
    """One spectrometer handle.  Mirrors spectrometer_create / feed / integrate / destroy."""

    def __init__(self, n_if: int, bits: int, n_fft: int, hop: int = 0, window="rect", pairs=None,
                 accum_fp64: bool = False, device: int = 0, max_batch_segments: int = 0,
                 code_stats: bool = False):
        lib = load()
        cfg = polaris_config()
        cfg.n_if, cfg.bits, cfg.n_fft, cfg.hop = n_if, bits, n_fft, hop
        self._taps = None
        if isinstance(window, str):
            cfg.window = {"rect": WIN_RECT, "hann": WIN_HANN}[window]
        elif isinstance(window, int):
            cfg.window = window
        else:
            self._taps = np.ascontiguousarray(window, dtype=np.float32)
            cfg.window = WIN_CUSTOM
            cfg.taps = self._taps.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        self._pairs = None
        if pairs is not None:
            self._pairs = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1))
            cfg.n_pair = len(self._pairs) // 2
            cfg.pairs = self._pairs.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        cfg.accum_fp64 = int(bool(accum_fp64))
        cfg.device = device
        cfg.max_batch_segments = max_batch_segments
        cfg.code_stats = int(bool(code_stats))
        h = ctypes.c_void_p()
        rc = lib.spectrometer_create(ctypes.byref(cfg), ctypes.byref(h))
        if rc != OK:
            raise PolarisError(rc, lib.spectrometer_last_error(None).decode())
        self._h = h
        self.n_if, self.bits, self.n_fft = n_if, bits, n_fft
        self.n_bins = int(lib.spectrometer_n_bins(h))
        self.n_pairs = int(lib.spectrometer_n_pairs(h))
        self.device = device

    def _check(self, rc):
        if rc != OK:
            raise PolarisError(rc, load().spectrometer_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().spectrometer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def feed(self, packed, n_samples: int, on_device: bool | None = None, stream=None, host_async: bool = False) -> None:
        """packed: one array/tensor of uint32 words per IF (numpy -> host, torch CUDA -> device).
        host_async (host input only): queue the copy and return at once; the host arrays
        (pinned, for an asynchronous copy) must stay unchanged until the stream passes."""
        if on_device is None:
            on_device = not isinstance(packed[0], np.ndarray)
        if not on_device:
            packed = [np.ascontiguousarray(p, dtype=np.uint32) for p in packed]
        arr = (ctypes.c_void_p * self.n_if)(*[_ptr(p) for p in packed])
        self._keep = packed
        mode = INPUT_DEVICE if on_device else (INPUT_HOST_ASYNC if host_async else INPUT_HOST)
        self._check(load().spectrometer_feed(self._h, arr, int(n_samples), mode, _stream_ptr(stream)))

    @staticmethod
    def _params(feed: int, psi: float, gains):
        p = polaris_stokes_params()
        p.feed, p.psi_m = feed, psi
        g = None
        if gains is not None:
            g = np.ascontiguousarray(np.array([[complex(a).real, complex(a).imag, complex(b).real, complex(b).imag]
                                               for a, b in gains], dtype=np.float32).reshape(-1))
            p.gains = g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        return p, g

    def integrate(self, feed: int = FEED_LINEAR, psi: float = 0.0, gains=None, out=None):
        """Close the integration; returns dict(autos, cross (complex64), stokes, n_segments) as numpy.

        out: optional dict of preallocated C-contiguous float32 arrays 'autos' [n_if, nb],
        'cross' [n_pair, nb, 2], 'stokes' [n_pair, 4, nb] to fill (views of pinned host
        memory make the device-to-host copies direct); missing entries are allocated."""
        nb, npair = self.n_bins, self.n_pairs
        out = {} if out is None else out

        def buf(key, shape):
            a = out.get(key)
            if a is None:
                return np.empty(shape, np.float32)
            if a.dtype != np.float32 or tuple(a.shape) != shape or not a.flags["C_CONTIGUOUS"]:
                raise ValueError(f"out[{key!r}] must be a C-contiguous float32 array of shape {shape}")
            return a

        autos = buf("autos", (self.n_if, nb))
        cross = buf("cross", (npair, nb, 2)) if npair else None
        stokes = buf("stokes", (npair, 4, nb)) if npair else None
        nseg = ctypes.c_int64(0)
        p, g = self._params(feed, psi, gains)
        self._check(load().spectrometer_integrate(self._h, ctypes.byref(p), autos.ctypes.data,
                                                  None if cross is None else cross.ctypes.data,
                                                  None if stokes is None else stokes.ctypes.data, ctypes.byref(nseg)))
        del g
        if cross is None:
            cross = np.empty((0, nb, 2), np.float32)
            stokes = np.empty((0, 4, nb), np.float32)
        return {"autos": autos, "cross": cross.view(np.complex64)[..., 0], "stokes": stokes,
                "n_segments": int(nseg.value)}

    def integrate_device(self, autos, cross, stokes, feed: int = FEED_LINEAR, psi: float = 0.0, gains=None,
                         stream=None) -> int:
        """Outputs into device tensors (float32: autos [n_if, nb], cross [n_pair, nb, 2],
        stokes [n_pair, 4, nb]; None skips).  Returns the segment count."""
        nseg = ctypes.c_int64(0)
        p, g = self._params(feed, psi, gains)
        self._check(load().spectrometer_integrate_device(
            self._h, ctypes.byref(p), None if autos is None else _ptr(autos), None if cross is None else _ptr(cross),
            None if stokes is None else _ptr(stokes), ctypes.byref(nseg), _stream_ptr(stream)))
        del g
        return int(nseg.value)

    def integrate_async(self, out, feed: int = FEED_LINEAR, psi: float = 0.0, gains=None, stream=None) -> int:
        """Queue the readout and the copies into the HOST arrays of `out` ('autos' [n_if, nb],
        'cross' [n_pair, nb, 2], 'stokes' [n_pair, 4, nb], float32, C-contiguous; pinned for
        asynchronous copies; missing keys skip) on `stream` without waiting.  The arrays
        are valid once the stream has passed this call.  Returns the segment count."""
        nseg = ctypes.c_int64(0)
        p, g = self._params(feed, psi, gains)
        ptr = [None if out.get(k) is None else _ptr(out[k]) for k in ("autos", "cross", "stokes")]
        self._check(load().spectrometer_integrate_async(self._h, ctypes.byref(p), ptr[0], ptr[1], ptr[2],
                                                        ctypes.byref(nseg), _stream_ptr(stream)))
        del g
        return int(nseg.value)

    def launch_choices(self) -> dict:
        """Segments per kernel pass and the CTA-per-SM caps of the two FFT kernels (0: as many
        as fit), as the handle uses them."""
        mb, c1, c2 = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(load().spectrometer_get_launch(self._h, ctypes.byref(mb), ctypes.byref(c1), ctypes.byref(c2)))
        return {"max_batch_segments": mb.value, "phase1_ctas_per_sm": c1.value, "phase2_ctas_per_sm": c2.value}

    def set_launch_caps(self, phase1_ctas_per_sm: int, phase2_ctas_per_sm: int) -> None:
        self._check(load().spectrometer_set_launch_caps(self._h, int(phase1_ctas_per_sm), int(phase2_ctas_per_sm)))

    def kernel_launches(self) -> int:
        return int(load().spectrometer_kernel_launches(self._h))

    def set_profiling(self, on: bool) -> None:
        self._check(load().spectrometer_set_profiling(self._h, int(bool(on))))

    KERNEL_KINDS = ("phase1_decode_rowdft", "phase2_coldft_correlate", "readout_stokes", "code_histogram")

    def kernel_times(self):
        """{kind: (total_ms, launches)} for launches bracketed since set_profiling(True)."""
        n = len(self.KERNEL_KINDS)
        ms = (ctypes.c_double * n)()
        nl = (ctypes.c_int64 * n)()
        self._check(load().spectrometer_kernel_times(self._h, ms, nl, n))
        return {k: (ms[i], int(nl[i])) for i, k in enumerate(self.KERNEL_KINDS)}

    def code_histogram(self, reset: bool = False) -> np.ndarray:
        """Per-IF code counts [n_if, 2^bits] (uint64) over the segments integrated since creation
        or the last reset (needs code_stats=True)."""
        out = np.zeros((self.n_if, 1 << self.bits), np.uint64)
        self._check(load().spectrometer_code_histogram(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                                       int(bool(reset))))
        return out

    def debug_unpack(self, words: np.ndarray, n: int) -> np.ndarray:
        w = np.ascontiguousarray(words, dtype=np.uint32)
        out = np.empty(max(n, 1), np.float32)
        self._check(load().spectrometer_debug_unpack(self._h, w.ctypes.data, int(n), out.ctypes.data))
        return out[:n]

    def debug_unpack_staged(self, words_a: np.ndarray, words_b, n: int, layout: int = 0):
        """Levels of n samples (whole segments) of IF a and IF b (words_b None: a pair without
        an IF b) through the FFT kernel's staged decoder; layout 0 interleaved, 1 dense.
        Returns (levels_a, levels_b or None)."""
        wa = np.ascontiguousarray(words_a, dtype=np.uint32)
        wb = None if words_b is None else np.ascontiguousarray(words_b, dtype=np.uint32)
        oa = np.empty(n, np.float32)
        ob = None if wb is None else np.empty(n, np.float32)
        self._check(load().spectrometer_debug_unpack_staged(self._h, wa.ctypes.data,
                                                            None if wb is None else wb.ctypes.data, int(n),
                                                            int(layout), oa.ctypes.data,
                                                            None if ob is None else ob.ctypes.data))
        return oa, ob


def run_noalloc(packed, n_samples: int, bits: int, n_fft: int, autos, cross, stokes, hop: int = 0, window="rect",
                pairs=None, accum_fp64: bool = False, device: int = 0, feed: int = FEED_LINEAR, psi: float = 0.0,
                gains=None, stream=None) -> int:
    """spectrometer_run_noalloc: one integration of device-resident packed streams into
    device output tensors, using only the library's static device array (no allocation
    by the library).  For callers that cannot allocate device memory at this point, e.g.
    a real-time loop that must not synchronise the device, or a host that owns all device
    memory.  Returns the segment count."""
    lib = load()
    cfg = polaris_config()
    cfg.n_if, cfg.bits, cfg.n_fft, cfg.hop = len(packed), bits, n_fft, hop
    keep = []
    if isinstance(window, str):
        cfg.window = {"rect": WIN_RECT, "hann": WIN_HANN}[window]
    else:
        t = np.ascontiguousarray(window, dtype=np.float32)
        keep.append(t)
        cfg.window = WIN_CUSTOM
        cfg.taps = t.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    if pairs is not None:
        pr = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1))
        keep.append(pr)
        cfg.n_pair = len(pr) // 2
        cfg.pairs = pr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    cfg.accum_fp64 = int(bool(accum_fp64))
    cfg.device = device
    arr = (ctypes.c_void_p * len(packed))(*[_ptr(p) for p in packed])
    p, g = Spectrometer._params(feed, psi, gains)
    nseg = ctypes.c_int64(0)
    rc = lib.spectrometer_run_noalloc(ctypes.byref(cfg), arr, int(n_samples), ctypes.byref(p),
                                      None if autos is None else _ptr(autos), None if cross is None else _ptr(cross),
                                      None if stokes is None else _ptr(stokes), ctypes.byref(nseg),
                                      _stream_ptr(stream))
    del g, keep
    if rc != OK:
        raise PolarisError(rc, lib.spectrometer_last_error(None).decode())
    return int(nseg.value)


class Adjoint:
    """Differentiable leakage calibration (polaris_adj_*): forward model, loss and
    gradients for two circular-feed IFs.  Tensors are CUDA tensors (float32 unless stated)."""

    def __init__(self, n_fft: int, bits: int, device: int = 0):
        h = ctypes.c_void_p()
        rc = load().polaris_adj_create(int(n_fft), int(bits), int(device), ctypes.byref(h))
        if rc != OK:
            raise PolarisError(rc, load().polaris_adj_last_error(None).decode())
        self._h, self.n_fft, self.bits, self.device = h, n_fft, bits, device
        self.n_bins = n_fft // 2 + 1

    def close(self):
        if getattr(self, "_h", None):
            load().polaris_adj_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def run(self, packed, n_samples: int, window, gains, leak, target=None, grads: bool = False, stream=None):
        """dict(stokes [4, nb], loss (float64, 1 element) and, with grads=True, grad_window [N],
        grad_gains [4], grad_leak [2, nb, 2]).  packed: two CUDA tensors of packed words."""
        import torch

        dev = window.device
        nb = self.n_bins
        out = {"stokes": torch.empty((4, nb), dtype=torch.float32, device=dev)}
        if target is not None:
            out["loss"] = torch.empty((1,), dtype=torch.float64, device=dev)
        if grads:
            out["grad_window"] = torch.empty((self.n_fft,), dtype=torch.float32, device=dev)
            out["grad_gains"] = torch.empty((4,), dtype=torch.float32, device=dev)
            out["grad_leak"] = torch.empty((2, nb, 2), dtype=torch.float32, device=dev)
        arr = (ctypes.c_void_p * 2)(*[_ptr(p) for p in packed])
        ins = [t.contiguous() for t in (window, gains, leak)]
        tgt = None if target is None else target.contiguous()
        rc = load().polaris_adj_run(self._h, arr, int(n_samples), _ptr(ins[0]), _ptr(ins[1]), _ptr(ins[2]),
                                    None if tgt is None else _ptr(tgt), _ptr(out["stokes"]),
                                    _ptr(out["loss"]) if "loss" in out else None,
                                    _ptr(out["grad_window"]) if grads else None,
                                    _ptr(out["grad_gains"]) if grads else None,
                                    _ptr(out["grad_leak"]) if grads else None, _stream_ptr(stream))
        if rc != OK:
            raise PolarisError(rc, load().polaris_adj_last_error(self._h).decode())
        return out


def leakage_loss(adj: "Adjoint", packed, n_samples: int, window, gains, leak, target):
    """The calibration loss as a differentiable function of window, gains and leak
    (torch.autograd), its gradient from the library's adjoint."""
    import torch

    class _LeakageLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, w, g, d):
            need = any(ctx.needs_input_grad)
            r = adj.run(packed, n_samples, w.detach(), g.detach(), d.detach(), target, grads=need,
                        stream=torch.cuda.current_stream(w.device))
            if need:
                ctx.save_for_backward(r["grad_window"], r["grad_gains"], r["grad_leak"])
            return r["loss"][0]

        @staticmethod
        def backward(ctx, gout):
            gw, gg, gd = ctx.saved_tensors
            s = gout.to(torch.float32)
            return s * gw, s * gg, s * gd

    return _LeakageLoss.apply(window, gains, leak)


class TensorCoreSpectrometer:
    """Tensor-core DFT spectrometer for one FFT pair (polaris_tc_*): the precision variant
    of the transform, radix-64 DFTs as tcgen05 GEMMs with split 16-bit operands, FP64
    accumulators.  Inputs are CUDA tensors of packed words; outputs are float64 tensors."""

    PRECISIONS = {"bf16x3": TC_BF16X3, "fp16x3": TC_FP16X3, "bf16": TC_BF16X1}

    def __init__(self, bits: int, n_fft: int, precision="bf16x3", window="rect", device: int = 0):
        prec = self.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        taps = None
        if isinstance(window, str):
            win = {"rect": WIN_RECT, "hann": WIN_HANN}[window]
        else:
            self._taps = np.ascontiguousarray(window, dtype=np.float32)
            win, taps = WIN_CUSTOM, self._taps.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        rc = load().polaris_tc_create(int(n_fft), int(bits), win, taps, prec, int(device), ctypes.byref(h))
        if rc != OK:
            raise PolarisError(rc, load().polaris_tc_last_error(None).decode())
        self._h, self.bits, self.n_fft, self.device = h, bits, n_fft, device
        self.n_bins = n_fft // 2 + 1

    def _check(self, rc):
        if rc != OK:
            raise PolarisError(rc, load().polaris_tc_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            load().polaris_tc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_wait_limit(self, limit: int) -> None:
        self._check(load().polaris_tc_set_wait_limit(self._h, int(limit)))

    def feed(self, packed, n_samples: int, stream=None) -> None:
        arr = (ctypes.c_void_p * 2)(*[_ptr(p) for p in packed])
        self._check(load().polaris_tc_feed(self._h, arr, int(n_samples), _stream_ptr(stream)))

    def integrate(self, stream=None):
        """dict(autos [2, nb], cross [nb] complex128, stokes [4, nb], n_segments) on the host."""
        import torch

        nb = self.n_bins
        dev = torch.device("cuda", self.device)
        autos = torch.empty((2, nb), dtype=torch.float64, device=dev)
        cross = torch.empty((nb, 2), dtype=torch.float64, device=dev)
        stokes = torch.empty((4, nb), dtype=torch.float64, device=dev)
        nseg = ctypes.c_int64()
        self._check(load().polaris_tc_integrate(self._h, _ptr(autos), _ptr(cross), _ptr(stokes), ctypes.byref(nseg),
                                                _stream_ptr(stream)))
        c = cross.cpu().numpy()
        return {"autos": autos.cpu().numpy(), "cross": c[:, 0] + 1j * c[:, 1], "stokes": stokes.cpu().numpy(),
                "n_segments": nseg.value}
