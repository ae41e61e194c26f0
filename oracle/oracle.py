"""ctypes wrapper around ``polaris_oracle.c`` (FP64 CPU oracle).

TEST INFRASTRUCTURE ONLY (see the package docstring).  The C file is built with
gcc into ``oracle/liboracle.so`` by :func:`build` (called from
``__graft_entry__.build()`` and lazily on first use).

Each wrapper states the passage of the paper it follows:
  decode      - Fig. 2 caption ("data translation": integer codes to floats)
  window      - Sec. 3.1 (rectangular window online; other windows possible, Sec. 5)
  dft / fft   - the FFT of each segment (Fig. 1, Fig. 2 captions), unnormalised, e^{-i}
  accumulate  - power and cross spectra <XX*>, <YY*>, <XY*> summed over the
                integration (Fig. 1 caption, Table 1, Sec. 2 functions (3)-(4))
  stokes      - Eq. (2) (linear feeds); circular-feed reading in polaris_oracle.c
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polaris_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_U32 = ctypes.POINTER(ctypes.c_uint32)
_I32 = ctypes.POINTER(ctypes.c_int)
_I64 = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math) and return the .so path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oracle_decode.argtypes = [ctypes.c_int, _U32, ctypes.c_int64, _D]
            lib.oracle_window.argtypes = [ctypes.c_int, ctypes.c_int64, _F, _D]
            lib.oracle_dft.argtypes = [ctypes.c_int64, _D, _D, _D, _D]
            lib.oracle_fft.argtypes = [ctypes.c_int64, _D, _D]
            lib.oracle_stokes.argtypes = [ctypes.c_int, ctypes.c_double, _D, _D, ctypes.c_int64, _D, _D, _D, _D]
            lib.oracle_spectra_levels.argtypes = [
                ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _F, ctypes.c_int, _I32,
                ctypes.POINTER(_D), ctypes.c_int64, _D, _D, _I64,
            ]
            lib.oracle_code_histogram.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64,
                                                  ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                                  ctypes.POINTER(ctypes.c_uint64)]
            lib.oracle_power.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), _D, _D]
            lib.oracle_leak_forward.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p),
                                                ctypes.c_int64, _D, _D, _D, _D, _D, _D]
            lib.oracle_leak_grad.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_void_p),
                                             ctypes.c_int64, _D, _D, _D, _D, _D, _D, _D]
            lib.oracle_accumulate.argtypes = [
                ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int, _F, ctypes.c_int, _I32,
                ctypes.POINTER(_U32), ctypes.c_int64, _D, _D, _I64,
            ]
            for f in ("oracle_decode", "oracle_window", "oracle_dft", "oracle_fft", "oracle_stokes", "oracle_accumulate",
                      "oracle_spectra_levels", "oracle_code_histogram", "oracle_power", "oracle_leak_forward",
                      "oracle_leak_grad"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def default_pairs(n_if: int):
    """Table 1 pairs IF names X0, X1, Y0, Y1 as (X0, Y0), (X1, Y1): for an even
    number of IFs, IF i pairs with IF i + n_if/2.  Odd counts have no default pairs."""
    if n_if % 2:
        return []
    h = n_if // 2
    return [(i, i + h) for i in range(h)]


def decode(bits: int, words: np.ndarray, n: int) -> np.ndarray:
    lib = _load()
    w = np.ascontiguousarray(words, dtype=np.uint32)
    out = np.empty(max(n, 1), dtype=np.float64)
    _check(lib.oracle_decode(bits, _p(w, _U32), n, _p(out, _D)), "decode")
    return out[:n]


def window(kind: int, n: int, taps=None) -> np.ndarray:
    lib = _load()
    out = np.empty(n, dtype=np.float64)
    t = None if taps is None else np.ascontiguousarray(taps, dtype=np.float32)
    _check(lib.oracle_window(kind, n, None if t is None else _p(t, _F), _p(out, _D)), "window")
    return out


def dft(x: np.ndarray) -> np.ndarray:
    lib = _load()
    x = np.asarray(x, dtype=np.complex128)
    xr, xi = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    yr, yi = np.empty_like(xr), np.empty_like(xi)
    _check(lib.oracle_dft(len(x), _p(xr, _D), _p(xi, _D), _p(yr, _D), _p(yi, _D)), "dft")
    return yr + 1j * yi


def fft(x: np.ndarray) -> np.ndarray:
    lib = _load()
    x = np.asarray(x, dtype=np.complex128)
    re, im = np.ascontiguousarray(x.real).copy(), np.ascontiguousarray(x.imag).copy()
    _check(lib.oracle_fft(len(x), _p(re, _D), _p(im, _D)), "fft")
    return re + 1j * im


def stokes(aa, bb, ab, feed: int = 0, psi: float = 0.0, ga=1.0 + 0j, gb=1.0 + 0j) -> np.ndarray:
    """Stokes (4, nbin) from power spectra aa, bb and complex cross ab = sum A conj(B)."""
    lib = _load()
    aa = np.ascontiguousarray(aa, dtype=np.float64)
    bb = np.ascontiguousarray(bb, dtype=np.float64)
    abc = np.asarray(ab, dtype=np.complex128)
    abi = np.ascontiguousarray(np.stack([abc.real, abc.imag], axis=-1).reshape(-1))
    g1 = np.array([complex(ga).real, complex(ga).imag], dtype=np.float64)
    g2 = np.array([complex(gb).real, complex(gb).imag], dtype=np.float64)
    out = np.empty((4, len(aa)), dtype=np.float64)
    _check(lib.oracle_stokes(feed, psi, _p(g1, _D), _p(g2, _D), len(aa), _p(aa, _D), _p(bb, _D), _p(abi, _D),
                             _p(out, _D)), "stokes")
    return out


def accumulate(packed, bits: int, n_fft: int, n_samples: int, hop: int | None = None, window_kind: int = 0,
               taps=None, pairs=None):
    """Decode, segment, window, FFT and accumulate.

    packed: list of uint32 arrays, one per IF.  Returns (autos[n_if, N/2+1],
    cross[n_pair, N/2+1] complex, n_segments)."""
    lib = _load()
    n_if = len(packed)
    hop = n_fft if hop is None else hop
    pairs = default_pairs(n_if) if pairs is None else list(pairs)
    nbin = n_fft // 2 + 1
    words = [np.ascontiguousarray(p, dtype=np.uint32) for p in packed]
    arr = (_U32 * n_if)(*[_p(w, _U32) for w in words])
    pr = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1)) if pairs else np.zeros(1, np.int32)
    autos = np.zeros((n_if, nbin), dtype=np.float64)
    cross = np.zeros((max(len(pairs), 1), nbin, 2), dtype=np.float64)
    t = None if taps is None else np.ascontiguousarray(taps, dtype=np.float32)
    nseg = ctypes.c_int64(0)
    _check(lib.oracle_accumulate(n_if, bits, n_fft, hop, window_kind, None if t is None else _p(t, _F), len(pairs),
                                 _p(pr, _I32), arr, n_samples, _p(autos, _D), _p(cross, _D), ctypes.byref(nseg)),
           "accumulate")
    crossc = cross[..., 0] + 1j * cross[..., 1]
    return autos, crossc[: len(pairs)], int(nseg.value)


def spectra_levels(levels, n_fft: int, hop: int | None = None, window_kind: int = 0, taps=None, pairs=None):
    """Steps 2-5 on decoded float levels (list of float64 arrays, one per IF, equal length).
    Returns (autos[n_if, N/2+1], cross[n_pair, N/2+1] complex, n_segments)."""
    lib = _load()
    n_if = len(levels)
    hop = n_fft if hop is None else hop
    pairs = default_pairs(n_if) if pairs is None else list(pairs)
    nbin = n_fft // 2 + 1
    lv = [np.ascontiguousarray(x, dtype=np.float64) for x in levels]
    n = min(len(x) for x in lv)
    arr = (_D * n_if)(*[_p(x, _D) for x in lv])
    pr = np.ascontiguousarray(np.array(pairs, dtype=np.int32).reshape(-1)) if pairs else np.zeros(1, np.int32)
    autos = np.zeros((n_if, nbin), dtype=np.float64)
    cross = np.zeros((max(len(pairs), 1), nbin, 2), dtype=np.float64)
    t = None if taps is None else np.ascontiguousarray(taps, dtype=np.float32)
    nseg = ctypes.c_int64(0)
    _check(lib.oracle_spectra_levels(n_if, n_fft, hop, window_kind, None if t is None else _p(t, _F), len(pairs),
                                     _p(pr, _I32), arr, n, _p(autos, _D), _p(cross, _D), ctypes.byref(nseg)),
           "spectra_levels")
    crossc = cross[..., 0] + 1j * cross[..., 1]
    return autos, crossc[: len(pairs)], int(nseg.value)


def spectrometer(packed, bits: int, n_fft: int, n_samples: int, hop: int | None = None, window_kind: int = 0,
                 taps=None, pairs=None, feed: int = 0, psi: float = 0.0, gains=None):
    """Whole path: returns dict(autos, cross, stokes[n_pair, 4, nbin], n_segments).
    gains: optional list of (Ga, Gb) per pair (complex)."""
    n_if = len(packed)
    pairs = default_pairs(n_if) if pairs is None else list(pairs)
    autos, cross, nseg = accumulate(packed, bits, n_fft, n_samples, hop, window_kind, taps, pairs)
    st = np.zeros((len(pairs), 4, n_fft // 2 + 1))
    for p, (a, b) in enumerate(pairs):
        ga, gb = (1.0, 1.0) if gains is None else gains[p]
        st[p] = stokes(autos[a], autos[b], cross[p], feed=feed, psi=psi, ga=ga, gb=gb)
    return {"autos": autos, "cross": cross, "stokes": st, "n_segments": nseg}


def code_histogram(packed, bits: int, n_fft: int, n_samples: int, hop: int | None = None) -> np.ndarray:
    """Per-IF code counts [n_if, 2^bits] over every whole segment (Sec. 2 bit distribution)."""
    hop = n_fft if hop is None else hop
    words = [np.ascontiguousarray(p, dtype=np.uint32) for p in packed]
    arr = (ctypes.c_void_p * len(words))(*[w.ctypes.data for w in words])
    out = np.zeros((len(words), 1 << bits), np.uint64)
    _check(_load().oracle_code_histogram(len(words), bits, n_fft, hop, arr, n_samples,
                                         out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))), "code_histogram")
    return out


def power(bits: int, counts) -> tuple[float, float]:
    """(moment2, sigma_over_threshold) of one IF's code histogram."""
    c = np.ascontiguousarray(np.asarray(counts, dtype=np.uint64).reshape(-1))
    m2 = np.zeros(1)
    sg = np.zeros(1)
    _check(_load().oracle_power(bits, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _p(m2, _D), _p(sg, _D)),
           "power")
    return float(m2[0]), float(sg[0])


def _leak_args(packed, window, gains, leak, target):
    words = [np.ascontiguousarray(p, dtype=np.uint32) for p in packed]
    arr = (ctypes.c_void_p * 2)(*[w.ctypes.data for w in words])
    f = [np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1)) if x is not None else None
         for x in (window, gains, leak, target)]
    return words, arr, f


def leak_forward(packed, bits: int, n_fft: int, n_samples: int, window, gains, leak, target=None):
    """(stokes [4, nbin], loss or None) of the leakage model (circular feeds, two IFs)."""
    words, arr, (w, g, d, t) = _leak_args(packed, window, gains, leak, target)
    nbin = n_fft // 2 + 1
    st = np.zeros(4 * nbin)
    loss = np.zeros(1)
    _check(_load().oracle_leak_forward(bits, n_fft, arr, n_samples, _p(w, _D), _p(g, _D), _p(d, _D),
                                       None if t is None else _p(t, _D), _p(st, _D), _p(loss, _D)), "leak_forward")
    return st.reshape(4, nbin), (float(loss[0]) if t is not None else None)


def leak_grad(packed, bits: int, n_fft: int, n_samples: int, window, gains, leak, target):
    """Gradients of the loss: (grad_window [N], grad_gains [4], grad_leak [2, nbin, 2])."""
    words, arr, (w, g, d, t) = _leak_args(packed, window, gains, leak, target)
    nbin = n_fft // 2 + 1
    gw, gg, gd = np.zeros(n_fft), np.zeros(4), np.zeros(4 * nbin)
    _check(_load().oracle_leak_grad(bits, n_fft, arr, n_samples, _p(w, _D), _p(g, _D), _p(d, _D), _p(t, _D),
                                    _p(gw, _D), _p(gg, _D), _p(gd, _D)), "leak_grad")
    return gw, gg, gd.reshape(2, nbin, 2)
