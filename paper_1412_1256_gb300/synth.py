"""Seeded synthetic IF streams: the stand-in for the K5/VSSP32 sampler.

This module makes test and benchmark inputs only.  It holds none of the
spectrometer's arithmetic (no decoding, windowing, transform or correlation of
the data it makes): it draws Gaussian noise and tones, quantises them the way a
b-bit sampler would, and packs the codes into 32-bit words.  Both the CUDA path
and the CPU oracle consume its output; neither is imported here.

Sample format (the packing codec, our reading; the paper does not describe the
sampler's word format): one planar stream of little-endian uint32 words per IF;
sample j of a word sits in bits [j*b, (j+1)*b), least significant first.
Codes: b < 8 -> unsigned code c whose level is 2c - (2^b - 1); b = 8 -> the
two's-complement int8 value itself.

Workload recipes (the paper's observations are not available; these stand in):
  * ``config_tiny``: 2 IFs (X, Y), int8, Gaussian noise sigma = 20 plus a common
    tone of amplitude 0.3 sigma = 6 at bin 100 of a 1024-point FFT, Y lagging X
    by 90 degrees; 65536 samples per IF (64 segments).
  * ``config_paper``: 4 IFs (X0, X1, Y0, Y1), 2-bit (thresholds +-0.98 sigma,
    levels +-1, +-3), 131072-point segments, Gaussian noise plus three Gaussian
    lines of FWHM 20 channels whose peak spectral density is 5x the continuum,
    at channels 16384 (unpolarised), 32768 (linearly polarised, chi = 30 deg)
    and 49152 (circularly polarised, Y lagging X by 90 deg).
  * ``config_circular``: 2 circular-feed IFs (R, L), int8 (noise sigma = 20),
    16384-point segments, 256 segments; unpolarised noise plus one Gaussian line
    (FWHM 200 channels, peak 3x the continuum, at channel 3000) with fractional
    Stokes q = 0.3, u = -0.2, v = 0.1 (in the circular basis <|R|^2> ~ I + V,
    <|L|^2> ~ I - V, <R conj L> ~ Q + iU).
  * ``config_precision``: 2 IFs (X, Y), int8, 262144-point segments (10 s at 16 Msps =
    610 segments); unit continuum plus a Gaussian line 40 dB above it (peak 10^4, FWHM
    20 channels, at channel 40000) whose circular polarisation follows the Zeeman-like
    antisymmetric profile V = 1e-3 dI/dnu (one channel as the frequency unit, Eq. 1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "samples_per_word", "pack", "unpack_codes", "quantize", "quantize_2bit", "quantize_int8",
    "quantize_1bit", "quantize_4bit", "config_tiny", "config_paper", "paper_block", "random_codes",
    "config_circular", "config_precision",
]


def samples_per_word(bits: int) -> int:
    if bits not in (1, 2, 4, 8):
        raise ValueError("bits must be 1, 2, 4 or 8")
    return 32 // bits


def pack(codes: np.ndarray, bits: int) -> np.ndarray:
    """Pack unsigned b-bit codes (any integer dtype, values < 2^b) into uint32 words,
    sample j of a word in bits [j*b, (j+1)*b).  len(codes) must be a multiple of 32/b."""
    spw = samples_per_word(bits)
    c = np.asarray(codes).astype(np.uint32) & np.uint32((1 << bits) - 1)
    if c.size % spw:
        raise ValueError("sample count must be a multiple of 32/bits")
    c = c.reshape(-1, spw)
    shifts = (np.arange(spw, dtype=np.uint32) * np.uint32(bits))[None, :]
    return np.bitwise_or.reduce(c << shifts, axis=1).astype(np.uint32)


def unpack_codes(words: np.ndarray, bits: int, n: int | None = None) -> np.ndarray:
    """Inverse of :func:`pack`: the raw unsigned codes (not levels)."""
    spw = samples_per_word(bits)
    w = np.asarray(words, dtype=np.uint32)
    shifts = (np.arange(spw, dtype=np.uint32) * np.uint32(bits))[None, :]
    c = ((w[:, None] >> shifts) & np.uint32((1 << bits) - 1)).reshape(-1)
    return c if n is None else c[:n]


def quantize_2bit(v: np.ndarray, sigma: float = 1.0, thr: float = 0.98) -> np.ndarray:
    """4-level sampler: v < -thr*s -> code 0 (level -3); [-thr*s, 0) -> 1 (-1);
    [0, thr*s) -> 2 (+1); >= thr*s -> 3 (+3).  A value of exactly 0 goes to +1."""
    t = thr * sigma
    return (np.where(v < -t, 0, np.where(v < 0, 1, np.where(v < t, 2, 3)))).astype(np.uint8)


def quantize_int8(v: np.ndarray) -> np.ndarray:
    """8-bit sampler: round half to even, clamp to [-128, 127]; returns the code
    bytes (two's complement) as uint8."""
    q = np.clip(np.rint(v), -128, 127).astype(np.int16)
    return (q & 0xFF).astype(np.uint8)


def quantize_1bit(v: np.ndarray) -> np.ndarray:
    """Sign sampler: v >= 0 -> code 1 (+1), else code 0 (-1)."""
    return (v >= 0).astype(np.uint8)


def quantize_4bit(v: np.ndarray, step: float) -> np.ndarray:
    """16-level uniform sampler with odd levels 2c-15: code = clamp(floor(v/step) + 8, 0, 15)."""
    return np.clip(np.floor(v / step) + 8, 0, 15).astype(np.uint8)


def quantize(v: np.ndarray, bits: int, sigma: float = 1.0) -> np.ndarray:
    if bits == 1:
        return quantize_1bit(v)
    if bits == 2:
        return quantize_2bit(v, sigma)
    if bits == 4:
        return quantize_4bit(v, sigma / 2.0)
    if bits == 8:
        return quantize_int8(v)
    raise ValueError("bits must be 1, 2, 4 or 8")


def random_codes(rng: np.random.Generator, n: int, bits: int) -> np.ndarray:
    """Uniformly random codes (every code value equally likely)."""
    return rng.integers(0, 1 << bits, size=n, dtype=np.int64).astype(np.uint8 if bits <= 8 else np.uint32)


def config_tiny(seed: int = 1412, n_samples: int = 65536, n_fft: int = 1024, k0: int = 100, sigma: float = 20.0,
                amp: float = 6.0):
    """Small two-IF int8 workload: noise + common tone, Y lagging X by 90 degrees.
    Returns (list of 2 packed uint32 arrays, dict of parameters)."""
    rng = np.random.default_rng(seed)
    n = np.arange(n_samples, dtype=np.float64)
    ph = 2.0 * np.pi * k0 * n / n_fft
    x = rng.normal(0.0, sigma, n_samples) + amp * np.cos(ph)
    y = rng.normal(0.0, sigma, n_samples) + amp * np.cos(ph - np.pi / 2)
    packed = [pack(quantize_int8(x), 8), pack(quantize_int8(y), 8)]
    return packed, dict(bits=8, n_fft=n_fft, n_samples=n_samples, k0=k0, window="hann")


def _gauss_profile(nbin: int, center: float, fwhm: float) -> np.ndarray:
    k = np.arange(nbin, dtype=np.float64)
    s = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    return np.exp(-0.5 * ((k - center) / s) ** 2)


def paper_block(rng: np.random.Generator, n_fft: int = 131072, line_peak: float = 5.0, fwhm: float = 20.0,
                chi_deg: float = 30.0):
    """One n_fft-sample block of an (X, Y) pair with the three-line spectrum, as floats
    of unit variance.  Synthesised in the frequency domain so that a block is one
    segment: independent complex Gaussian coefficients per channel whose variance
    follows continuum + lines, then an inverse real transform (generator only).
    The returned blocks are not normalised."""
    nb = n_fft // 2 + 1
    ch = n_fft // 2  # channel count used for placing the lines
    g1 = line_peak * _gauss_profile(nb, ch * 0.25, fwhm)
    g2 = line_peak * _gauss_profile(nb, ch * 0.50, fwhm)
    g3 = line_peak * _gauss_profile(nb, ch * 0.75, fwhm)

    def cg(scale):
        return (rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) * np.sqrt(scale / 2.0)

    chi = np.deg2rad(chi_deg)
    # continuum + unpolarised line 1: independent in X and Y
    fx = cg(1.0 + g1)
    fy = cg(1.0 + g1)
    # line 2: one common signal, projected on X and Y at angle chi (linear polarisation)
    s2 = cg(g2)
    fx += np.cos(chi) * s2
    fy += np.sin(chi) * s2
    # line 3: common signal, Y lagging X by 90 degrees (circular polarisation)
    s3 = cg(g3)
    fx += s3
    fy += s3 * np.exp(-0.5j * np.pi)
    fx[0] = fx[0].real
    fy[0] = fy[0].real
    fx[-1] = fx[-1].real
    fy[-1] = fy[-1].real
    # inverse real transform; the caller normalises the stream to unit variance
    return np.fft.irfft(fx, n_fft), np.fft.irfft(fy, n_fft)


def config_paper(seed: int = 1256, n_segments: int = 61, n_fft: int = 131072, n_if: int = 4, bits: int = 2):
    """Paper-shaped workload: n_if IF streams of n_segments * n_fft samples
    (default 4 x 61 x 131072 = one 1-s integration at 8 Msps), each pair of IFs
    (i, i + n_if/2) carrying the three-line spectrum.  Returns (list of packed
    uint32 arrays, dict of parameters)."""
    rng = np.random.default_rng(seed)
    h = n_if // 2
    streams = [[] for _ in range(n_if)]
    for _ in range(n_segments):
        for p in range(h):
            x, y = paper_block(rng, n_fft)
            streams[p].append(x)
            streams[p + h].append(y)
    packed = []
    for s in streams:
        v = np.concatenate(s)
        sd = v.std()
        packed.append(pack(quantize(v / sd, bits), bits))
    return packed, dict(bits=bits, n_fft=n_fft, n_samples=n_segments * n_fft, window="rect")


def config_circular(seed: int = 1412, n_fft: int = 16384, n_segments: int = 256, q: float = 0.3, u: float = -0.2,
                    v: float = 0.1, line_peak: float = 3.0, center: float = 3000.0, fwhm: float = 200.0,
                    sigma: float = 20.0):
    """Two circular-feed IFs (R, L) as packed int8 streams: unpolarised noise plus a line
    with fractional Stokes (q, u, v), synthesised per segment in the frequency domain
    (generator only) from two independent complex Gaussian series S1, S2 per channel:
    R = a S1, L = b S1 + c S2 with a = sqrt(1 + v), b = (q - iu) / a and
    |c|^2 = 1 - v - |b|^2, so that <|R|^2> = 1 + v, <|L|^2> = 1 - v, <R conj L> = q + iu
    per unit of line power.  Needs q^2 + u^2 + v^2 <= 1.
    Returns (list of 2 packed uint32 arrays, dict of parameters)."""
    if q * q + u * u + v * v > 1.0:
        raise ValueError("fractional polarisation above 1")
    rng = np.random.default_rng(seed)
    nb = n_fft // 2 + 1
    prof = line_peak * _gauss_profile(nb, center, fwhm)
    a = np.sqrt(1.0 + v)
    b = (q - 1j * u) / a
    c = np.sqrt(max(0.0, 1.0 - v - abs(b) ** 2))

    def cg(scale):
        return (rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) * np.sqrt(scale / 2.0)

    rs, ls = [], []
    for _ in range(n_segments):
        s1, s2 = cg(prof), cg(prof)
        fr = cg(1.0) + a * s1
        fl = cg(1.0) + b * s1 + c * s2
        for f in (fr, fl):
            f[0] = f[0].real
            f[-1] = f[-1].real
        rs.append(np.fft.irfft(fr, n_fft))
        ls.append(np.fft.irfft(fl, n_fft))
    # one scale for both streams: separate normalisations would unbalance the continuum
    xr, xl = np.concatenate(rs), np.concatenate(ls)
    scale = sigma / np.sqrt(0.5 * (xr.var() + xl.var()))
    packed = [pack(quantize_int8(x * scale), 8) for x in (xr, xl)]
    return packed, dict(bits=8, n_fft=n_fft, n_samples=n_segments * n_fft, q=q, u=u, v=v, center=center,
                        fwhm=fwhm, line_peak=line_peak, window="hann")


def config_precision(seed: int = 1256, n_fft: int = 262144, n_segments: int = 610, line_db: float = 40.0,
                     fwhm: float = 20.0, center: float = 40000.0, v_scale: float = 1e-3, sigma: float = 20.0):
    """Two linear-feed IFs (X, Y) as packed int8 streams: unit continuum plus a strong
    Gaussian line (peak 10^(line_db/10) times the continuum) whose Stokes V is
    v_scale * dI/dnu (a Zeeman-like antisymmetric profile, one channel as the unit), made
    per segment in the frequency domain (generator only): the line's X and Y parts are
    X = S1, Y = -i v S1 + sqrt(1 - v^2) S2 with v = V / I_line per channel, so that
    <|X|^2> = <|Y|^2> = I_line and <X conj Y> = i v I_line.
    Returns (list of 2 packed uint32 arrays, dict of parameters)."""
    rng = np.random.default_rng(seed)
    nb = n_fft // 2 + 1
    k = np.arange(nb, dtype=np.float64)
    sd = fwhm / (2.0 * np.sqrt(2.0 * np.log(2.0)))
    prof = 10.0 ** (line_db / 10.0) * np.exp(-0.5 * ((k - center) / sd) ** 2)
    v = -v_scale * (k - center) / sd ** 2          # V / I_line of the derivative profile
    v = np.clip(v, -1.0, 1.0)
    c = np.sqrt(1.0 - v * v)

    def cg(scale):
        return (rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) * np.sqrt(scale / 2.0)

    xs, ys = [], []
    for _ in range(n_segments):
        s1, s2 = cg(prof), cg(prof)
        fx = cg(1.0) + s1
        fy = cg(1.0) - 1j * v * s1 + c * s2
        for f in (fx, fy):
            f[0] = f[0].real
            f[-1] = f[-1].real
        xs.append(np.fft.irfft(fx, n_fft))
        ys.append(np.fft.irfft(fy, n_fft))
    xr, yr = np.concatenate(xs), np.concatenate(ys)
    scale = sigma / np.sqrt(0.5 * (xr.var() + yr.var()))
    packed = [pack(quantize_int8(x * scale), 8) for x in (xr, yr)]
    return packed, dict(bits=8, n_fft=n_fft, n_samples=n_segments * n_fft, center=center, fwhm=fwhm,
                        line_db=line_db, v_scale=v_scale, window="hann")
