"""Pins of the oracle's segmentation, window and accumulation steps against
closed forms and the paper's printed resolution function (Sec. 3.1)."""
import os

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def tone(n, k0, amp=1.0, phase=0.0, N=None):
    N = N or n
    t = np.arange(n, dtype=np.float64)
    return amp * np.cos(2 * np.pi * k0 * t / N + phase)


def test_rect_window_bin_centred_tone(orc):
    # rectangular window: a tone at bin k0 gives (A N / 2)^2 per segment in bin k0, zero elsewhere
    N, k0, A, S = 256, 37, 1.5, 3
    autos, _, nseg = orc.spectra_levels([tone(N * S, k0, A, 0.4, N)], N)
    assert nseg == S
    peak = S * (A * N / 2) ** 2
    assert abs(autos[0][k0] - peak) <= 1e-11 * peak
    rest = np.delete(autos[0], k0)
    assert np.max(rest) <= 1e-20 * peak  # round-off only


def test_hann_window_tone_three_bins(orc):
    # periodic Hann = 1/2 - 1/4 e^{+} - 1/4 e^{-}: amplitudes 1/4 (k0) and -1/8 (k0 +- 1) of A N
    N, k0, A = 256, 40, 2.0
    autos, _, _ = orc.spectra_levels([tone(N, k0, A)], N, window_kind=1)
    P = autos[0]
    assert abs(P[k0] - (A * N / 4) ** 2) <= 1e-10 * P[k0]
    for k in (k0 - 1, k0 + 1):
        assert abs(P[k] / P[k0] - 0.25) <= 1e-12
    rest = np.delete(P, [k0 - 1, k0, k0 + 1])
    assert np.max(rest) <= 1e-18 * P[k0]


def test_window_values(orc):
    N = 64
    w = orc.window(1, N)
    assert w[0] == 0.0 and abs(w[N // 2] - 1.0) < 1e-15 and abs(w[N // 4] - 0.5) < 1e-15
    assert np.allclose(w[1:], w[1:][::-1])  # periodic Hann: symmetric about N/2
    taps = np.linspace(0.1, 1.0, N).astype(np.float32)
    assert np.array_equal(orc.window(2, N, taps), taps.astype(np.float64))
    assert np.array_equal(orc.window(0, N), np.ones(N))


def test_four_point_integer_accumulation(orc):
    # N = 4 transforms of integers are Gaussian integers: sums are exact
    rng = np.random.default_rng(4)
    S = 50
    a = rng.integers(-3, 4, 4 * S)
    b = rng.integers(-3, 4, 4 * S)
    autos, cross, nseg = orc.spectra_levels([a.astype(float), b.astype(float)], 4, pairs=[(0, 1)])
    assert nseg == S

    def X(v):  # closed form of the 4-point DFT, bins 0..2
        p, q, r, s = v
        return [complex(p + q + r + s), complex(p - r, -(q - s)), complex(p - q + r - s)]

    wa = np.zeros(3)
    wb = np.zeros(3)
    wc = np.zeros(3, complex)
    for i in range(S):
        xa, xb = X(a[4 * i: 4 * i + 4]), X(b[4 * i: 4 * i + 4])
        for k in range(3):
            wa[k] += abs(xa[k]) ** 2
            wb[k] += abs(xb[k]) ** 2
            wc[k] += xa[k] * np.conj(xb[k])
    assert np.array_equal(autos[0], wa) and np.array_equal(autos[1], wb)
    assert np.array_equal(cross[0], wc)


def test_segmentation_and_hop(orc):
    # a single impulse at t0 contributes a flat |X|^2 = 1 to every segment that contains it
    N, hop, n, t0 = 64, 32, 1000, 100
    lev = np.zeros(n)
    lev[t0] = 1.0
    autos, _, nseg = orc.spectra_levels([lev], N, hop=hop)
    assert nseg == (n - N) // hop + 1
    containing = sum(1 for s in range(nseg) if s * hop <= t0 < s * hop + N)
    assert containing == 2
    assert np.allclose(autos[0], containing, rtol=0, atol=1e-12)


def _golden():
    vals = {}
    for line in open(os.path.join(HERE, "golden", "resolution_fwhm.txt")):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    return vals


def test_resolution_function_fwhm_matches_paper(orc):
    """Sec. 3.1: rectangular window -> sinc^2 response with FWHM 0.886 channel (54.07 Hz)."""
    g = _golden()
    N, k0 = 1024, 200
    deltas = np.linspace(0.0, 0.6, 121)
    resp = []
    for dlt in deltas:
        autos, _, _ = orc.spectra_levels([tone(N, k0 + dlt)], N)
        resp.append(autos[0][k0])
    resp = np.array(resp) / resp[0]
    i = np.nonzero(resp < 0.5)[0][0]
    d_half = deltas[i - 1] + (0.5 - resp[i - 1]) * (deltas[i] - deltas[i - 1]) / (resp[i] - resp[i - 1])
    fwhm = 2 * d_half
    assert abs(fwhm - g["fwhm_channels"]) < 1e-3
    chan_hz = g["bandwidth_hz"] / g["channels"]
    assert abs(fwhm * chan_hz - g["fwhm_hz"]) < 0.1


@pytest.mark.parametrize("bits", [2, 8])
def test_packed_path_equals_levels_path(orc, bits):
    # accumulate(packed) = decode then spectra_levels on the decoded levels
    from paper_1412_1256_gb300 import synth

    rng = np.random.default_rng(bits)
    n, N = 4096, 512
    codes = [synth.random_codes(rng, n, bits) for _ in range(2)]
    packed = [synth.pack(c, bits) for c in codes]
    a1, c1, _ = orc.accumulate(packed, bits, N, n)
    a2, c2, _ = orc.spectra_levels([orc.decode(bits, p, n) for p in packed], N)
    assert np.array_equal(a1, a2) and np.array_equal(c1, c2)
