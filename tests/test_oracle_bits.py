"""Pins of the oracle's bit-distribution statistics (Sec. 2: each IF's total power comes
from the histogram of its digitised samples; Sec. 3.2.2 tests that measurement).

The histogram is pinned by hand-packed words and by the segment-overlap count; the power
estimates by closed forms (uniform histograms), the textbook quantile 1/Phi^-1(3/4), an
independent inverse-erfc routine, and sampling statistics of Gaussian inputs."""
import math

import numpy as np
import pytest

from paper_1412_1256_gb300 import synth


def _words(hexes):
    return np.array(hexes, dtype=np.uint32)


@pytest.mark.parametrize("bits,word,expect", [
    # 0xE4 = 11 10 01 00: codes 0, 1, 2, 3 once per byte (LSB first)
    (2, 0xE4E4E4E4, [4, 4, 4, 4]),
    # nibbles 0x0..0x7 once each
    (4, 0x76543210, [1, 1, 1, 1, 1, 1, 1, 1, 0, 0, 0, 0, 0, 0, 0, 0]),
    (1, 0x0000FFFF, [16, 16]),
    (1, 0x80000001, [30, 2]),
])
def test_histogram_hand_packed_word(orc, bits, word, expect):
    spw = 32 // bits
    got = orc.code_histogram([_words([word])], bits, spw, spw)
    assert got.tolist() == [expect]


def test_histogram_int8_bytes(orc):
    w = _words([0x80FF7F00])  # bytes 0x00, 0x7F, 0xFF, 0x80 -> codes 0, 127, 255, 128
    got = orc.code_histogram([w], 8, 4, 4)[0]
    assert got.sum() == 4 and got[0] == got[127] == got[255] == got[128] == 1


def test_histogram_counts_segments_not_stream(orc):
    """hop = N/2: interior samples belong to two segments and count twice; the tail beyond
    the last whole segment counts not at all."""
    bits, N = 2, 32
    rng = np.random.default_rng(3)
    n = 5 * N // 2 + 16                # 2.5 segments of data plus a ragged tail
    n -= n % 16
    codes = rng.integers(0, 4, n)
    w = synth.pack(codes, bits)
    got = orc.code_histogram([w], bits, N, n, hop=N // 2)[0]
    nseg = (n - N) // (N // 2) + 1
    expect = np.zeros(4, np.int64)
    for s in range(nseg):
        expect += np.bincount(codes[s * N // 2: s * N // 2 + N], minlength=4)
    assert got.tolist() == expect.tolist()
    assert got.sum() == nseg * N


@pytest.mark.parametrize("bits,m2", [(1, 1.0), (2, 5.0), (4, 85.0), (8, 5461.5)])
def test_moment2_uniform_histogram(orc, bits, m2):
    # mean of level^2 over all codes: 2-bit (9+1+1+9)/4; 4-bit 2*(1+9+...+225)/16;
    # 8-bit (2*sum_{v<=127} v^2 + 128^2)/256
    got, sig = orc.power(bits, np.full(1 << bits, 7, np.uint64))
    assert got == pytest.approx(m2, rel=1e-15)
    if bits != 2:
        assert math.isnan(sig)


def test_sigma_half_outer_is_inverse_quartile(orc):
    """p_outer = 1/2: erfc(v0/(sigma sqrt2)) = 1/2 gives sigma/v0 = 1/Phi^-1(3/4)."""
    _, sig = orc.power(2, [1, 1, 1, 1])
    assert sig == pytest.approx(1.0 / 0.6744897501960817, rel=1e-14)


@pytest.mark.parametrize("p", [1e-6, 0.01, 0.3173105078629141, 0.9, 0.999999])
def test_sigma_against_independent_erfcinv(orc, p):
    special = pytest.importorskip("scipy.special")
    n = 10 ** 15
    k = int(round(p * n))
    counts = [k // 2, (n - k) // 2, n - k - (n - k) // 2, k - k // 2]
    pe = (counts[0] + counts[3]) / sum(counts)
    _, sig = orc.power(2, counts)
    # near p = 1, erfc^-1(p) ~ (1 - p) sqrt(pi) / 2 inherits the rounding of 1 - p: the
    # attainable relative accuracy is about 1e-16 / (1 - p)
    assert sig == pytest.approx(1.0 / (math.sqrt(2.0) * special.erfcinv(pe)), rel=max(1e-12, 1e-14 / (1.0 - pe)))


def test_sigma_degenerate_is_nan(orc):
    assert math.isnan(orc.power(2, [0, 5, 5, 0])[1])   # no outer codes
    assert math.isnan(orc.power(2, [5, 0, 0, 5])[1])   # only outer codes


@pytest.mark.parametrize("sigma", [0.7, 1.0, 1.6])
def test_sigma_recovers_gaussian_rms(orc, sigma):
    """Quantise N(0, sigma^2) with thresholds +-0.98 (fixed); the outer fraction gives
    sigma / 0.98 within sampling error (about 0.3% at 2^20 samples)."""
    rng = np.random.default_rng(int(sigma * 100))
    v = rng.standard_normal(1 << 20) * sigma
    codes = synth.quantize_2bit(v, sigma=1.0, thr=0.98)
    h = orc.code_histogram([synth.pack(codes, 2)], 2, 1 << 20, 1 << 20)[0]
    _, sig = orc.power(2, h)
    assert sig == pytest.approx(sigma / 0.98, rel=0.01)


def test_int8_moment2_tracks_input_power(orc):
    """8-bit: the mean square level is the input variance plus the 1/12 of rounding."""
    rng = np.random.default_rng(8)
    v = rng.standard_normal(1 << 20) * 20.0
    codes = synth.quantize_int8(v)
    h = orc.code_histogram([synth.pack(codes, 8)], 8, 1 << 20, 1 << 20)[0]
    m2, _ = orc.power(8, h)
    assert m2 == pytest.approx(400.0 + 1.0 / 12.0, rel=0.01)
