"""GPU parity of the bit-distribution statistics (Sec. 2, Sec. 3.2.2): per-IF code
histograms from the CUDA path equal the oracle's exactly (integer counts), over overlapping
segments and ragged feeds; the library's power estimates agree with the oracle's."""
import math

import numpy as np
import pytest

from paper_1412_1256_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pol():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_1256_gb300 import polaris

    polaris.load()
    return polaris


def _streams(seed, n_if, n, bits):
    rng = np.random.default_rng(seed)
    return [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)]


@pytest.mark.parametrize("bits", [1, 2, 4, 8])
@pytest.mark.parametrize("logn", [10, 17])
def test_histogram_bit_exact(pol, orc, bits, logn):
    n_fft = 1 << logn
    nseg = 40 if logn == 10 else 3
    n = n_fft * nseg
    packed = _streams(50 + bits + logn, 3, n, bits)
    with pol.Spectrometer(3, bits, n_fft, pairs=[(0, 1)], code_stats=True) as sp:
        sp.feed(packed, n)
        sp.integrate()
        got = sp.code_histogram()
    ref = orc.code_histogram(packed, bits, n_fft, n)
    assert got.dtype == np.uint64 and got.shape == (3, 1 << bits)
    assert np.array_equal(got, ref)
    assert int(got.sum()) == 3 * nseg * n_fft


def test_histogram_overlap_ragged_feeds_and_reset(pol, orc):
    """50% overlap (samples in two segments count twice) and uneven feeds (segments
    assembled from carried samples); reset starts the next count from zero."""
    bits, n_fft, hop = 2, 4096, 2048
    n = n_fft * 9 + 1024
    packed = _streams(77, 4, n, bits)
    chunks = [1024, 5000 - 5000 % 16, 16, 9000 - 9000 % 16]
    chunks.append(n - sum(chunks))
    with pol.Spectrometer(4, bits, n_fft, hop=hop, code_stats=True) as sp:
        pos = 0
        for c in chunks:
            sp.feed([p[pos // 16:(pos + c) // 16] for p in packed], c)
            pos += c
        got = sp.code_histogram(reset=True)
        again = sp.code_histogram()
    ref = orc.code_histogram(packed, bits, n_fft, n, hop=hop)
    assert np.array_equal(got, ref)
    assert int(again.sum()) == 0


def test_histogram_needs_code_stats(pol):
    with pol.Spectrometer(2, 2, 1024) as sp:
        with pytest.raises(pol.PolarisError) as ei:
            sp.code_histogram()
        assert ei.value.code == pol.ESTATE


@pytest.mark.parametrize("bits", [1, 2, 4, 8])
def test_power_estimates_match_oracle(pol, orc, bits):
    rng = np.random.default_rng(900 + bits)
    v = rng.standard_normal(1 << 18)
    codes = synth.quantize(v, bits, sigma=1.0) if bits != 8 else synth.quantize_int8(v * 20.0)
    packed = [synth.pack(codes, bits)]
    with pol.Spectrometer(1, bits, 1 << 12, code_stats=True) as sp:
        sp.feed(packed, 1 << 18)
        h_gpu = sp.code_histogram()[0]
    # both estimators take the oracle's histogram (an oracle input never comes from the GPU);
    # the GPU's histogram must equal it
    h = orc.code_histogram(packed, bits, 1 << 12, 1 << 18)[0]
    assert np.array_equal(np.asarray(h_gpu, np.uint64), np.asarray(h, np.uint64))
    m2, sg = pol.power_from_histogram(bits, h)
    m2_ref, sg_ref = orc.power(bits, h)
    assert m2 == pytest.approx(m2_ref, rel=1e-13)
    if bits == 2:
        assert sg == pytest.approx(sg_ref, rel=1e-12)
        assert sg == pytest.approx(1.0 / 0.98, rel=0.02)
    else:
        assert math.isnan(sg) and math.isnan(sg_ref)


def test_power_rejects_bad_input(pol):
    with pytest.raises(pol.PolarisError):
        pol.power_from_histogram(3, [1, 2, 3])
    with pytest.raises(pol.PolarisError):
        pol.power_from_histogram(2, [0, 0, 0, 0])
