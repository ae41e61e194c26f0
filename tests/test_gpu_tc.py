"""GPU parity of the tensor-core DFT spectrometer (polaris_tc_*) against the FP64 oracle:
radix-64 DFTs as tcgen05 GEMMs with split 16-bit operands (fp16 x3, bf16 x3) and the
plain bf16 product, at 64^2 and 64^3 points, every bit width, several feeds and batches,
and the bounded completion wait.

Error bounds (normalised as in the FP32 parity tests: autos and I by themselves, cross by
sqrt(A_a A_b), Q, U, V by I): a split operand keeps about 22 (fp16) or 17 (bf16)
significant bits and the dropped lo x lo product is of the same order, per radix-64 pass;
two or three passes and FP32 accumulation in tensor memory give ~1e-6 (fp16 x3) and ~1e-5
(bf16 x3) relative errors per bin; one bf16 product keeps 8 bits (~4e-3 per operand).  The
bounds below leave a factor of about 5 over the measured errors."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth
from tests.helpers import spectra_errors

pytestmark = pytest.mark.gpu

TOL = {"fp16x3": 1e-5, "bf16x3": 2e-4, "bf16": 5e-2}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_1256_gb300 import polaris

    polaris.load()
    return torch, polaris


def _dev(torch, packed):
    return [torch.from_numpy(p.view(np.int32)).cuda() for p in packed]


def _as_pair(got):
    return {"autos": got["autos"], "cross": got["cross"][None], "stokes": got["stokes"][None]}


def _noise(seed, n, bits):
    rng = np.random.default_rng(seed)
    if bits == 8:
        return [synth.pack(synth.quantize_int8(rng.standard_normal(n) * 20.0), 8) for _ in range(2)]
    return [synth.pack(synth.quantize(rng.standard_normal(n), bits), bits) for _ in range(2)]


@pytest.mark.parametrize("window", ["rect", "hann"])
def test_all_precisions_at_4096(env, orc, window):
    torch, pol = env
    n_fft, nseg = 4096, 40
    n = n_fft * nseg
    packed = _noise(11, n, 8)
    ref = orc.spectrometer(packed, 8, n_fft, n, window_kind={"rect": 0, "hann": 1}[window], pairs=[(0, 1)])
    dev = _dev(torch, packed)
    errs = {}
    for prec in ("fp16x3", "bf16x3", "bf16"):
        with pol.TensorCoreSpectrometer(8, n_fft, prec, window) as sp:
            sp.feed(dev, n)
            got = sp.integrate()
        assert got["n_segments"] == nseg
        errs[prec] = max(spectra_errors(_as_pair(got), ref, [(0, 1)]).values())
        assert errs[prec] <= TOL[prec], (prec, errs)
    assert errs["fp16x3"] < errs["bf16x3"] < errs["bf16"], errs


@pytest.mark.parametrize("bits", [1, 2, 4])
def test_every_width(env, orc, bits):
    torch, pol = env
    n_fft, nseg = 4096, 24
    n = n_fft * nseg
    packed = _noise(20 + bits, n, bits)
    ref = orc.spectrometer(packed, bits, n_fft, n, pairs=[(0, 1)])
    with pol.TensorCoreSpectrometer(bits, n_fft, "bf16x3") as sp:
        sp.feed(_dev(torch, packed), n)
        got = sp.integrate()
    # 1-bit spectra of 24 segments have near-empty channels: floor the denominators
    err = spectra_errors(_as_pair(got), ref, [(0, 1)], floor_frac=0.05)
    assert max(err.values()) <= TOL["bf16x3"], err


def test_full_size_precision_workload(env, orc):
    """64^3 points: the precision workload (a line 40 dB above the continuum with a 1e-3
    derivative V profile), a few segments, both split precisions against the oracle."""
    torch, pol = env
    packed, cfg = synth.config_precision(n_segments=8)
    n_fft, n = cfg["n_fft"], cfg["n_samples"]
    ref = orc.spectrometer(packed, 8, n_fft, n, window_kind=1, pairs=[(0, 1)])
    dev = _dev(torch, packed)
    for prec in ("fp16x3", "bf16x3"):
        with pol.TensorCoreSpectrometer(8, n_fft, prec, "hann") as sp:
            sp.feed(dev, n)
            got = sp.integrate()
        # 8 segments leave some of the 131073 channels far below their mean power:
        # denominators are floored at 5% of the channel mean
        err = spectra_errors(_as_pair(got), ref, [(0, 1)], floor_frac=0.05)
        assert max(err.values()) <= TOL[prec], (prec, err)


def test_feeds_batches_and_integration_boundary(env, orc):
    """1030 segments (more than one 1024-segment batch at 64^2) in uneven feeds, then a
    second integration that holds only what was fed after the first."""
    torch, pol = env
    n_fft = 4096
    nseg = 1030
    n = n_fft * nseg
    packed = _noise(5, n, 2)
    dev = _dev(torch, packed)
    words = n_fft * 2 // 32
    with pol.TensorCoreSpectrometer(2, n_fft, "fp16x3") as sp:
        pos = 0
        for c in (7, 1000, 23):
            sp.feed([d[pos * words:(pos + c) * words] for d in dev], c * n_fft)
            pos += c
        got = sp.integrate()
        assert got["n_segments"] == nseg
        ref = orc.spectrometer(packed, 2, n_fft, n, pairs=[(0, 1)])
        assert max(spectra_errors(_as_pair(got), ref, [(0, 1)]).values()) <= TOL["fp16x3"]
        sp.feed([d[:5 * words] for d in dev], 5 * n_fft)
        got2 = sp.integrate()
    ref2 = orc.spectrometer([p[:5 * words] for p in packed], 2, n_fft, 5 * n_fft, pairs=[(0, 1)])
    assert got2["n_segments"] == 5
    assert max(spectra_errors(_as_pair(got2), ref2, [(0, 1)]).values()) <= TOL["fp16x3"]


def test_argument_errors(env):
    torch, pol = env
    for args in ((8, 2048), (3, 4096), (8, 4096, 7)):
        with pytest.raises(pol.PolarisError) as ei:
            pol.TensorCoreSpectrometer(*args)
        assert ei.value.code == pol.EINVAL
    with pol.TensorCoreSpectrometer(8, 4096) as sp:
        packed = _dev(torch, _noise(1, 4096 * 2, 8))
        with pytest.raises(pol.PolarisError) as ei:
            sp.feed(packed, 4096 + 100)
        assert ei.value.code == pol.EINVAL


def test_completion_wait_timeout(env, orc):
    """A completion wait forced to run out (limit 0): ETIMEOUT, then ESTATE; the context
    stays usable (no fault, trap or hang: the CTA still waits, bounded, for its products)."""
    torch, pol = env
    n_fft, nseg = 4096, 8
    n = n_fft * nseg
    packed = _noise(9, n, 8)
    dev = _dev(torch, packed)
    with pol.TensorCoreSpectrometer(8, n_fft) as sp:
        sp.set_wait_limit(0)
        sp.feed(dev, n)
        with pytest.raises(pol.PolarisError) as ei:
            sp.integrate()
        assert ei.value.code == pol.ETIMEOUT
        with pytest.raises(pol.PolarisError) as ei:
            sp.feed(dev, n)
        assert ei.value.code == pol.ESTATE
    with pol.TensorCoreSpectrometer(8, n_fft) as sp:
        sp.feed(dev, n)
        got = sp.integrate()
    ref = orc.spectrometer(packed, 8, n_fft, n, pairs=[(0, 1)])
    assert max(spectra_errors(_as_pair(got), ref, [(0, 1)]).values()) <= TOL["bf16x3"]
