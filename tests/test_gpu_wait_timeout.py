"""Bounded device-side waits (phase 2's prefetch barrier, N >= 2^17): forcing every wait to
run out at once must give POLARIS_ETIMEOUT on the host, NaN outputs from the device path,
an unusable handle -- and a GPU context that keeps working for the next handle.  No fault,
trap or hang is involved: the kernel still waits (bounded) for its own copies, releases its
tensor memory and returns."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth
from tests.helpers import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pol():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_1256_gb300 import polaris

    polaris.load()
    return polaris


def _streams(seed, n_if, n, bits=2):
    rng = np.random.default_rng(seed)
    return [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)]


def test_timeout_host_path_then_context_usable(pol, orc):
    n_fft, nseg = 1 << 17, 4
    n = n_fft * nseg
    packed = _streams(31, 2, n)
    pol.set_wait_limit(0)
    try:
        sp = pol.Spectrometer(2, 2, n_fft)
        sp.feed(packed, n)
        with pytest.raises(pol.PolarisError) as ei:
            sp.integrate()
        assert ei.value.code == pol.ETIMEOUT
        with pytest.raises(pol.PolarisError) as ei:
            sp.feed(packed, n)
        assert ei.value.code == pol.ESTATE
        sp.close()
    finally:
        pol.set_wait_limit(-1)
    # the context is intact: a fresh handle gives the oracle's spectra
    with pol.Spectrometer(2, 2, n_fft) as sp:
        sp.feed(packed, n)
        got = sp.integrate()
    ref = orc.spectrometer(packed, 2, n_fft, n)
    assert_close(got, ref, [(0, 1)], 1e-5)


def test_timeout_device_path_gives_nan(pol):
    torch = pytest.importorskip("torch")
    n_fft, nseg = 1 << 17, 3
    n = n_fft * nseg
    packed = [torch.from_numpy(p.view(np.int32)).cuda() for p in _streams(32, 2, n)]
    nb = n_fft // 2 + 1
    autos = torch.zeros((2, nb), dtype=torch.float32, device="cuda")
    cross = torch.zeros((1, nb, 2), dtype=torch.float32, device="cuda")
    stokes = torch.zeros((1, 4, nb), dtype=torch.float32, device="cuda")
    pol.set_wait_limit(0)
    try:
        with pol.Spectrometer(2, 2, n_fft) as sp:
            stream = torch.cuda.current_stream()
            sp.feed(packed, n, on_device=True, stream=stream)
            sp.integrate_device(autos, cross, stokes, stream=stream)
            torch.cuda.synchronize()
            assert torch.isnan(autos).all() and torch.isnan(cross).all() and torch.isnan(stokes).all()
    finally:
        pol.set_wait_limit(-1)
    torch.cuda.synchronize()
