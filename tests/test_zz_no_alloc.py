"""The allocation-free entry point (spectrometer_run_noalloc) against the existing
handle path (create + feed + integrate_device) on two calls in a row, and against the
FP64 oracle for every window kind, FP64 accumulation and a small N with many segments,
all through the C ABI.  It is for callers that cannot allocate device memory when they
need a spectrum (real-time loops that must not synchronise the device, hosts that own all
device memory): it keeps its scratch in the library's static device array instead.
Collected last on purpose."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth
from tests.helpers import assert_close, spectra_errors

pytestmark = pytest.mark.gpu
TOL = 1e-5  # the tolerance of the parity tests


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_1256_gb300 import polaris

    polaris.load()
    return torch, polaris


def _outputs(torch, n_if, n_pair, nbin):
    dev = torch.device("cuda", 0)
    return (torch.zeros((n_if, nbin), dtype=torch.float32, device=dev),
            torch.zeros((n_pair, nbin, 2), dtype=torch.float32, device=dev),
            torch.zeros((n_pair, 4, nbin), dtype=torch.float32, device=dev))


def _as_result(autos, cross, stokes):
    c = cross.cpu().numpy()
    return {"autos": autos.cpu().numpy(), "cross": c[..., 0] + 1j * c[..., 1], "stokes": stokes.cpu().numpy()}


def test_noalloc_matches_handle_path_two_calls(env):
    torch, polaris = env
    n_if, bits, n_fft, nseg = 4, 2, 131072, 20  # two batches of the static slab
    n = nseg * n_fft
    nbin = n_fft // 2 + 1
    pairs = [(0, 2), (1, 3)]
    stream = torch.cuda.current_stream()
    for call in range(2):
        rng = np.random.default_rng(4242 + call)
        packed = [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)]
        dpk = [torch.from_numpy(p.view(np.int32)).cuda() for p in packed]
        # existing entry point
        a1, c1, s1 = _outputs(torch, n_if, 2, nbin)
        with polaris.Spectrometer(n_if, bits, n_fft) as sp:
            sp.feed(dpk, n, on_device=True, stream=stream)
            assert sp.integrate_device(a1, c1, s1, stream=stream) == nseg
        # allocation-free entry point
        a2, c2, s2 = _outputs(torch, n_if, 2, nbin)
        assert polaris.run_noalloc(dpk, n, bits, n_fft, a2, c2, s2, stream=stream) == nseg
        torch.cuda.synchronize()
        err = spectra_errors(_as_result(a2, c2, s2), _as_result(a1, c1, s1), pairs)
        assert all(v <= TOL for v in err.values()), (call, err)


def test_noalloc_rejects_sizes_beyond_its_array(env):
    torch, polaris = env
    n_fft = 1 << 19
    dpk = [torch.zeros(16, dtype=torch.int32, device="cuda") for _ in range(8)]
    with pytest.raises(polaris.PolarisError) as ei:
        polaris.run_noalloc(dpk, n_fft, 2, n_fft, None, None, None)
    assert ei.value.code == polaris.EINVAL
    assert "static limit" in str(ei.value)


@pytest.mark.parametrize("logn,bits,nseg,window,fp64", [
    (17, 2, 6, "rect", False),
    (14, 8, 10, "hann", False),
    (13, 4, 12, "taps", True),
    (16, 1, 6, "hann", True),
    (10, 2, 600, "rect", False),   # small N, many segments in one pass
    (12, 8, 300, "taps", False),
])
def test_noalloc_matches_oracle(env, orc, logn, bits, nseg, window, fp64):
    torch, polaris = env
    n_fft = 1 << logn
    n = nseg * n_fft
    nbin = n_fft // 2 + 1
    rng = np.random.default_rng(700 + logn + bits)
    packed = [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(4)]
    dpk = [torch.from_numpy(p.view(np.int32)).cuda() for p in packed]
    taps = rng.uniform(0.2, 1.0, n_fft).astype(np.float32) if window == "taps" else None
    a, c, s = _outputs(torch, 4, 2, nbin)
    assert polaris.run_noalloc(dpk, n, bits, n_fft, a, c, s, window=taps if taps is not None else window,
                               accum_fp64=fp64) == nseg
    torch.cuda.synchronize()
    kind = {"rect": 0, "hann": 1, "taps": 2}[window]
    ref = orc.spectrometer(packed, bits, n_fft, n, window_kind=kind, taps=taps)
    assert_close(_as_result(a, c, s), ref, [(0, 2), (1, 3)], TOL)


def test_rejected_arguments_queue_nothing(env, orc):
    """A bad feed type or a zero gain is rejected before anything is queued: the outputs
    keep their contents, and the next valid call still matches the oracle."""
    torch, polaris = env
    n_fft, bits, nseg = 4096, 2, 8
    n = nseg * n_fft
    nbin = n_fft // 2 + 1
    rng = np.random.default_rng(99)
    packed = [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(2)]
    dpk = [torch.from_numpy(p.view(np.int32)).cuda() for p in packed]
    a, c, s = (t.fill_(7.0) for t in _outputs(torch, 2, 1, nbin))
    torch.cuda.synchronize()
    for kw in (dict(feed=5), dict(gains=[(0.0, 1.0)]), dict(gains=[(1.0, 0.0)])):
        with pytest.raises(polaris.PolarisError) as ei:
            polaris.run_noalloc(dpk, n, bits, n_fft, a, c, s, **kw)
        assert ei.value.code == polaris.EINVAL
        torch.cuda.synchronize()
        for t in (a, c, s):
            assert bool((t == 7.0).all())
    gains = [(1.1 - 0.2j, 0.9 + 0.05j)]
    assert polaris.run_noalloc(dpk, n, bits, n_fft, a, c, s, feed=polaris.FEED_CIRCULAR, psi=0.4, gains=gains) == nseg
    torch.cuda.synchronize()
    ref = orc.spectrometer(packed, bits, n_fft, n, feed=1, psi=0.4, gains=gains)
    assert_close(_as_result(a, c, s), ref, [(0, 1)], TOL)
