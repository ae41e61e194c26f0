"""The allocation-free entry point (spectrometer_run_noalloc) against the existing
handle path (create + feed + integrate_device), through the C ABI, on two calls in a
row.  It is for callers that cannot allocate device memory when they need a spectrum
(graph capture, real-time loops, hosts that own all device memory): it keeps its
scratch in the library's static device array instead.  Collected last on purpose."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth
from tests.helpers import spectra_errors

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
