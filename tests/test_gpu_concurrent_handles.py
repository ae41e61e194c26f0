"""Independent integrations kept in flight on several spectrometer handles, each on its own
CUDA stream (the pattern bench.py times): interleaved feeds and integrations of distinct
data must each match the oracle, i.e. the handles share no state on the device (slabs,
accumulators, tensor maps) and the per-thread tensor-map cache keeps their maps apart."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth
from tests.helpers import assert_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_1256_gb300 import polaris

    polaris.load()
    return torch, polaris


@pytest.mark.parametrize("logn,nseg,bits", [(17, 3, 2), (12, 40, 8)])
def test_three_handles_three_streams(env, orc, logn, nseg, bits):
    torch, pol = env
    n_fft, n_if, H, steps = 1 << logn, 4, 3, 6
    n = n_fft * nseg
    rng = np.random.default_rng(900 + logn)
    host = [[synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)] for _ in range(steps)]
    dev = [[torch.from_numpy(h.view(np.int32)).cuda() for h in step] for step in host]
    nb = n_fft // 2 + 1
    outs = [(torch.zeros((n_if, nb), device="cuda"), torch.zeros((2, nb, 2), device="cuda"),
             torch.zeros((2, 4, nb), device="cuda")) for _ in range(steps)]
    handles = [pol.Spectrometer(n_if, bits, n_fft) for _ in range(H)]
    streams = [torch.cuda.Stream() for _ in range(H)]
    torch.cuda.synchronize()  # inputs and zeroed outputs (current stream) before the side streams
    try:
        # every step queued before any is waited for: the handles' kernels interleave
        for i in range(steps):
            sp, st = handles[i % H], streams[i % H]
            sp.feed(dev[i], n, on_device=True, stream=st)
            assert sp.integrate_device(*outs[i], stream=st) == nseg
        torch.cuda.synchronize()
        for i in range(steps):
            autos, cross, stokes = (t.cpu().numpy() for t in outs[i])
            ref = orc.spectrometer(host[i], bits, n_fft, n)
            got = {"autos": autos, "cross": cross[..., 0] + 1j * cross[..., 1], "stokes": stokes,
                   "n_segments": ref["n_segments"]}
            assert_close(got, ref, [(0, 2), (1, 3)], 1e-5)
    finally:
        for sp in handles:
            sp.close()


def test_benchmark_launch_configuration_full_size(env, orc):
    """The launch configuration bench.py times, at the full paper-shaped size: 4 IFs, 2-bit,
    131072-point segments, 61 per integration (one 1-s integration of the three-line
    spectrum), device-resident input, three handles on three streams with phase 1 capped at
    bench.DEFAULT_CAPS, four integrations in flight before any is read, every one against
    the oracle."""
    torch, pol = env
    import bench

    caps = tuple(int(x) for x in bench.DEFAULT_CAPS.split(","))
    n_fft, n_if, H, steps, nseg = 131072, 4, 3, 4, 61
    host = [synth.config_paper(seed=1256 + 7 * i, n_segments=nseg)[0] for i in range(steps)]
    n = nseg * n_fft
    dev = [[torch.from_numpy(h.view(np.int32)).cuda() for h in step] for step in host]
    nb = n_fft // 2 + 1
    outs = [(torch.zeros((n_if, nb), device="cuda"), torch.zeros((2, nb, 2), device="cuda"),
             torch.zeros((2, 4, nb), device="cuda")) for _ in range(steps)]
    handles = [pol.Spectrometer(n_if, 2, n_fft) for _ in range(H)]
    for sp in handles:
        sp.set_launch_caps(*caps)
    streams = [torch.cuda.Stream() for _ in range(H)]
    torch.cuda.synchronize()
    try:
        for i in range(steps):
            sp, st = handles[i % H], streams[i % H]
            sp.feed(dev[i], n, on_device=True, stream=st)
            assert sp.integrate_device(*outs[i], stream=st) == nseg
        torch.cuda.synchronize()
        for i in range(steps):
            autos, cross, stokes = (t.cpu().numpy() for t in outs[i])
            ref = orc.spectrometer(host[i], 2, n_fft, n)
            got = {"autos": autos, "cross": cross[..., 0] + 1j * cross[..., 1], "stokes": stokes,
                   "n_segments": ref["n_segments"]}
            assert_close(got, ref, [(0, 2), (1, 3)], 1e-5)
    finally:
        for sp in handles:
            sp.close()
