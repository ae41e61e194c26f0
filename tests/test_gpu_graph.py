"""CUDA-graph capture of the device path: feed (device input) + integrate_device of one or
several spectrometers, captured once and replayed, must give the oracle's spectra on every
replay.  Replays are valid for feeds of whole segments (hop = n_fft, nothing carried): a
handle's host-side state only advances while the graph is being captured."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_1256_gb300 import polaris

    polaris.load()
    return torch, polaris


def _dev_streams(torch, seed, n_if, n, bits):
    rng = np.random.default_rng(seed)
    host = [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)]
    return host, [torch.from_numpy(h.view(np.int32)).cuda() for h in host]


def _check(torch, orc, host, bits, n_fft, n, pairs, outs):
    autos, cross, stokes = (t.cpu().numpy() for t in outs)
    ref = orc.spectrometer(host, bits, n_fft, n, pairs=pairs)
    got = {"autos": autos, "cross": cross[..., 0] + 1j * cross[..., 1], "stokes": stokes,
           "n_segments": ref["n_segments"]}
    from tests.helpers import assert_close
    assert_close(got, ref, pairs, 1e-5)


@pytest.mark.parametrize("logn,bits", [(17, 2), (12, 8)])
def test_graph_replay_single(env, orc, logn, bits):
    torch, pol = env
    n_fft, nseg = 1 << logn, 5 if logn == 17 else 40
    n = n_fft * nseg
    host, dev = _dev_streams(torch, 70 + logn, 2, n, bits)
    nb = n_fft // 2 + 1
    outs = (torch.zeros((2, nb), device="cuda"), torch.zeros((1, nb, 2), device="cuda"),
            torch.zeros((1, 4, nb), device="cuda"))
    stream = torch.cuda.Stream()
    with pol.Spectrometer(2, bits, n_fft) as sp:
        with torch.cuda.stream(stream):  # one ordinary pass first (per-kernel set-up)
            sp.feed(dev, n, on_device=True, stream=stream)
            sp.integrate_device(*outs, stream=stream)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            sp.feed(dev, n, on_device=True, stream=torch.cuda.current_stream())
            sp.integrate_device(*outs, stream=torch.cuda.current_stream())
        for _ in range(3):
            for t in outs:
                t.zero_()
            g.replay()
            torch.cuda.synchronize()
            _check(torch, orc, host, bits, n_fft, n, [(0, 1)], outs)


def test_graph_replay_heterogeneous_batch(env, orc):
    """Several independent 2-IF spectrometers of different sizes and widths in one graph."""
    torch, pol = env
    cfgs = [(12, 2, 24), (14, 8, 6), (16, 2, 3), (17, 8, 2), (13, 4, 10)]
    stream = torch.cuda.Stream()
    items = []
    for i, (logn, bits, nseg) in enumerate(cfgs):
        n_fft = 1 << logn
        n = n_fft * nseg
        host, dev = _dev_streams(torch, 500 + i, 2, n, bits)
        nb = n_fft // 2 + 1
        outs = (torch.zeros((2, nb), device="cuda"), torch.zeros((1, nb, 2), device="cuda"),
                torch.zeros((1, 4, nb), device="cuda"))
        sp = pol.Spectrometer(2, bits, n_fft)
        with torch.cuda.stream(stream):
            sp.feed(dev, n, on_device=True, stream=stream)
            sp.integrate_device(*outs, stream=stream)
        items.append((sp, host, dev, n_fft, n, bits, outs))
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        cs = torch.cuda.current_stream()
        for sp, host, dev, n_fft, n, bits, outs in items:
            sp.feed(dev, n, on_device=True, stream=cs)
            sp.integrate_device(*outs, stream=cs)
    for _ in range(2):
        g.replay()
        torch.cuda.synchronize()
        for sp, host, dev, n_fft, n, bits, outs in items:
            _check(torch, orc, host, bits, n_fft, n, [(0, 1)], outs)
    for it in items:
        it[0].close()
