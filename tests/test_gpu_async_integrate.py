"""spectrometer_integrate_async (readout and host copies queued, no synchronisation) and
the launch-time reuse of encoded tensor maps: two handles fed alternately with equal and
unequal chunks from pinned host memory, every integration checked against the oracle and
against the synchronous path."""
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


def _pinned_out(torch, n_if, n_pair, nb):
    return {"autos": torch.empty((n_if, nb), pin_memory=True),
            "cross": torch.empty((n_pair, nb, 2), pin_memory=True),
            "stokes": torch.empty((n_pair, 4, nb), pin_memory=True)}


def test_async_integrate_two_handles_alternating(env, orc):
    torch, pol = env
    n_if, bits, n_fft = 4, 2, 1 << 17
    pairs = [(0, 2), (1, 3)]
    rng = np.random.default_rng(321)
    chunks = [3, 3, 2, 3, 3]  # segments per feed: equal chunks reuse the encoded maps
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    sps = [pol.Spectrometer(n_if, bits, n_fft), pol.Spectrometer(n_if, bits, n_fft)]
    try:
        for i, c in enumerate(chunks):
            n = c * n_fft
            packed = [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)]
            pinned = [torch.from_numpy(p.view(np.int32)).pin_memory() for p in packed]
            host = [t.numpy().view(np.uint32) for t in pinned]
            sp, st = sps[i % 2], streams[i % 2]
            out = _pinned_out(torch, n_if, len(pairs), n_fft // 2 + 1)
            sp.feed(host, n, on_device=False, stream=st, host_async=(i % 2 == 1))
            nseg = sp.integrate_async(out, stream=st)
            assert nseg == c
            st.synchronize()
            cr = out["cross"].numpy()
            got = {"autos": out["autos"].numpy(), "cross": cr[..., 0] + 1j * cr[..., 1],
                   "stokes": out["stokes"].numpy()}
            ref = orc.spectrometer(packed, bits, n_fft, n)
            assert_close(got, ref, pairs, 1e-5)
            # the synchronous path on the same data agrees (segment ranges are merged into
            # the accumulators with float atomics, so only to rounding)
            sp.feed(host, n, on_device=False, stream=st)
            sync = sp.integrate()
            for k in ("autos", "stokes"):
                np.testing.assert_allclose(sync[k], got[k], rtol=1e-6, atol=1e-6 * np.abs(got[k]).max())
    finally:
        for sp in sps:
            sp.close()


def test_async_integrate_needs_segments(env):
    torch, pol = env
    with pol.Spectrometer(2, 2, 1024) as sp:
        with pytest.raises(pol.PolarisError) as ei:
            sp.integrate_async(_pinned_out(torch, 2, 1, 513))
        assert ei.value.code == pol.ESTATE


@pytest.mark.parametrize("pad_words", [0, 48])
def test_host_feed_from_rows_of_one_array(env, orc, pad_words):
    """IF streams that are rows of one host array (constant stride, with or without padding
    after each row) go over in one pitched copy; uneven feeds keep the carry right."""
    torch, pol = env
    n_if, bits, n_fft, hop = 4, 2, 4096, 2048
    n = n_fft * 9 + 1024
    rng = np.random.default_rng(55 + pad_words)
    packed = [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)]
    words = n * bits // 32
    big = np.zeros((n_if, words + pad_words), np.uint32)
    for i in range(n_if):
        big[i, :words] = packed[i]
    with pol.Spectrometer(n_if, bits, n_fft, hop=hop) as sp:
        pos = 0
        for c in (4096, 20480, n - 24576):
            sp.feed([big[i, pos // 16:(pos + c) // 16] for i in range(n_if)], c)
            pos += c
        got = sp.integrate()
    ref = orc.spectrometer(packed, bits, n_fft, n, hop=hop)
    assert_close(got, ref, [(0, 2), (1, 3)], 1e-5)


def test_feed_mode_is_checked(env):
    torch, pol = env
    import ctypes

    with pol.Spectrometer(2, 2, 1024) as sp:
        words = np.zeros(64, np.uint32)
        arr = (ctypes.c_void_p * 2)(words.ctypes.data, words.ctypes.data)
        rc = pol.load().spectrometer_feed(sp._h, arr, 1024, 3, None)
        assert rc == pol.EINVAL


def test_async_host_feeds_on_many_streams(env, orc):
    """Asynchronous host feeds on several streams: eight integrations of distinct data on four
    handles and four streams, all queued before any is waited for, each against the oracle;
    then the feeds of four of them captured into CUDA graphs (one per handle and stream),
    replayed once and checked again."""
    torch, pol = env
    n_if, bits, n_fft, nseg, H, steps = 4, 2, 1 << 14, 5, 4, 8
    pairs = [(0, 2), (1, 3)]
    n = nseg * n_fft
    rng = np.random.default_rng(99)
    packed = [[synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)] for _ in range(steps)]
    pinned = [[torch.from_numpy(p.view(np.int32)).pin_memory() for p in step] for step in packed]
    host = [[t.numpy().view(np.uint32) for t in step] for step in pinned]
    nb = n_fft // 2 + 1
    outs = [_pinned_out(torch, n_if, len(pairs), nb) for _ in range(steps)]
    streams = [torch.cuda.Stream() for _ in range(H)]
    sps = [pol.Spectrometer(n_if, bits, n_fft) for _ in range(H)]

    def check(i):
        cr = outs[i]["cross"].numpy()
        got = {"autos": outs[i]["autos"].numpy(), "cross": cr[..., 0] + 1j * cr[..., 1],
               "stokes": outs[i]["stokes"].numpy()}
        assert_close(got, orc.spectrometer(packed[i], bits, n_fft, n), pairs, 1e-5)

    try:
        torch.cuda.synchronize()
        for i in range(steps):
            sp, st = sps[i % H], streams[i % H]
            sp.feed(host[i], n, on_device=False, stream=st, host_async=True)
            assert sp.integrate_async(outs[i], stream=st) == nseg
        torch.cuda.synchronize()
        for i in range(steps):
            check(i)
        for o in outs:
            for t in o.values():
                t.fill_(7.0)
        # captured: host-async feeds of the first H steps, one per handle on its own stream
        graphs = []
        for k in range(H):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=streams[k]):
                sps[k].feed(host[k], n, on_device=False, stream=streams[k], host_async=True)
                sps[k].integrate_async(outs[k], stream=streams[k])
            graphs.append(g)
        torch.cuda.synchronize()
        for g in graphs:
            g.replay()
        torch.cuda.synchronize()
        for k in range(H):
            check(k)
    finally:
        for sp in sps:
            sp.close()
