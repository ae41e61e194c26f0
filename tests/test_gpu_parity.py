"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bar: unpacking bit-exact; spectra and Stokes within 1e-5 max relative error per
channel (normalisation in tests/helpers.py) for the FP32 path.
"""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth
from tests.helpers import assert_close

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def pol():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_1256_gb300 import polaris

    polaris.load()
    return polaris


def _run(pol, packed, bits, n_fft, n, hop=0, window="rect", pairs=None, chunks=None, **kw):
    n_if = len(packed)
    with pol.Spectrometer(n_if, bits, n_fft, hop=hop, window=window, pairs=pairs, **kw) as sp:
        if chunks is None:
            sp.feed(packed, n)
        else:
            spw = 32 // bits
            pos = 0
            for c in chunks:
                w0, w1 = pos // spw, (pos + c) // spw
                sp.feed([p[w0:w1] for p in packed], c)
                pos += c
        return sp.integrate()


def _oracle(orc, packed, bits, n_fft, n, hop=None, window_kind=0, taps=None, pairs=None):
    return orc.spectrometer(packed, bits, n_fft, n, hop=hop, window_kind=window_kind, taps=taps, pairs=pairs)


def _random_streams(seed, n_if, n, bits):
    rng = np.random.default_rng(seed)
    return [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)]


def test_tiny_config_hann_int8(pol, orc):
    packed, meta = synth.config_tiny()
    n = meta["n_samples"]
    got = _run(pol, packed, 8, 1024, n, window="hann")
    ref = _oracle(orc, packed, 8, 1024, n, window_kind=1)
    assert got["n_segments"] == ref["n_segments"] == 64
    assert_close(got, ref, [(0, 1)], TOL)


@pytest.mark.parametrize("logn", list(range(4, 19)))
def test_sizes_two_pairs_2bit(pol, orc, logn):
    n_fft = 1 << logn
    nseg = 8 if logn >= 15 else 24
    n = nseg * n_fft
    packed = _random_streams(logn, 4, n, 2)
    got = _run(pol, packed, 2, n_fft, n)
    ref = _oracle(orc, packed, 2, n_fft, n)
    assert got["n_segments"] == nseg
    assert_close(got, ref, [(0, 2), (1, 3)], TOL)


@pytest.mark.parametrize("bits", [1, 2, 4, 8])
def test_bits(pol, orc, bits):
    n_fft, nseg = 4096, 16
    n = n_fft * nseg
    packed = _random_streams(100 + bits, 2, n, bits)
    got = _run(pol, packed, bits, n_fft, n)
    ref = _oracle(orc, packed, bits, n_fft, n)
    assert_close(got, ref, [(0, 1)], TOL)


@pytest.mark.parametrize("logn", [13, 14, 15, 16, 17, 18, 19, 20])
@pytest.mark.parametrize("bits", [1, 2, 4, 8])
def test_staged_sizes_every_width(pol, orc, logn, bits):
    """Every (size, sample width) of the shared-memory-staged phase 1: tile widths, stage
    buffers and the TMA/scattered output paths differ per pair.  Three IFs, so one FFT pair
    has no IF b; the window alternates between rect and Hann."""
    n_fft, nseg = 1 << logn, 3
    n = n_fft * nseg
    packed = _random_streams(1000 + 10 * logn + bits, 3, n, bits)
    hann = (logn + bits) % 2 == 1
    got = _run(pol, packed, bits, n_fft, n, window="hann" if hann else "rect", pairs=[(0, 1)])
    ref = _oracle(orc, packed, bits, n_fft, n, window_kind=1 if hann else 0, pairs=[(0, 1)])
    assert got["n_segments"] == nseg
    assert_close(got, ref, [(0, 1)], TOL)


@pytest.mark.parametrize("logn,fp64", [(10, False), (11, False), (12, True), (13, False)])
def test_small_n_accumulator_copies_two_integrations(pol, orc, logn, fp64):
    """Small N, where a pass gives each warp a range of a few segments and the ranges of a
    (pair, unit group) add into several accumulator copies that the readout sums: two
    integrations in a row on one handle (the second must not see the first's sums), enough
    segments for many ranges per group, FP32 and FP64 accumulation."""
    n_fft, bits, nseg = 1 << logn, 2, 600 if logn <= 11 else 160
    n = n_fft * nseg
    with pol.Spectrometer(4, bits, n_fft, accum_fp64=fp64) as sp:
        for k in range(2):
            packed = _random_streams(3000 + 10 * logn + k, 4, n, bits)
            sp.feed(packed, n)
            got = sp.integrate()
            ref = _oracle(orc, packed, bits, n_fft, n)
            assert got["n_segments"] == nseg
            assert_close(got, ref, [(0, 2), (1, 3)], TOL)


def test_paper_config_one_integration(pol, orc):
    """4 IFs, 2-bit, N = 131072, 61 segments (one 1-s integration), three-line spectrum."""
    packed, meta = synth.config_paper(n_segments=61)
    n = meta["n_samples"]
    got = _run(pol, packed, 2, 131072, n)
    ref = _oracle(orc, packed, 2, 131072, n)
    assert got["n_segments"] == 61
    assert_close(got, ref, [(0, 2), (1, 3)], TOL)


def test_overlap_and_ragged_feeds(pol, orc):
    """50% overlap (Sec. 3.1) and a stream fed in uneven pieces: carry-over of partial segments."""
    n_fft, bits = 2048, 2
    n = 2048 * 20 + 512
    packed = _random_streams(7, 4, n, bits)
    chunks = [1024, 4096, 16, 7168, 2048 * 5, n - (1024 + 4096 + 16 + 7168 + 2048 * 5)]
    got = _run(pol, packed, bits, n_fft, n, hop=1024, chunks=chunks)
    ref = _oracle(orc, packed, bits, n_fft, n, hop=1024)
    assert got["n_segments"] == ref["n_segments"]
    assert_close(got, ref, [(0, 2), (1, 3)], TOL)


@pytest.mark.parametrize("logn,bits,codes,nseg", [(17, 2, [0, 1, 2, 3], 3), (20, 8, [0x80, 0x7F], 2)])
def test_constant_streams_closed_form(pol, orc, logn, bits, codes, nseg):
    """Degenerate input at the benchmark's transform size (2^17 points, 2-bit, four IFs) and at
    the largest (2^20, 8-bit, the extreme levels -128 and 127): every sample of IF i is the same
    code, i.e. the constant level L_i, fed in two pieces with an empty feed between them.  With
    a rectangular window each segment's spectrum is N L_i at bin 0 and zero elsewhere, so over
    S segments autos[i][0] = S (N L_i)^2 and cross[p][0] = S N^2 L_a L_b (real), every other
    bin vanishes (a transform of a constant meets only exact zeros off bin 0), and the Stokes
    of bin 0 are Eq. (2) of those sums."""
    n_fft = 1 << logn
    n = n_fft * nseg
    packed = [synth.pack(np.full(n, c), bits) for c in codes]
    levels = [float(orc.decode(bits, p[:1], 1)[0]) for p in packed]
    assert levels[0] != levels[-1]
    half = n // 2
    got = _run(pol, packed, bits, n_fft, n, chunks=[half, 0, n - half])
    assert got["n_segments"] == nseg
    for i, L in enumerate(levels):
        a, a0 = got["autos"][i].astype(np.float64), nseg * (n_fft * L) ** 2
        assert abs(a[0] - a0) <= 1e-6 * a0, i
        assert np.abs(a[1:]).max() <= 1e-9 * a0, i
    for p, (ia, ib) in enumerate(orc.default_pairs(len(codes))):
        c = got["cross"][p].astype(np.complex128)
        c0 = nseg * n_fft**2 * levels[ia] * levels[ib]
        assert abs(c[0] - c0) <= 1e-6 * abs(c0), p
        assert np.abs(c[1:]).max() <= 1e-9 * abs(c0), p
        st_ref = orc.stokes(np.array([nseg * (n_fft * levels[ia]) ** 2]), np.array([nseg * (n_fft * levels[ib]) ** 2]),
                            np.array([c0 + 0j]))
        st = got["stokes"][p].astype(np.float64)
        scale = np.abs(st_ref).max()
        assert np.abs(st[:, 0] - st_ref[:, 0]).max() <= 1e-6 * scale, p
        assert np.abs(st[:, 1:]).max() <= 1e-9 * scale, p


def test_custom_taps_fp64_accum(pol, orc):
    n_fft, nseg = 16384, 12
    n = n_fft * nseg
    rng = np.random.default_rng(5)
    taps = rng.uniform(0.2, 1.0, n_fft).astype(np.float32)
    packed = _random_streams(9, 2, n, 8)
    got = _run(pol, packed, 8, n_fft, n, window=taps, accum_fp64=True)
    ref = _oracle(orc, packed, 8, n_fft, n, window_kind=2, taps=taps)
    assert_close(got, ref, [(0, 1)], TOL)


@pytest.mark.parametrize("n_if,pairs", [(1, None), (3, None), (3, [(2, 0)]), (6, None), (8, [(7, 0), (3, 4)])])
def test_if_counts_and_pairs(pol, orc, n_if, pairs):
    n_fft, nseg = 1024, 20
    n = n_fft * nseg
    packed = _random_streams(11 + n_if, n_if, n, 4)
    got = _run(pol, packed, 4, n_fft, n, pairs=pairs)
    ref = _oracle(orc, packed, 4, n_fft, n, pairs=pairs)
    ps = orc.default_pairs(n_if) if pairs is None else pairs
    assert_close(got, ref, ps, TOL)


@pytest.mark.parametrize("feed,psi", [(0, 0.3), (1, -0.7)])
def test_stokes_params(pol, orc, feed, psi):
    packed, meta = synth.config_tiny()
    n = meta["n_samples"]
    gains = [(1.2 - 0.3j, 0.8 + 0.1j)]
    with pol.Spectrometer(2, 8, 1024, window="hann") as sp:
        sp.feed(packed, n)
        got = sp.integrate(feed=feed, psi=psi, gains=gains)
    ref = orc.spectrometer(packed, 8, 1024, n, window_kind=1, feed=feed, psi=psi, gains=gains)
    assert_close(got, ref, [(0, 1)], TOL)


@pytest.mark.parametrize("bits", [1, 2, 4, 8])
def test_unpack_bit_exact_every_code(pol, orc, bits):
    rng = np.random.default_rng(bits)
    spw = 32 // bits
    codes = np.concatenate([np.tile(np.arange(1 << bits), max(1, 64 // (1 << bits))),
                            synth.random_codes(rng, 4096, bits)])
    codes = codes[: len(codes) - len(codes) % spw]
    words = synth.pack(codes, bits)
    with pol.Spectrometer(1, bits, 1024) as sp:
        got = sp.debug_unpack(words, len(codes))
    ref = orc.decode(bits, words, len(codes))
    assert np.array_equal(got.astype(np.float64), ref)


def _every_code_at_every_slot(n, bits):
    """Codes with every value at every sample slot of a word: sample j of word w carries
    (j + w (32/b + 1)) mod 2^b, and 32/b + 1 is odd, so w runs through all codes per slot."""
    spw = 32 // bits
    idx = np.arange(n, dtype=np.int64)
    return ((idx % spw + (idx // spw) * (spw + 1)) % (1 << bits)).astype(np.uint8)


@pytest.mark.parametrize("logn", [13, 14, 15, 16, 17, 18, 19, 20])
@pytest.mark.parametrize("bits", [1, 2, 4, 8])
def test_staged_decoder_bit_exact(pol, orc, logn, bits):
    """From N = 2^13 up the FFT kernel decodes from a shared-memory stage with a rotation per
    column and both IFs in one packed subtraction.  Through that device code (both stage
    layouts, pairs with and without an IF b), every code at every rotation of the tile loop
    decodes to exactly the oracle's level.  (1-bit at 2^19 and 2^20 is not staged: there the
    kernel decodes per lane as spectrometer_debug_unpack, checked above.)"""
    n_fft = 1 << logn
    n = 2 * n_fft  # one segment of every code at every slot, one of random codes
    rng = np.random.default_rng(50 + 10 * logn + bits)
    ca = np.concatenate([_every_code_at_every_slot(n_fft, bits), synth.random_codes(rng, n_fft, bits)])
    cb = np.concatenate([synth.random_codes(rng, n_fft, bits), _every_code_at_every_slot(n_fft, bits)[::-1]])
    wa, wb = synth.pack(ca, bits), synth.pack(cb, bits)
    ref_a, ref_b = orc.decode(bits, wa, n), orc.decode(bits, wb, n)
    with pol.Spectrometer(2, bits, n_fft) as sp:
        if bits == 1 and logn >= 19:
            with pytest.raises(pol.PolarisError) as ei:
                sp.debug_unpack_staged(wa, wb, n)
            assert ei.value.code == pol.EINVAL
            return
        for layout in (0, 1):
            ga, gb = sp.debug_unpack_staged(wa, wb, n, layout)
            assert np.array_equal(ga.astype(np.float64), ref_a), (layout, "IF a")
            assert np.array_equal(gb.astype(np.float64), ref_b), (layout, "IF b")
            ga1, _ = sp.debug_unpack_staged(wa, None, n, layout)
            assert np.array_equal(ga1.astype(np.float64), ref_a), (layout, "single IF")


def test_integrate_without_segments_is_state_error(pol):
    with pol.Spectrometer(2, 2, 1024) as sp:
        with pytest.raises(pol.PolarisError) as ei:
            sp.integrate()
        assert ei.value.code == pol.ESTATE
        sp.feed([np.zeros(32, np.uint32)] * 2, 512)  # less than one segment: still nothing
        with pytest.raises(pol.PolarisError):
            sp.integrate()


def test_invalid_configs(pol):
    for kw in [dict(n_if=0, bits=2, n_fft=1024), dict(n_if=2, bits=3, n_fft=1024), dict(n_if=2, bits=2, n_fft=1000),
               dict(n_if=2, bits=2, n_fft=1024, hop=8), dict(n_if=2, bits=2, n_fft=1024, pairs=[(0, 0)]),
               dict(n_if=2, bits=1, n_fft=16), dict(n_if=2, bits=2, n_fft=1 << 21)]:
        with pytest.raises(pol.PolarisError) as ei:
            pol.Spectrometer(**kw)
        assert ei.value.code == pol.EINVAL


def test_alloc_limit_gives_enomem(pol):
    pol.set_alloc_limit(1 << 20)
    try:
        with pytest.raises(pol.PolarisError) as ei:
            pol.Spectrometer(4, 2, 131072)
        assert ei.value.code == pol.ENOMEM
    finally:
        pol.set_alloc_limit(-1)
    with pol.Spectrometer(4, 2, 1024):
        pass


def test_precision_workload_full_size_fp32_path(pol, orc):
    """The precision workload at full size through the FP32 path, as the benchmark times it:
    2 IFs, int8, 262144-point segments, Hann window, 610 segments (10 s at 16 Msps) in one
    feed of device-resident input on one handle.  Like the benchmark's ring, segment s is a
    copy of distinct segment s mod 16, so the expected sums are the oracle's sums over the 16
    distinct segments, each weighted by its number of copies (sums of identical terms, and
    Stokes linear in the sums, with unit gains and psi = 0)."""
    torch = pytest.importorskip("torch")
    packed, cfg = synth.config_precision(seed=1256, n_segments=16)
    n_fft, n_u, nseg = cfg["n_fft"], 16, 610
    wps = n_fft // 4  # int8: four samples per word
    ring = []
    for p in packed:
        big = np.empty(nseg * wps, np.uint32)
        for s in range(nseg):
            u = s % n_u
            big[s * wps:(s + 1) * wps] = p[u * wps:(u + 1) * wps]
        ring.append(torch.from_numpy(big.view(np.int32)).cuda())
    nb = n_fft // 2 + 1
    autos = torch.zeros((2, nb), device="cuda")
    cross = torch.zeros((1, nb, 2), device="cuda")
    stokes = torch.zeros((1, 4, nb), device="cuda")
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    with pol.Spectrometer(2, 8, n_fft, window="hann") as sp:
        sp.feed(ring, nseg * n_fft, on_device=True, stream=st)
        assert sp.integrate_device(autos, cross, stokes, stream=st) == nseg
        st.synchronize()
    ref = {"autos": 0.0, "cross": 0.0, "stokes": 0.0}
    for u in range(n_u):
        w = len(range(u, nseg, n_u))
        r = orc.spectrometer([p[u * wps:(u + 1) * wps] for p in packed], 8, n_fft, n_fft, window_kind=1)
        for key in ref:
            ref[key] = ref[key] + w * np.asarray(r[key])
    c = cross.cpu().numpy()
    got = {"autos": autos.cpu().numpy(), "cross": c[..., 0] + 1j * c[..., 1], "stokes": stokes.cpu().numpy()}
    assert_close(got, ref, [(0, 1)], TOL)
