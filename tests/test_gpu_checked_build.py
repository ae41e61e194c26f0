"""The bounds-checked build (-DPOLARIS_CHECK): every global-memory index of the spectrometer
kernels that the hardware does not check is tested against its buffer's extent, and a bad
one is recorded in the device status word instead of being used.  Parity cases covering the
paths of the hot kernels (unstaged and staged phase 1, TMA and scattered slab stores, the
carry staging of ragged feeds, accumulator copies, code statistics, the allocation-free
entry point) run through that build against the FP64 oracle with no check firing; a test
hook that understates the slab's extent then shows that the checks are live (POLARIS_EBOUNDS,
no access outside a buffer, the context still usable).

The checked library is loaded in a child process (POLARIS_LIB), so that this process keeps
the normal build."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent('''
    import sys
    import numpy as np
    sys.path.insert(0, ROOT)
    import oracle
    from paper_1412_1256_gb300 import polaris, synth
    from tests.helpers import assert_close
    lib = polaris.load()
    assert lib.polaris_checked_build() == 1
    oracle.build()

    def streams(seed, n_if, n, bits):
        rng = np.random.default_rng(seed)
        return [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(n_if)]

    def run(packed, bits, n_fft, n, chunks=None, **kw):
        with polaris.Spectrometer(len(packed), bits, n_fft, **kw) as sp:
            if chunks is None:
                sp.feed(packed, n)
            else:
                spw, pos = 32 // bits, 0
                for c in chunks:
                    sp.feed([p[pos // spw:(pos + c) // spw] for p in packed], c)
                    pos += c
            return sp.integrate()

    cases = [  # (n_if, bits, logn, nseg, kwargs)
        (4, 2, 10, 200, {}),                                # unstaged phase 1, accumulator copies
        (3, 4, 13, 4, dict(window="hann", pairs=[(0, 1)])),  # staged, TMA input and output
        (4, 2, 17, 3, {}),                                  # the paper-shaped size
        (2, 8, 18, 2, dict(accum_fp64=True)),               # joint output block
        (2, 1, 19, 2, {}),                                  # unstaged large N
        (4, 2, 12, 40, dict(max_batch_segments=7)),         # several passes, two slab halves
    ]
    for i, (n_if, bits, logn, nseg, kw) in enumerate(cases):
        n_fft = 1 << logn
        n = n_fft * nseg
        packed = streams(10 + i, n_if, n, bits)
        got = run(packed, bits, n_fft, n, **kw)
        kind = 1 if kw.get("window") == "hann" else 0
        ref = oracle.spectrometer(packed, bits, n_fft, n, window_kind=kind, pairs=kw.get("pairs"))
        pairs = kw.get("pairs") or oracle.default_pairs(n_if)
        assert_close(got, ref, pairs, 1e-5)
    # ragged feeds with 50% overlap (carried samples staged), code statistics on
    n_fft, bits = 4096, 2
    n = 4096 * 9 + 512
    packed = streams(77, 4, n, bits)
    chunks = [1024, 4096, 16, 7168, 4096 * 5, n - (1024 + 4096 + 16 + 7168 + 4096 * 5)]
    with polaris.Spectrometer(4, bits, n_fft, hop=2048, code_stats=True) as sp:
        spw, pos = 32 // bits, 0
        for c in chunks:
            sp.feed([p[pos // spw:(pos + c) // spw] for p in packed], c)
            pos += c
        got = sp.integrate()
        hist = sp.code_histogram()
    ref = oracle.spectrometer(packed, bits, n_fft, n, hop=2048)
    assert_close(got, ref, [(0, 2), (1, 3)], 1e-5)
    assert int(hist.sum()) == 4 * n_fft * got["n_segments"]
    # the allocation-free entry point through the checked kernels
    import torch
    dev = [torch.from_numpy(p.view(np.int32)).cuda() for p in streams(5, 2, 4096 * 12, 8)]
    nb = 4096 // 2 + 1
    a = torch.zeros((2, nb), device="cuda")
    c = torch.zeros((1, nb, 2), device="cuda")
    s = torch.zeros((1, 4, nb), device="cuda")
    assert polaris.run_noalloc(dev, 4096 * 12, 8, 4096, a, c, s) == 12
    torch.cuda.synchronize()
    assert bool(torch.isfinite(a).all()) and bool(torch.isfinite(s).all())
    # the checks are live: with the slab's extent understated they fire, nothing is touched
    # outside a buffer, and the context stays usable
    assert lib.polaris_set_check_understate(1) == 0
    packed = streams(3, 2, 4096 * 8, 2)
    try:
        with polaris.Spectrometer(2, 2, 4096) as sp:
            sp.feed(packed, 4096 * 8)
            sp.integrate()
        raise AssertionError("no bounds check fired")
    except polaris.PolarisError as e:
        assert e.code == polaris.EBOUNDS, e
    assert lib.polaris_set_check_understate(0) == 0
    got = run(packed, 2, 4096, 4096 * 8)
    assert_close(got, oracle.spectrometer(packed, 2, 4096, 4096 * 8), [(0, 1)], 1e-5)
    print("CHECKED_OK")
''').replace("ROOT", repr(ROOT))


def test_checked_build_parity_and_live_checks():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1412_1256_gb300 import build

    lib = build.build_checked()
    env = dict(os.environ, POLARIS_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "CHECKED_OK" in r.stdout, (r.stdout[-3000:], r.stderr[-3000:])
