"""Launch choices on the GPU: a handle created with max_batch_segments = 0 uses the tuned
table's entry for its size and width (else the built-in rule), and the spectra do not depend
on the choice: segments per pass and CTA-per-SM caps against the FP64 oracle."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth, tune
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


def test_handles_use_the_tuned_table(pol):
    entries = {(l, b): (m, c1, c2) for (l, b, m, c1, c2) in tune.parse_header(open(tune.HEADER).read())}
    for logn in (10, 13, 17, 20):
        for bits in (2, 8):
            with pol.Spectrometer(2, bits, 1 << logn) as sp:
                got = sp.launch_choices()
            e = entries.get((logn, bits))
            if e is not None:
                if e[0] > 0:
                    assert got["max_batch_segments"] == e[0]
                assert (got["phase1_ctas_per_sm"], got["phase2_ctas_per_sm"]) == (e[1], e[2])
            else:
                assert (got["phase1_ctas_per_sm"], got["phase2_ctas_per_sm"]) == (0, 0)
            with pol.Spectrometer(2, bits, 1 << logn, max_batch_segments=7) as sp:
                assert sp.launch_choices() == {"max_batch_segments": 7, "phase1_ctas_per_sm": 0,
                                               "phase2_ctas_per_sm": 0}


@pytest.mark.parametrize("logn,bits,nseg,batch,caps", [
    (11, 2, 300, 0, (1, 1)),
    (14, 8, 40, 16, (1, 0)),
    (17, 2, 6, 0, (0, 1)),
    (19, 2, 3, 2, (1, 1)),
])
def test_spectra_do_not_depend_on_launch_choices(pol, orc, logn, bits, nseg, batch, caps):
    n_fft = 1 << logn
    n = nseg * n_fft
    rng = np.random.default_rng(31 + logn)
    packed = [synth.pack(synth.random_codes(rng, n, bits), bits) for _ in range(4)]
    with pol.Spectrometer(4, bits, n_fft, max_batch_segments=batch) as sp:
        sp.set_launch_caps(*caps)
        sp.feed(packed, n)
        got = sp.integrate()
    ref = orc.spectrometer(packed, bits, n_fft, n)
    assert got["n_segments"] == nseg
    assert_close(got, ref, [(0, 2), (1, 3)], 1e-5)
    with pol.Spectrometer(2, bits, n_fft) as sp:
        with pytest.raises(pol.PolarisError) as ei:
            sp.set_launch_caps(-1, 0)
        assert ei.value.code == pol.EINVAL
