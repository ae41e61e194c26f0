"""Pins of the oracle's leakage model and its gradient (our model: two circular-feed IFs,
per-IF complex gains, per-bin complex leakage, circular Stokes, quadratic loss).

- With no leakage and unit gains the model's Stokes are the spectrometer's circular-feed
  Stokes (Sec. 2.1 path, pinned elsewhere).
- A target equal to the model's Stokes gives zero loss and zero gradient.
- The analytic gradient matches central finite differences of the loss (h = 1e-3 for the
  window and gains, 1e-4 for the leakage) for window taps, gains and leakage terms."""
import numpy as np
import pytest

from paper_1412_1256_gb300 import synth

N, NSEG, BITS = 64, 6, 8


def _case(seed=5):
    rng = np.random.default_rng(seed)
    n = N * NSEG
    packed = [synth.pack(synth.quantize_int8(rng.standard_normal(n) * 20.0), 8) for _ in range(2)]
    nbin = N // 2 + 1
    w = 0.5 - 0.5 * np.cos(2 * np.pi * np.arange(N) / N) + 0.05 * rng.standard_normal(N)
    mag = rng.uniform(0.8, 1.2, 2)
    ph = rng.uniform(-np.pi, np.pi, 2)
    gains = np.array([mag[0] * np.cos(ph[0]), mag[0] * np.sin(ph[0]), mag[1] * np.cos(ph[1]), mag[1] * np.sin(ph[1])])
    leak = rng.uniform(-0.035, 0.035, (2, nbin, 2))
    return packed, n, w, gains, leak


def test_no_leakage_unit_gain_is_circular_spectrometer(orc):
    packed, n, w, _, leak = _case()
    gains = np.array([1.0, 0.0, 1.0, 0.0])
    st, _ = orc.leak_forward(packed, BITS, N, n, w, gains, np.zeros_like(leak))
    ref = orc.spectrometer(packed, BITS, N, n, window_kind=2, taps=w.astype(np.float32), pairs=[(0, 1)], feed=1)
    # the spectrometer takes float32 taps: compare against the same rounded window
    st32, _ = orc.leak_forward(packed, BITS, N, n, w.astype(np.float32).astype(np.float64), gains, np.zeros_like(leak))
    np.testing.assert_allclose(st32, ref["stokes"][0], rtol=1e-12, atol=1e-9 * np.abs(ref["stokes"][0]).max())
    assert np.abs(st - st32).max() < 1e-3 * np.abs(st).max()


def test_target_at_model_gives_zero_loss_and_gradient(orc):
    packed, n, w, gains, leak = _case(7)
    st, _ = orc.leak_forward(packed, BITS, N, n, w, gains, leak)
    _, loss = orc.leak_forward(packed, BITS, N, n, w, gains, leak, st)
    assert loss == 0.0
    gw, gg, gd = orc.leak_grad(packed, BITS, N, n, w, gains, leak, st)
    assert np.abs(gw).max() == 0.0 and np.abs(gg).max() == 0.0 and np.abs(gd).max() == 0.0


def _fd(f, x, idx, h):
    xp, xm = x.copy(), x.copy()
    xp.flat[idx] += h
    xm.flat[idx] -= h
    return (f(xp) - f(xm)) / (2 * h)


def test_gradient_matches_central_differences(orc):
    packed, n, w, gains, leak = _case(11)
    st, _ = orc.leak_forward(packed, BITS, N, n, w, gains, leak)
    rng = np.random.default_rng(3)
    target = st * 0.9 + rng.standard_normal(st.shape) * 0.05 * np.abs(st).mean()
    gw, gg, gd = orc.leak_grad(packed, BITS, N, n, w, gains, leak, target)

    def loss_w(x):
        return orc.leak_forward(packed, BITS, N, n, x, gains, leak, target)[1]

    def loss_g(x):
        return orc.leak_forward(packed, BITS, N, n, w, x, leak, target)[1]

    def loss_d(x):
        return orc.leak_forward(packed, BITS, N, n, w, gains, x, target)[1]

    for i in [0, 1, 7, 31, 32, 63]:
        assert gw[i] == pytest.approx(_fd(loss_w, w, i, 1e-3), rel=1e-3, abs=1e-6 * np.abs(gw).max())
    for i in range(4):
        assert gg[i] == pytest.approx(_fd(loss_g, gains, i, 1e-3), rel=1e-3, abs=1e-6 * np.abs(gg).max())
    flat = gd.reshape(-1)
    for i in [0, 1, 5, 2 * (N // 2), 2 * (N // 2) + 1, 2 * (N // 2 + 1) + 9, 4 * (N // 2 + 1) - 1]:
        assert flat[i] == pytest.approx(_fd(loss_d, leak, i, 1e-4), rel=1e-3, abs=1e-6 * np.abs(flat).max())


def test_circular_source_carries_its_fractional_stokes(orc):
    """The differentiable workload's generator: with unit gains and no leakage, the line's
    excess over the continuum has Q/I, U/I, V/I equal to the fractions it was built with
    (a check of the input recipe, through the oracle's circular-feed Stokes)."""
    packed, cfg = synth.config_circular(seed=3, n_fft=1024, n_segments=256, center=200.0, fwhm=60.0,
                                        line_peak=4.0)
    n_fft, n = cfg["n_fft"], cfg["n_samples"]
    nb = n_fft // 2 + 1
    st, _ = orc.leak_forward(packed, 8, n_fft, n, np.ones(n_fft), np.array([1.0, 0.0, 1.0, 0.0]),
                             np.zeros((2, nb, 2)))
    on = slice(185, 216)
    off = np.r_[20:120, 300:500]
    excess = st[:, on].sum(1) - st[:, off].mean(1) * (on.stop - on.start)
    frac = excess[1:] / excess[0]
    np.testing.assert_allclose(frac, [cfg["q"], cfg["u"], cfg["v"]], atol=0.02)
    # off the line the source is unpolarised
    assert np.abs(st[1:, off].mean(1)).max() < 0.02 * st[0, off].mean()
