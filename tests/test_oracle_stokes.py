"""Pins of the oracle's Stokes step (Eq. 2, Sec. 2.1) against polarisation closed
forms: fully linearly and circularly polarised tones give Q/I, U/I or V/I of +-1,
a rotated source or parallactic angle rotates Q + iU by e^{2i(chi + psi)}, gains
divide out, circular and linear feeds agree on the same sky signal, and
I^2 >= Q^2 + U^2 + V^2 for any input (Cauchy-Schwarz)."""
import numpy as np
import pytest

N, K0, S = 256, 23, 2


def _tone(amp, phase):
    t = np.arange(N * S, dtype=np.float64)
    return amp * np.cos(2 * np.pi * K0 * t / N + phase)


def _stokes(orc, x, y, feed=0, psi=0.0, ga=1.0, gb=1.0):
    autos, cross, _ = orc.spectra_levels([x, y], N, pairs=[(0, 1)])
    st = orc.stokes(autos[0], autos[1], cross[0], feed=feed, psi=psi, ga=ga, gb=gb)
    return st[:, K0]


def test_linear_x_only_gives_q_plus_one(orc):
    I, Q, U, V = _stokes(orc, _tone(1, 0.3), np.zeros(N * S))
    assert abs(Q / I - 1) < 1e-12 and abs(U / I) < 1e-12 and abs(V / I) < 1e-12


def test_linear_y_only_gives_q_minus_one(orc):
    I, Q, U, V = _stokes(orc, np.zeros(N * S), _tone(1, 0.3))
    assert abs(Q / I + 1) < 1e-12


def test_linear_45_gives_u_plus_one(orc):
    s = _tone(1 / np.sqrt(2), 0.1)
    I, Q, U, V = _stokes(orc, s, s)
    assert abs(U / I - 1) < 1e-12 and abs(Q / I) < 1e-12 and abs(V / I) < 1e-12


@pytest.mark.parametrize("lag,sign", [(np.pi / 2, 1), (-np.pi / 2, -1)])
def test_circular_gives_v_pm_one(orc, lag, sign):
    # Y lagging X by 90 degrees -> V/I = +1 (with the forward e^{-i} transform); leading -> -1
    I, Q, U, V = _stokes(orc, _tone(1, 0.2), _tone(1, 0.2 - lag))
    assert abs(V / I - sign) < 1e-12 and abs(Q / I) < 1e-12 and abs(U / I) < 1e-12


@pytest.mark.parametrize("chi", [0.1, 0.7, 1.3, 2.5])
@pytest.mark.parametrize("psi", [0.0, 0.35, -1.1])
def test_general_angle_and_parallactic_rotation(orc, chi, psi):
    I, Q, U, V = _stokes(orc, _tone(np.cos(chi), 0.5), _tone(np.sin(chi), 0.5), psi=psi)
    assert abs(Q / I - np.cos(2 * (chi + psi))) < 1e-12
    assert abs(U / I - np.sin(2 * (chi + psi))) < 1e-12
    assert abs(V / I) < 1e-12


@pytest.mark.parametrize("chi", [0.2, 1.0])
@pytest.mark.parametrize("psi", [0.0, 0.6])
def test_circular_feeds_agree_with_linear(orc, chi, psi):
    # the same linearly polarised wave seen by circular feeds, R = (X + iY)/sqrt2, L = (X - iY)/sqrt2
    # at positive frequency: R(t) = cos(wt + ph + chi)/sqrt2, L(t) = cos(wt + ph - chi)/sqrt2
    lin = _stokes(orc, _tone(np.cos(chi), 0.5), _tone(np.sin(chi), 0.5), psi=psi)
    r = _tone(1 / np.sqrt(2), 0.5 + chi)
    l = _tone(1 / np.sqrt(2), 0.5 - chi)
    circ = _stokes(orc, r, l, feed=1, psi=psi)
    assert np.allclose(lin, circ, rtol=0, atol=1e-12 * lin[0])


def test_circular_feed_circular_wave(orc):
    # Y lagging X by 90 degrees: R = sqrt2 X, L = 0  -> V/I = +1 on circular feeds too
    I, Q, U, V = _stokes(orc, _tone(np.sqrt(2), 0.3), np.zeros(N * S), feed=1)
    assert abs(V / I - 1) < 1e-12 and abs(Q / I) < 1e-12


def test_gains_divide_out(orc):
    chi = 0.4
    ref = _stokes(orc, _tone(np.cos(chi), 0.5), _tone(np.sin(chi), 0.5))
    # receiver with voltage gains: X scaled by 1.3, Y scaled by 0.7 and delayed by phi
    phi = 0.8
    got = _stokes(orc, _tone(1.3 * np.cos(chi), 0.5), _tone(0.7 * np.sin(chi), 0.5 - phi),
                  ga=1.3, gb=0.7 * np.exp(-1j * phi))
    assert np.allclose(got, ref, rtol=0, atol=1e-12 * ref[0])


def test_polarised_fraction_bounded(orc):
    rng = np.random.default_rng(8)
    x = rng.standard_normal(N * 16)
    y = 0.6 * x + rng.standard_normal(N * 16)
    autos, cross, _ = orc.spectra_levels([x, y], N, pairs=[(0, 1)])
    I, Q, U, V = orc.stokes(autos[0], autos[1], cross[0])
    assert np.all(I ** 2 - Q ** 2 - U ** 2 - V ** 2 >= -1e-9 * I ** 2)
