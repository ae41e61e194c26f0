"""Pins of the oracle's transform step (the FFT of each segment) against things
other than itself: a brute-force DFT, numpy's FFT, hand-written closed forms,
and Parseval's identity for the one-sided spectrum."""
import numpy as np
import pytest


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
def test_radix2_matches_bruteforce_dft(orc, n):
    rng = np.random.default_rng(100 + n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    a, b = orc.fft(x), orc.dft(x)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.linalg.norm(x) * np.sqrt(n)


@pytest.mark.parametrize("n", [2, 16, 256, 4096, 16384])
def test_radix2_matches_numpy(orc, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.max(np.abs(orc.fft(x) - np.fft.fft(x))) <= 1e-12 * np.linalg.norm(x) * np.sqrt(np.log2(n) + 1)


@pytest.mark.parametrize("n", [3, 5, 12, 64])
def test_bruteforce_dft_matches_numpy(orc, n):
    rng = np.random.default_rng(7 * n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.max(np.abs(orc.dft(x) - np.fft.fft(x))) <= 1e-12 * np.linalg.norm(x) * n


def test_four_point_closed_form(orc):
    # X_k for N = 4 written out: W_4 = -i
    a, b, c, d = 3.0, -1.0, 2.0, 5.0
    want = [a + b + c + d, (a - c) - 1j * (b - d), a - b + c - d, (a - c) + 1j * (b - d)]
    got = orc.fft(np.array([a, b, c, d], dtype=complex))
    assert np.allclose(got, want, rtol=0, atol=1e-14)


def test_forward_sign_convention(orc):
    # forward transform uses e^{-i}: a positive-frequency complex exponential lands in bin +k0
    n, k0 = 64, 5
    x = np.exp(2j * np.pi * k0 * np.arange(n) / n)
    X = orc.fft(x)
    assert abs(X[k0] - n) < 1e-11
    X[k0] = 0
    assert np.max(np.abs(X)) < 1e-11


@pytest.mark.parametrize("kind", [0, 1])
def test_parseval_one_sided(orc, kind):
    n = 512
    rng = np.random.default_rng(3)
    lev = rng.integers(-128, 128, n).astype(np.float64)
    autos, _, nseg = orc.spectra_levels([lev], n, window_kind=kind)
    assert nseg == 1
    w = orc.window(kind, n)
    lhs = np.sum((w * lev) ** 2)
    P = autos[0]
    rhs = (P[0] + P[-1] + 2.0 * np.sum(P[1:-1])) / n
    assert abs(lhs - rhs) <= 1e-11 * lhs
