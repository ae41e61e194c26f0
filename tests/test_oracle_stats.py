"""Statistical pins of the oracle (radiometer analogues of Sec. 3.4 and the
cross-correlation discussion of Sec. 5): for white noise the per-channel relative
spread of the accumulated power falls as 1/sqrt(S), and for independent X, Y the
normalised cross power |rho|^2 averages 1/S (the Rayleigh bias noted in Sec. 5)."""
import numpy as np
import pytest


@pytest.mark.parametrize("S", [4, 16, 64])
def test_radiometer_one_over_sqrt_s(orc, S):
    N = 1024
    rng = np.random.default_rng(S)
    x = rng.standard_normal(N * S)
    autos, _, _ = orc.spectra_levels([x], N)
    P = autos[0][1:-1]  # DC and Nyquist bins are real-valued (different statistics)
    rel_sd = P.std() / P.mean()
    assert abs(rel_sd * np.sqrt(S) - 1.0) < 0.12


@pytest.mark.parametrize("S", [8, 32])
def test_independent_noise_cross_consistent_with_zero(orc, S):
    N = 2048
    rng = np.random.default_rng(100 + S)
    x, y = rng.standard_normal(N * S), rng.standard_normal(N * S)
    autos, cross, _ = orc.spectra_levels([x, y], N, pairs=[(0, 1)])
    rho2 = (np.abs(cross[0]) ** 2 / (autos[0] * autos[1]))[1:-1]
    nch = len(rho2)
    # |rho|^2 ~ Beta(1, S-1): mean 1/S, sd ~ 1/S
    assert abs(rho2.mean() * S - 1.0) < 5.0 / np.sqrt(nch)
