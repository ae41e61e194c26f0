"""Shared test helpers: error metrics of the GPU path against the FP64 oracle.

Normalisation (Cross, Q, U, V can be ~0, so a plain relative error is ill-posed):
  autos and I : |d| / |ref|
  cross       : |d| / sqrt(A_a A_b)
  Q, U, V     : |d| / I
"""
import numpy as np


def spectra_errors(got, ref, pairs, floor_frac: float = 0.0):
    """Max errors per output family.  floor_frac > 0 replaces each denominator by
    max(denominator, floor_frac * its channel mean) (used by structural tests with
    very few segments, where single channels can be arbitrarily close to zero)."""
    def den(x):
        x = np.abs(np.asarray(x, dtype=np.float64))
        return np.maximum(x, floor_frac * np.mean(x)) if floor_frac > 0 else x

    out = {}
    ra = np.asarray(ref["autos"], np.float64)
    out["autos"] = float(np.max(np.abs(got["autos"] - ra) / den(ra)))
    if len(pairs):
        ex, es = 0.0, 0.0
        for p, (a, b) in enumerate(pairs):
            sc = den(np.sqrt(ra[a] * ra[b]))
            ex = max(ex, float(np.max(np.abs(got["cross"][p] - ref["cross"][p]) / sc)))
            I = den(ref["stokes"][p][0])
            es = max(es, float(np.max(np.abs(got["stokes"][p] - ref["stokes"][p]) / I[None, :])))
        out["cross"] = ex
        out["stokes"] = es
    return out


def assert_close(got, ref, pairs, tol: float, floor_frac: float = 0.0):
    err = spectra_errors(got, ref, pairs, floor_frac)
    bad = {k: v for k, v in err.items() if not v <= tol}
    assert not bad, f"errors above {tol}: {err}"
    return err
