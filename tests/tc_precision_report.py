"""Per-bin errors of every transform engine against the FP64 oracle on the precision
workload (2 IFs, int8, 262144-point segments, a line 40 dB above the continuum with a
1e-3 dI/dnu V profile, Hann window): the FP32 CUDA-core spectrometer and the tensor-core
DFT spectrometer at fp16 x3, bf16 x3 and bf16.  Test infrastructure (it runs the oracle);
needs a GPU.  Usage: python tests/tc_precision_report.py [n_segments]"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main():
    import torch

    import oracle
    from paper_1412_1256_gb300 import polaris, synth
    from tests.helpers import spectra_errors

    nseg = int(sys.argv[1]) if len(sys.argv) > 1 else 16
    packed, cfg = synth.config_precision(n_segments=nseg)
    n_fft, n = cfg["n_fft"], cfg["n_samples"]
    nb = n_fft // 2 + 1
    oracle.build()
    ref = oracle.spectrometer(packed, 8, n_fft, n, window_kind=1, pairs=[(0, 1)])
    dev = [torch.from_numpy(p.view(np.int32)).cuda() for p in packed]
    line = slice(int(cfg["center"] - 3 * cfg["fwhm"]), int(cfg["center"] + 3 * cfg["fwhm"]))

    def report(got):
        e = spectra_errors(got, ref, [(0, 1)], floor_frac=0.05)
        ra = ref["autos"]
        rel = np.abs(got["autos"] - ra) / np.abs(ra)
        I = ref["stokes"][0][0]
        dv = np.abs(got["stokes"][0][3] - ref["stokes"][0][3]) / I
        return {"max_autos": e["autos"], "max_cross": e["cross"], "max_stokes": e["stokes"],
                "median_autos": float(np.median(rel)), "max_V_over_I_on_line": float(dv[line].max()),
                "ref_max_abs_V_over_I_on_line": float(np.abs(ref["stokes"][0][3][line] / I[line]).max())}

    out = {"n_segments": nseg}
    with polaris.Spectrometer(2, 8, n_fft, window="hann", accum_fp64=True) as sp:
        sp.feed(dev, n, on_device=True)
        g = sp.integrate()
    out["fp32"] = report(g)
    for prec in ("fp16x3", "bf16x3", "bf16"):
        with polaris.TensorCoreSpectrometer(8, n_fft, prec, "hann") as tc:
            tc.feed(dev, n)
            g = tc.integrate()
        out[prec] = report({"autos": g["autos"], "cross": g["cross"][None], "stokes": g["stokes"][None]})
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
