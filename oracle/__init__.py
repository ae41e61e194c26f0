"""FP64 CPU oracle for the PolariS hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import or call anything here.
The product path (``paper_1412_1256_gb300``) never imports this package, and
this package never imports the product path: they share no code.
"""
from .oracle import (  # noqa: F401
    build,
    decode,
    window,
    dft,
    fft,
    stokes,
    accumulate,
    spectra_levels,
    spectrometer,
    default_pairs,
    code_histogram,
    power,
    leak_forward,
    leak_grad,
)
