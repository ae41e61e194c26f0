"""GB300-native PolariS spectrometer hot path (arXiv:1412.1256).

``paper_1412_1256_gb300.polaris`` is the thin ctypes binding over the CUDA
library ``libpolaris.so`` (C ABI in ``include/polaris.h``); it is imported
lazily so that the input generator ``paper_1412_1256_gb300.synth`` can be used
without loading CUDA.
"""

__all__ = ["polaris", "synth"]


def __getattr__(name):
    if name in ("polaris", "synth"):
        import importlib

        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
