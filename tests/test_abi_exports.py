"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/polaris.h declares (no compute calls: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "polaris.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b(\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def test_header_declares_the_boundary():
    d = _declared()
    for f in ("spectrometer_create", "spectrometer_feed", "spectrometer_integrate", "spectrometer_destroy"):
        assert f in d


def test_library_exports_every_declared_symbol():
    from paper_1412_1256_gb300 import build, polaris

    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert set(polaris.EXPORTS) == set(_declared())


def test_normal_build_has_no_bounds_checks():
    """The default library is built without -DPOLARIS_CHECK: its check hook refuses."""
    from paper_1412_1256_gb300 import polaris

    lib = polaris.load()
    assert lib.polaris_checked_build() == 0
    assert lib.polaris_set_check_understate(1) == polaris.EINVAL
