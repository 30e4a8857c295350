"""The C-ABI library builds for sm_103a, loads, and exports every symbol of include/*.h."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ddst_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("ddst_setup", "ddst_build_transfer", "ddst_compress", "ddst_solve",
                     "ddst_solve_adjoint", "ddst_destroy", "ddst_last_error"):
        assert required in names


def test_library_builds_loads_and_exports_all_symbols():
    import ctypes

    from paper_2510_25991_gb300 import build as B
    from paper_2510_25991_gb300 import _lib

    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in sorted(_declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a signature for every exported entry point
    assert set(_lib.SIGNATURES) == _declared_symbols()
    _lib.load(path)


def test_options_default_without_gpu():
    from paper_2510_25991_gb300 import ddst as D
    o = D.ddst_options_default()
    assert o.precision == 1 and o.k_max == 64 and o.oversample == 10 and o.leaf_size == 128
    assert o.gmres_tol == 0.0 and o.refine_max >= 1  # automatic inner tolerance
