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


def _square(n):
    import numpy as np
    return np.ones((n + 1, n + 1))


@pytest.mark.parametrize("problem,message", [
    (dict(dim=2, n=10, w=3), "n % w == 0"),          # slab width does not divide n
    (dict(dim=2, n=10, w=10), "n/w >= 2"),           # a single slab has no interface
    (dict(dim=4, n=10, w=5), "dim must be 2 or 3"),
    (dict(dim=3, n=256, w=32), "exceeds 8192"),      # block 63 * 255 above the large-block limit
])
def test_setup_rejects_bad_problems_without_gpu(problem, message):
    """Argument checks run on the host before any device work and leave a message."""
    from paper_2510_25991_gb300 import ddst as D
    problem = dict(problem, a=_square(problem["n"]))
    with pytest.raises(D.DDSTError) as e:
        D.ddst_setup_batch([problem])
    assert e.value.name == "INVALID_ARG" and message in str(e.value)


def test_setup_rejects_bad_options_and_lists_without_gpu():
    from paper_2510_25991_gb300 import ddst as D
    ok = dict(dim=2, n=16, w=4, a=_square(16))
    with pytest.raises(D.DDSTError, match="precision must be"):
        D.ddst_setup_batch([ok], D.ddst_options_default(precision=7))
    # explicit transfer operators are formed only for blocks the single-CTA kernels take
    with pytest.raises(D.DDSTError, match="explicit transfer operators need"):
        D.ddst_setup_batch([dict(dim=2, n=512, w=128, a=_square(512))],
                           D.ddst_options_default(explicit_S=1))
    with pytest.raises(D.DDSTError, match="explicit transfer operators need"):
        D.ddst_setup_batch([dict(dim=2, n=160, w=40, a=_square(160))],
                           D.ddst_options_default(precision=0, explicit_S=1))
    with pytest.raises(D.DDSTError, match="a is NULL"):
        D.ddst_setup_batch([dict(ok, a=None)])
    with pytest.raises(D.DDSTError, match="bad problem list"):
        D.ddst_setup_batch([])


def test_null_context_errors_without_gpu():
    """Every entry point answers a NULL context with INVALID_ARG and a message."""
    import numpy as np

    from paper_2510_25991_gb300 import ddst as D
    x = np.zeros(4)
    calls = [lambda: D.ddst_build_transfer(None), lambda: D.ddst_compress(None, 1e-8),
             lambda: D.ddst_solve(None, x, x, x), lambda: D.ddst_solve_adjoint(None, x),
             lambda: D.ddst_interface_trace(None, 0, x), lambda: D.ddst_query(None),
             lambda: D.ddst_get_precision(None)]
    for call in calls:
        # leave a different message first, so a stale one cannot pass
        with pytest.raises(D.DDSTError, match="dim must be 2 or 3"):
            D.ddst_setup_batch([dict(dim=4, n=8, w=4, a=_square(8))])
        with pytest.raises(D.DDSTError) as e:
            call()
        assert e.value.name == "INVALID_ARG" and "NULL" in str(e.value)


def test_context_free_error_message_is_per_thread():
    """ddst_last_error(NULL) holds the calling thread's own last message."""
    import threading

    from paper_2510_25991_gb300 import ddst as D
    from paper_2510_25991_gb300 import _lib as L
    lib = L.load()
    with pytest.raises(D.DDSTError, match="dim must be 2 or 3"):
        D.ddst_setup_batch([dict(dim=4, n=8, w=4, a=_square(8))])
    seen = {}

    def other():
        with pytest.raises(D.DDSTError):
            D.ddst_setup_batch([dict(dim=2, n=10, w=3, a=_square(10))])
        seen["other"] = lib.ddst_last_error(None).decode()

    t = threading.Thread(target=other)
    t.start()
    t.join()
    assert "n % w == 0" in seen["other"]
    assert "dim must be 2 or 3" in lib.ddst_last_error(None).decode()


def test_options_reject_unknown_names_and_precisions():
    from paper_2510_25991_gb300 import ddst as D
    assert D.ddst_options_default(precision="auto").precision == 2
    assert D.ddst_options_default(precision="FP64", leaf_size=64).leaf_size == 64
    with pytest.raises(TypeError, match="unknown option 'leafsize'"):
        D.ddst_options_default(leafsize=64)
    with pytest.raises(ValueError, match="precision must be"):
        D.ddst_options_default(precision="half")


def test_array_sizes_checked_before_the_library_is_called():
    import numpy as np

    from paper_2510_25991_gb300 import ddst as D
    prob = dict(dim=2, n=16)
    D._check_sizes(prob, f=np.zeros((15, 15)), g=np.zeros((17, 17)), u=np.zeros(225), a=None)
    with pytest.raises(ValueError, match="g has 225 entries"):
        D._check_sizes(prob, f=np.zeros((15, 15)), g=np.zeros((15, 15)))
    with pytest.raises(ValueError, match="u has 289 entries"):
        D._check_sizes(dict(dim=2, n=16), u=np.zeros((17, 17)))
    D._check_sizes(dict(dim=3, n=8), f=np.zeros(343), dLdg=np.zeros(729))
