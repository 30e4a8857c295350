"""The autotuner's cache file and key (host logic; no GPU needed).

The key names the device ("nodevice" here), the requested precision and every problem's
dimension, size, slab width and reaction flag.  An entry replaces only the knobs the caller left
automatic; storing a key again replaces its line and keeps the others; lines that do not parse
are skipped.
"""
import numpy as np
import pytest

from paper_2510_25991_gb300 import ddst as D


def _prob(n=64, w=16, dim=2, c=False):
    a = np.ones((n + 1,) * dim)
    return dict(dim=dim, n=n, w=w, a=a, c=a.copy() if c else None)


def test_key_lists_device_precision_and_every_problem_shape():
    k = D.ddst_autotune_key([_prob(), _prob(128, 32, c=True), _prob(32, 8, dim=3)], "auto")
    dev, prec, probs = k.split(";")
    assert dev.startswith("dev=") and prec == "prec=2"
    assert probs == "probs=d2n64w16,d2n128w32c,d3n32w8"
    assert D.ddst_autotune_key(_prob(), "mixed") != D.ddst_autotune_key(_prob(), "auto")


def test_store_then_lookup_applies_only_automatic_knobs(tmp_path):
    path = str(tmp_path / "tune.txt")
    key = D.ddst_autotune_key(_prob(), "auto")
    D.ddst_autotune_store(path, key, precision="mixed_tf32", tensor_cores=1, explicit_S=0,
                          gmres_tol=1e-4, check_every=4, factor_chunks=3, interface_solver=1)
    found, o = D.ddst_autotune_lookup(path, key, precision="auto")
    assert found
    assert (o["precision"], o["tensor_cores"], o["explicit_S"], o["gmres_tol"], o["check_every"],
            o["factor_chunks"], o["interface_solver"]) == ("mixed_tf32", 1, 0, 1e-4, 4, 3, 1)
    # knobs the caller set keep the caller's values
    found, o = D.ddst_autotune_lookup(path, key, precision="mixed", tensor_cores=0, explicit_S=1,
                                      gmres_tol=1e-6, check_every=2, factor_chunks=1,
                                      interface_solver=0)
    assert found
    assert (o["precision"], o["tensor_cores"], o["explicit_S"], o["gmres_tol"], o["check_every"],
            o["factor_chunks"], o["interface_solver"]) == ("mixed", 0, 1, 1e-6, 2, 1, 0)


def test_store_replaces_its_own_line_and_keeps_others(tmp_path):
    path = str(tmp_path / "tune.txt")
    k1 = D.ddst_autotune_key(_prob(), "mixed")
    k2 = D.ddst_autotune_key(_prob(128, 32), "mixed")
    D.ddst_autotune_store(path, k1, gmres_tol=1e-2)
    D.ddst_autotune_store(path, k2, gmres_tol=1e-3)
    D.ddst_autotune_store(path, k1, gmres_tol=1e-4)
    lines = open(path).read().splitlines()
    assert len(lines) == 2 and sum(l.startswith(k1 + "\t") for l in lines) == 1
    assert D.ddst_autotune_lookup(path, k1)[1]["gmres_tol"] == 1e-4
    assert D.ddst_autotune_lookup(path, k2)[1]["gmres_tol"] == 1e-3


def test_missing_file_and_malformed_lines_are_not_entries(tmp_path):
    path = str(tmp_path / "tune.txt")
    key = D.ddst_autotune_key(_prob(), "mixed")
    assert D.ddst_autotune_lookup(path, key) == (False, D.ddst_autotune_lookup(path, key)[1])
    with open(path, "w") as fh:
        fh.write(key + "\tprecision=1 tensor_cores=x explicit_S=-1 gmres_tol=1e-3 check_every=8 "
                 "factor_chunks=0 interface_solver=0\n")
        fh.write(key + "\tprecision=9 tensor_cores=1 explicit_S=-1 gmres_tol=1e-3 check_every=8 "
                 "factor_chunks=0 interface_solver=0\n")
        fh.write(key + "\tgmres_tol=1e-3\n")
        fh.write("no tab here\n")
    found, o = D.ddst_autotune_lookup(path, key)
    assert not found and o["gmres_tol"] == 0.0


def test_unwritable_cache_is_an_argument_error(tmp_path):
    key = D.ddst_autotune_key(_prob(), "mixed")
    with pytest.raises(D.DDSTError) as e:
        D.ddst_autotune_store(str(tmp_path / "missing_dir" / "tune.txt"), key)
    assert e.value.name == "INVALID_ARG"
