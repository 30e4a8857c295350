"""Static check of the Python files whose GPU paths the CPU suite cannot execute.

Every name a function reads as a global must be defined at module level or be a builtin, so
a misspelt name in the benchmark's timed region or in the binding cannot surface first on a
GPU machine.  Uses only the standard library's symbol tables.
"""
import builtins
import glob
import os
import symtable

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
FILES = ["bench.py", "__graft_entry__.py", "paper_2510_25991_gb300/ddst.py",
         "paper_2510_25991_gb300/_lib.py", "paper_2510_25991_gb300/build.py",
         "oracle/ddst_oracle.py", "ddst_inputs/__init__.py"] + sorted(
    os.path.relpath(f, ROOT) for f in glob.glob(os.path.join(ROOT, "tests", "test_*.py")))


def _undefined_globals(path):
    src = open(path).read()
    top = symtable.symtable(src, path, "exec")
    defined = set(top.get_identifiers())
    bad = set()

    def walk(t):
        for s in t.get_symbols():
            if s.is_global() and s.get_name() not in defined and not hasattr(builtins, s.get_name()):
                bad.add((t.get_name(), s.get_name()))
        for c in t.get_children():
            walk(c)

    walk(top)
    return sorted(bad)


@pytest.mark.parametrize("rel", FILES)
def test_no_undefined_global_names(rel):
    assert _undefined_globals(os.path.join(ROOT, rel)) == []


def test_checker_finds_a_planted_name(tmp_path):
    p = tmp_path / "m.py"
    p.write_text("import os\n\ndef f(x):\n    y = os.sep + x\n    return y + undefined_name\n")
    assert _undefined_globals(str(p)) == [("f", "undefined_name")]
