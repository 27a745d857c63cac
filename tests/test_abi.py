"""The C-ABI library builds for sm_103a, loads without a GPU and exports
every function that include/*.h declares.  No compute calls here."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(lhmm_\w+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def built_lib():
    from paper_2512_13267_gb300 import build_ext
    return ctypes.CDLL(build_ext.build())


def test_header_declares_entry_points():
    names = _declared()
    assert "lhmm_micro_create" in names and "lhmm_micro_advance" in names


@pytest.mark.parametrize("name", _declared())
def test_symbol_exported(built_lib, name):
    assert hasattr(built_lib, name), name


def test_status_strings_without_gpu(built_lib):
    f = built_lib.lhmm_status_string
    f.restype = ctypes.c_char_p
    f.argtypes = [ctypes.c_int]
    assert f(0) == b"ok"
    assert b"argument" in f(1)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2512_13267_gb300 import lhmm
    monkeypatch.setattr(lhmm, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(lhmm, "_lib", None)
    with pytest.raises(RuntimeError):
        lhmm.lib()
