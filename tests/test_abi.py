"""The C ABI library builds, loads without a GPU and exports every entry point
that include/parac.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "parac.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(parac_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_02977_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for fn in ("parac_factor", "parac_pcg", "parac_factor_many", "parac_factor_export", "parac_factor_free"):
        assert fn in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu(lib):
    lib.parac_status_string.restype = ctypes.c_char_p
    for code in range(8):
        assert lib.parac_status_string(code).startswith(b"PARAC_")


def test_binding_names_match_header():
    from paper_2505_02977_gb300 import parac
    assert sorted(parac.EXPORTED) == _declared()
    for n in parac.EXPORTED:
        assert callable(getattr(parac, n))
