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


def test_pcg_many_argument_checks_without_gpu(lib):
    """parac_pcg_many rejects malformed arguments before touching a device:
    a negative count, null arrays, a null handle (reported per system)."""
    V = ctypes.c_void_p
    lib.parac_pcg_many.argtypes = [ctypes.c_int32, ctypes.POINTER(V), ctypes.POINTER(V), ctypes.POINTER(V),
                                   ctypes.c_double, ctypes.c_int32, V, V]
    lib.parac_pcg_many.restype = ctypes.c_int
    EINVAL = 1
    assert lib.parac_pcg_many(-1, None, None, None, 1e-8, 10, None, None) == EINVAL
    assert lib.parac_pcg_many(2, None, None, None, 1e-8, 10, None, None) == EINVAL
    hs, bs, xs = (V * 1)(), (V * 1)(), (V * 1)()
    it = (ctypes.c_int32 * 1)(-5)
    assert lib.parac_pcg_many(1, hs, bs, xs, 1e-8, 10, ctypes.cast(it, V), None) == EINVAL
    assert it[0] == 0                                   # outputs written for every system
    assert lib.parac_pcg_many(0, None, None, None, 1e-8, 10, None, None) == 0


def test_pcg_many_binding_checks_lengths():
    from paper_2505_02977_gb300 import parac
    with pytest.raises(ValueError):
        parac.parac_pcg_many([object(), object()], [None])


def test_opts_layout_matches_header(tmp_path):
    """The binding's parac_opts has the header's size and every field at the
    header's offset (a C program built against include/parac.h prints them),
    and parac_opts_default fills the documented defaults through it."""
    import shutil
    import subprocess
    from paper_2505_02977_gb300 import parac
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    fields = [f[0] for f in parac.parac_opts._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "parac.h"\nint main(void) {\n'
                   '    printf("size %zu\\n", sizeof(parac_opts));\n'
                   + "".join(f'    printf("{f} %zu\\n", offsetof(parac_opts, {f}));\n' for f in fields)
                   + "    return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    assert int(got["size"]) == ctypes.sizeof(parac.parac_opts)
    for f in fields:
        assert int(got[f]) == getattr(parac.parac_opts, f).offset, f
    o = parac.parac_opts_default()
    assert o.g_precision == 64 and o.max_pool_regrow == 2 and o.spin_limit == 1 << 24 and o.samples == 1
    assert o.grid_help == parac.DEFAULT and o.grid_help_min == 0 and o.host_tables == parac.DEFAULT
    assert o.order == parac.ORDER_GIVEN and o.trace_path is None
