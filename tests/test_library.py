"""The C-ABI library builds, loads and exports every entry point of include/*.h (CPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w \t\*]*?\b(omm_[A-Za-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1312_1549_gb300 import build
    build.build()
    from paper_1312_1549_gb300 import _native
    return _native.lib()


def test_headers_declare_entry_points():
    names = declared_functions()
    for required in ("omm_create", "omm_solve", "omm_backward", "omm_free", "omm_update_H"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1312_1549_gb300 import _native
    assert sorted(_native.EXPORTED) == declared_functions()


def test_status_strings_without_gpu(lib):
    for code in range(10):
        assert lib.omm_status_str(code)


def test_create_rejects_bad_arguments_without_gpu(lib):
    import ctypes as ct
    from paper_1312_1549_gb300 import _native as N
    h = ct.c_void_p()
    # n >= m is rejected before any device work
    rc = lib.omm_create(4, 4, ct.c_void_p(1), ct.c_void_p(1), ct.c_void_p(1), 0.0, 1.0, None, None,
                        ct.byref(h))
    assert rc == 1 and not h.value
    assert b"n < m" in lib.omm_last_error()
    rc = lib.omm_create(8, 2, None, None, None, 0.0, 1.0, None, None, ct.byref(h))
    assert rc == 1


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1312_1549_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
