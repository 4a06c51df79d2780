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


def _struct_fields(name):
    """(type, field) pairs of `typedef struct { ... } name;` in include/omm.h, comments removed."""
    text = open(os.path.join(ROOT, "include", "omm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        m = re.match(r"(int|double)\s+(\w+)(\[(\d+)\])?$", decl)
        assert m, decl
        out.append((m.group(1), m.group(2), int(m.group(4)) if m.group(4) else None))
    return out


@pytest.mark.parametrize("cname,pyname", [("omm_opts", "OmmOpts"), ("omm_info", "OmmInfo")])
def test_binding_structs_match_the_header(cname, pyname):
    """The ctypes mirrors of omm_opts and omm_info have the header's fields, order and types."""
    import ctypes as ct
    from paper_1312_1549_gb300 import _native
    py = getattr(_native, pyname)._fields_
    hdr = _struct_fields(cname)
    assert [f for _, f, _ in hdr] == [f for f, _ in py]
    for (t, f, n), (_, pt) in zip(hdr, py):
        base = ct.c_int if t == "int" else ct.c_double
        assert pt == (base * n if n else base), f


def test_new_entry_points_reject_bad_arguments_without_gpu(lib):
    import ctypes as ct
    from paper_1312_1549_gb300 import _native as N
    h = ct.c_void_p()
    rc = lib.omm_create_hermitian(4, 4, ct.c_void_p(1), ct.c_void_p(1), None, 0.0, 1.0, None, None, ct.byref(h))
    assert rc == 1 and not h.value
    opts = N.OmmOpts(precision=N.PREC_MIXED, cholesky=1)
    rc = lib.omm_create_hermitian(8, 2, ct.c_void_p(1), ct.c_void_p(1), None, 0.0, 1.0, ct.byref(opts), None,
                                  ct.byref(h))
    assert rc == 1 and b"Cholesky" in lib.omm_last_error()
    opts = N.OmmOpts(precision=N.PREC_MIXED, precond_slices=11)
    rc = lib.omm_create(8, 2, ct.c_void_p(1), ct.c_void_p(1), ct.c_void_p(1), 0.0, 1.0, ct.byref(opts), None,
                        ct.byref(h))
    assert rc == 1 and b"precond_slices" in lib.omm_last_error()
    info = ct.c_int(0)
    rc = lib.omm_kernel_spd_inverse_precond(8, ct.c_void_p(1), ct.c_void_p(1), 10, ct.byref(info), None)
    assert rc == 1
    assert lib.omm_solve_hermitian(None, None, None, None, None, None) == 1
    assert lib.omm_backward_hermitian(None, None, None) == 1
