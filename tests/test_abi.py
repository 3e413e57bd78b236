"""The C ABI library loads and exports every symbol include/*.h declares (no GPU needed)."""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        txt = re.sub(r"//[^\n]*", "", txt)
        for m in re.finditer(r"\b(chase_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2205_02491_gb300 import build as b
    b.build()
    from paper_2205_02491_gb300 import _lib
    return _lib.load()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("chase_create", "chase_solve", "chase_eigvals", "chase_eigvecs", "chase_backward", "chase_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2205_02491_gb300 import _lib
    assert sorted(set(declared_symbols())) == sorted(set(_lib.EXPORTED))


def test_default_opts_and_workspace_formula(lib):
    import ctypes as C
    from paper_2205_02491_gb300 import _lib
    o = _lib.Opts()
    lib.chase_default_opts(C.byref(o))
    assert (o.maxdeg, o.lanczos_steps, o.lanczos_runs, o.maxiter) == (36, 25, 4, 30)
    b = lib.chase_workspace_bytes(30000, 1600, _lib.CHASE_C128, C.byref(o))
    # single-GPU form of Eq. GPU_mem without the n^2 term: at least 3 n ne + 2 ne^2 scalars
    assert b >= (3 * 30000 * 1600 + 2 * 1600 * 1600) * 16


def test_create_rejects_bad_arguments_without_gpu_work(lib):
    import ctypes as C
    from paper_2205_02491_gb300 import _lib
    ctx = C.c_void_p()
    # ne_max > n_max is rejected before any device call
    assert lib.chase_create(C.byref(ctx), 10, 20, _lib.CHASE_C128, None, None) == 1
    assert lib.chase_create(C.byref(ctx), 10, 5, 7, None, None) == 1
    assert lib.chase_solve(None, None, 1, 1, 1, 0, 1e-10, 1, 0, None, None) == 1


def _header_struct_fields(name):
    """(type, field) pairs of `typedef struct { ... } name;` in include/chase_gb300.h, in order."""
    txt = open(os.path.join(ROOT, "include", "chase_gb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", txt)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        typ, rest = decl.split(None, 1)
        for f in rest.split(","):
            fields.append((typ, f.strip()))
    return fields


@pytest.mark.parametrize("cname,pyname", [("chase_opts", "Opts"), ("chase_stats_t", "Stats")])
def test_ctypes_structs_mirror_the_header(cname, pyname):
    """The ctypes mirrors of the option and statistics structs have the header's fields, types and order
    (a mismatch would silently shift every field after it)."""
    import ctypes as C
    from paper_2205_02491_gb300 import _lib
    ctype = {"int": C.c_int, "int64_t": C.c_int64, "double": C.c_double}
    hdr = _header_struct_fields(cname)
    py = getattr(_lib, pyname)._fields_
    assert [f for _, f in hdr] == [f for f, _ in py]
    assert [ctype[t] for t, _ in hdr] == [t for _, t in py]
