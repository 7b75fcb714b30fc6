"""CPU checks of the C ABI: the library builds, loads and exports every entry
point that include/*.h declares; the binding's struct layouts match the
header's (field count and order).  No GPU calls."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for f in sorted(os.listdir(inc)):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(mrcg_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_12417_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("mrcg_solver_create", "mrcg_solve", "mrcg_apply_A", "mrcg_apply_mmr", "mrcg_inner_solve",
              "mrcg_solver_destroy", "mrcg_status_string"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings(lib):
    lib.mrcg_status_string.restype = C.c_char_p
    lib.mrcg_status_string.argtypes = [C.c_int]
    names = [lib.mrcg_status_string(i).decode() for i in range(8)]
    assert names == ["MRCG_OK", "MRCG_ERR_INVALID", "MRCG_ERR_NOT_SPD", "MRCG_ERR_BREAKDOWN", "MRCG_ERR_MAXITER",
                     "MRCG_ERR_NONFINITE", "MRCG_ERR_CUDA", "MRCG_ERR_OOM"]


def test_null_arguments_rejected_without_gpu(lib):
    import paper_1805_12417_gb300 as m
    L = m.lib()
    assert L.mrcg_solver_create(None, None) == m.ERR_INVALID
    assert L.mrcg_solve(None, None, None, 1e-10, 1e-3, 0, None) == m.ERR_INVALID
    assert L.mrcg_apply_A(None, None, None) == m.ERR_INVALID
    L.mrcg_solver_destroy(None)


def _c_struct_fields(name):
    src = open(os.path.join(ROOT, "include", "mrcg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", src).group(1)
    fields = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            fields.append(re.findall(r"(\w+)\s*$", part.strip())[0])
    return fields


@pytest.mark.parametrize("cname,pyname", [("mrcg_create_args", "CreateArgs"), ("mrcg_info", "Info"),
                                          ("mrcg_eig_info", "EigInfo"), ("mrcg_complex_args", "ComplexArgs"),
                                          ("mrcg_complex_info", "ComplexInfo")])
def test_binding_struct_layout_matches_header(cname, pyname):
    import paper_1805_12417_gb300 as m
    cf = _c_struct_fields(cname)
    pf = [f[0].rstrip("_") for f in getattr(m, pyname)._fields_]
    assert cf == pf


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No fallback: without libmrcg.so every entry point raises."""
    import numpy as np

    import paper_1805_12417_gb300 as m
    monkeypatch.setattr(m, "LIB_PATH", str(tmp_path / "libmrcg.so"))
    monkeypatch.setattr(m, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        m.lib()
    with pytest.raises(RuntimeError, match="not built"):
        m.solver_create(1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([2.0]))


def test_product_package_never_reaches_the_oracle():
    """The package (binding, build, profiling driver, CUDA sources) neither
    imports nor links anything under oracle/."""
    pkg = os.path.join(ROOT, "paper_1805_12417_gb300")
    hits = []
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                if re.search(r"\boracle\b|mrcg_oracle|orc_", src):
                    hits.append(f)
    assert hits == []
