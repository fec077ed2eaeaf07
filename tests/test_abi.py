"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point declared in include/ens.h; host-only calls
validate their arguments and report status codes."""
import ctypes
import os
import re

import pytest

import paper_1511_03703_gb300 as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_names():
    txt = open(os.path.join(ROOT, "include", "ens.h")).read()
    body = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ens_[a-z0-9_]+)\s*\(", body)))


def test_library_exports_every_declared_symbol():
    L = E.lib()
    names = declared_names()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name


def test_binding_covers_the_header():
    assert set(E.exported_symbols()) == set(declared_names())


def test_host_side_sizes_and_errors():
    assert E.mesh_sizes(8) == (729, 15625, 512)
    assert E.mesh_sizes(64) == (274625, 7189057, 262144)
    assert E.mesh_sizes(128) == (2146689, 57066625, 2097152)
    with pytest.raises(E.EnsError) as ei:
        E.mesh_sizes(0)
    assert ei.value.code == 2
    with pytest.raises(E.EnsError) as ei:
        E.dot_workspace_size(100, 3)
    assert ei.value.code == 2
    with pytest.raises(E.EnsError) as ei:
        E.kl_table_size(8, 65)
    assert ei.value.code == 2
    assert E.kl_table_size(64, 10) == 3 * 10 * 128 + 60
    assert E.dot_workspace_size(274625, 32) > 274625 // 32 * 32 * 8
    assert E.cg_workspace_size(274625, 32) > 3 * 274625 * 32 * 8
    assert E.lib().ens_status_string(6) == b"CG breakdown"


def test_library_is_built_for_sm103a_only():
    from paper_1511_03703_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(build.LIB)


def test_product_path_has_no_oracle_or_cpu_fallback():
    pkg = os.path.join(ROOT, "paper_1511_03703_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "ens_oracle" not in src, f


def test_binding_constants_match_the_header():
    """Every status code, dtype, flag and enum value the binding names has the
    value include/ens.h gives it (a drifted flag would select another path)."""
    import re
    import paper_1511_03703_gb300 as E
    txt = open(os.path.join(ROOT, "include", "ens.h")).read()
    consts = {}
    for name, expr in re.findall(r"#define\s+ENS_([A-Z0-9_]+)\s+\(?([0-9u <]+)\)?\s*$", txt, re.M):
        consts[name] = eval(expr.replace("u", ""))
    for name, val in re.findall(r"\bENS_([A-Z0-9_]+)\s*=\s*(\d+)", txt):
        consts[name] = int(val)
    checked = 0
    for name, val in consts.items():
        if hasattr(E, name):
            assert getattr(E, name) == val, (name, getattr(E, name), val)
            checked += 1
    # the binding's flags and codes are all among them
    for name in ("CG_X0_ZERO", "CG_K1_DEFER", "CG_BATCH_K1_WIDE", "PC_LANCZOS", "PC_CHEBYSHEV", "F64_DF",
                 "ERR_WORKSPACE", "NL_PRECOND_MG"):
        assert name in consts and hasattr(E, name), name
    assert checked >= 20, checked
