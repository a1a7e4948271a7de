"""CPU checks of the C-ABI library: it loads, exports every symbol include/amg.h
declares, and rejects invalid arguments before touching a GPU."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2007_00056_gb300 import amg, build

    build.build()
    return amg.lib()


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "amg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:\w+\s+)+\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "return")))


def test_header_declarations_are_exported(lib):
    from paper_2007_00056_gb300 import amg

    declared = _declared_functions()
    assert set(amg.EXPORTS) <= set(declared)
    out = subprocess.run(["nm", "-D", "--defined-only", amg.lib_path()], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (\w+)$", out, flags=re.M))
    missing = [n for n in declared if n not in exported]
    assert not missing, f"declared in include/amg.h but not exported: {missing}"
    for name in declared:
        assert hasattr(lib, name)


def test_default_params_and_strings(lib):
    from paper_2007_00056_gb300 import amg

    p = amg.amg_default_params()
    assert (p.passes, p.max_levels, p.coarse_max, p.nu_pre, p.nu_post) == (2, 10, 4096, 1, 1)
    assert p.stall_ratio == 0.85 and abs(p.omega - 2.0 / 3.0) < 1e-16
    assert (p.cycle, p.tie_break, p.edge_weight) == (amg.AMG_CYCLE_V, amg.AMG_TIE_SMALLER, amg.AMG_WEIGHT_ABS)
    assert lib.amg_default_params(None) == amg.AMG_ERR_INVALID_ARG
    for s in range(10):
        assert len(amg.status_string(s)) >= 2
    assert amg.status_string(5) == "Krylov breakdown"


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_2007_00056_gb300 import amg

    out = C.c_void_p(123)
    p = amg.amg_default_params()
    # n <= 0 and null pointers are rejected before any device call
    assert lib.amg_setup(0, 0, None, None, None, C.byref(p), None, C.byref(out)) == amg.AMG_ERR_INVALID_ARG
    assert out.value is None
    assert lib.amg_setup(5, 10, None, None, None, C.byref(p), None, C.byref(out)) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_setup(5, 10, 8, 8, 8, C.byref(p), None, None) == amg.AMG_ERR_INVALID_ARG
    bad = amg.amg_default_params(passes=0)
    assert lib.amg_setup(5, 10, 8, 8, 8, C.byref(bad), None, C.byref(out)) == amg.AMG_ERR_INVALID_ARG
    bad = amg.amg_default_params(omega=2.5)
    assert lib.amg_setup(5, 10, 8, 8, 8, C.byref(bad), None, C.byref(out)) == amg.AMG_ERR_INVALID_ARG
    for kw in (dict(cycle=3), dict(cycle=-1), dict(tie_break=2), dict(edge_weight=-1)):
        bad = amg.amg_default_params(**kw)
        assert lib.amg_setup(5, 10, 8, 8, 8, C.byref(bad), None, C.byref(out)) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_vcycle(None, 8, 16, None) == amg.AMG_ERR_INVALID_ARG
    info = amg.amg_solve_info()
    assert lib.pcg_solve(None, 8, 16, 1e-8, 10, 0, None, C.byref(info)) == amg.AMG_ERR_INVALID_ARG
    assert lib.bicgstab_solve(None, 8, 16, 1e-8, 10, None, C.byref(info)) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_solve(None, 8, 16, 1e-8, 10, None, C.byref(info)) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_coarse_cg_cluster_size(None) == -1
    assert lib.amg_num_levels(None) == -1
    assert lib.amg_setup_rounds(None, 0, 0) == -1
    lib.amg_destroy(None)  # no-op


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    """The binding raises instead of computing anything on the host."""
    from paper_2007_00056_gb300 import amg

    monkeypatch.setattr(amg, "_lib", None)
    monkeypatch.setattr(amg, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        amg.lib()


def _header_text():
    text = open(os.path.join(ROOT, "include", "amg.h")).read()
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def test_binding_constants_match_the_header():
    """Every enum constant the binding defines has the header's value."""
    from paper_2007_00056_gb300 import amg

    consts = dict((m.group(1), int(m.group(2)))
                  for m in re.finditer(r"\b(AMG_[A-Z0-9_]+)\s*=\s*(-?\d+)", _header_text()))
    checked = 0
    for name, value in consts.items():
        if hasattr(amg, name):
            assert getattr(amg, name) == value, name
            checked += 1
    assert checked >= 20


def test_params_struct_layout_matches_the_header():
    """amg_params and amg_solve_info: same fields, order and C types as the header."""
    from paper_2007_00056_gb300 import amg

    text = _header_text()
    ctype = {"int": C.c_int, "double": C.c_double, "amg_status": C.c_int}
    for struct, cls in (("amg_params", amg.amg_params), ("amg_solve_info", amg.amg_solve_info)):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + struct + r"\s*;", text).group(1)
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            typ, names = decl.split(None, 1)
            fields += [(n.strip(), ctype[typ]) for n in names.split(",")]
        assert [(n, t) for n, t in cls._fields_] == fields, struct
