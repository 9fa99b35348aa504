"""The C-ABI library builds, loads and exports every symbol of include/probe.h (CPU only).

Also exercises the host-side argument validation, which returns before any
device work is issued.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def built_lib():
    import __graft_entry__ as ge
    ge._build_module().build()
    from paper_1101_3615_gb300 import binding
    return binding


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "probe.h")).read()
    return sorted(set(re.findall(r"^(?:probe_status|const char\*|void)\s+(probe_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("probe_create", "probe_apply_F", "probe_apply_Fadj", "probe_apply_H",
                 "probe_apply_H_group", "probe_fit", "probe_apply_precond",
                 "probe_forward_nonlinear", "probe_gradient", "probe_last_error", "probe_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = C.CDLL(built_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert built_lib.probe_version().decode().startswith("matprobe")


def _grid(n=(20, 24), h=(10.0, 10.0), pad=4):
    from paper_1101_3615_gb300.binding import probe_grid
    g = probe_grid()
    g.ndim = 2
    g.n[0], g.n[1] = n
    g.h[0], g.h[1] = h
    g.pad = pad
    g.kahan = 1
    return g


def _create(built_lib, g, m0, src, rec, w, nt, dt):
    h = C.c_void_p()
    src = np.ascontiguousarray(src, np.int32)
    rec = np.ascontiguousarray(rec, np.int32)
    st = built_lib.probe_create(C.byref(h), C.byref(g), C.c_void_p(m0.ctypes.data), len(src),
                                C.c_void_p(src.ctypes.data), len(rec), C.c_void_p(rec.ctypes.data),
                                C.c_void_p(w.ctypes.data), nt, dt)
    return st, h


def test_host_side_validation_rejects_bad_arguments(built_lib):
    m0 = np.full((20, 24), 1 / 2000.0 ** 2, np.float32)
    w = np.zeros(50, np.float32)
    g = _grid()
    # CFL: c dt / h = 2000 * 4e-3 / 10 = 0.8 > 0.5547
    st, h = _create(built_lib, g, m0, [[2, 3]], [[0, 0]], w, 50, 4e-3)
    assert st == -1 and b"CFL" in built_lib.probe_last_error(None)
    st, h = _create(built_lib, g, m0, [[20, 3]], [[0, 0]], w, 50, 1e-3)        # source outside
    assert st == -1
    st, h = _create(built_lib, g, m0, [[2, 3]], [[0, 24]], w, 50, 1e-3)        # receiver outside
    assert st == -1
    bad = m0.copy()
    bad[3, 3] = np.nan
    st, h = _create(built_lib, g, bad, [[2, 3]], [[0, 0]], w, 50, 1e-3)
    assert st == -5                                                             # non-finite m0
    g3 = _grid()
    g3.ndim = 4
    st, h = _create(built_lib, g3, m0, [[2, 3]], [[0, 0]], w, 50, 1e-3)
    assert st == -1


def _header():
    return open(os.path.join(ROOT, "include", "probe.h")).read()


def test_binding_options_match_the_header():
    """Every PROBE_OPT_* of the header has the same value in the binding's option table."""
    from paper_1101_3615_gb300.binding import OPT
    decl = {m.group(1).lower(): int(m.group(2))
            for m in re.finditer(r"PROBE_OPT_(\w+)\s*=\s*(\d+)", _header())}
    assert decl, "no options declared"
    assert sorted(decl.values()) == sorted(OPT.values())
    for name, val in decl.items():
        assert OPT.get(name) == val, (name, val, OPT.get(name))


def test_binding_stats_struct_matches_the_header():
    """probe_stats: the binding's ctypes fields have the header's names, order and C types."""
    from paper_1101_3615_gb300.binding import probe_stats
    head = _header()
    end = head.index("} probe_stats;")
    body = head[head.rindex("typedef struct {", 0, end):end]
    fields = re.findall(r"^\s*(double|long long|int)\s+(\w+);", body, re.M)
    ctype = {"double": C.c_double, "long long": C.c_longlong, "int": C.c_int}
    assert [(n, ctype[t]) for t, n in fields] == [(n, t) for n, t in probe_stats._fields_]


def test_binding_names_every_declared_function(built_lib):
    """The binding exposes each C entry point of the header under its C name, with its
    argument types declared (one argtype per header parameter)."""
    head = _header()
    for name in declared_functions():
        fn = getattr(built_lib, name, None)
        assert fn is not None, f"binding lacks {name}"
        m = re.search(r"^(?:probe_status|const char\*|void)\s+" + name + r"\s*\(([^)]*)\)", head, re.M)
        params = [p for p in m.group(1).split(",") if p.strip() and p.strip() != "void"]
        assert fn.argtypes is not None and len(fn.argtypes) == len(params), (name, params)
