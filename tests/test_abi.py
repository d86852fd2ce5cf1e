"""CPU checks of the C ABI: libgrav.so loads without a GPU and exports every
function that include/grav.h declares; no compute call is made."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "grav.h")
LIB = os.path.join(ROOT, "paper_2602_03857_b300", "libgrav.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(grav_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        subprocess.check_call(["python", os.path.join(ROOT, "paper_2602_03857_b300", "build.py")])
    return ctypes.CDLL(LIB)


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ["grav_forward", "grav_adjoint", "grav_datainv_solve", "grav_ctx_create", "grav_ctx_destroy",
              "grav_last_error", "grav_plan_create", "grav_diag"]:
        assert f in fns


def test_every_declared_symbol_is_exported(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, f"declared in grav.h but not exported: {missing}"


def test_exports_match_nm():
    out = subprocess.run(["nm", "-D", "--defined-only", LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (grav_[a-z0-9_]+)", out))
    assert set(declared_functions()) <= exported


def test_python_binding_lists_all_symbols():
    import paper_2602_03857_b300 as g
    assert set(g.EXPORTED) <= set(declared_functions())
    assert g.version().startswith("libgrav")


def test_options_default_without_gpu(lib):
    import paper_2602_03857_b300 as g
    o = g.options()
    assert o.precision == g.GRAV_FP64 and o.z0 == 50.0 and o.lambda_scale == 1e-2
    assert o.near_cells == 8.0 and o.max_iter == 1000


def test_ctx_create_rejects_bad_device_without_gpu(lib):
    import paper_2602_03857_b300 as g
    h = ctypes.c_void_p()
    rc = g._lib.grav_ctx_create(ctypes.byref(h), -1, 0)
    assert rc != 0
    assert len(g._lib.grav_last_error(None)) > 0


def test_binding_constants_match_header():
    import paper_2602_03857_b300 as g
    text = open(HEADER).read()
    for name, val in re.findall(r"#define\s+(GRAV_[A-Z0-9_]+)\s+(-?\d+)\b", text):
        if hasattr(g, name):
            assert getattr(g, name) == int(val), name
    assert g.PRECISIONS == {"fp64": 0, "mixed": 1, "mixed_corner": 2}


def test_c_option_defaults(lib):
    import paper_2602_03857_b300 as g
    o = g.grav_options()
    g._lib.grav_options_default(ctypes.byref(o))
    assert o.precision == g.GRAV_FP64 and o.max_iter == 1000 and o.near_cells == 8.0
    assert o.reorth == 1000 and o.check_stations == 0 and o.precond == 0 and o.outer_max == 0


def test_preconditioner_options_without_gpu(lib):
    import paper_2602_03857_b300 as g
    o = g.options(precond="nystrom", nys_rank=120, nys_coarsen=2)
    assert (o.precond, o.nys_rank, o.nys_coarsen) == (2, 120, 2)
    assert g.options(precond="jacobi").precond == 1 and g.options().precond == 0
    c = g.grav_options()
    g._lib.grav_options_default(ctypes.byref(c))
    assert c.nys_rank == 0 and c.nys_coarsen == 0   # automatic sizes
    with pytest.raises(KeyError):
        g.options(precond="ilu")


def test_options_struct_matches_header(lib):
    """The binding's grav_options has the header's fields, in the header's
    order and C types, and grav_options_default fills every byte of it (a
    field the binding lacks or adds would leave sentinel bytes behind or
    shift the later fields)."""
    import paper_2602_03857_b300 as g
    text = open(HEADER).read()
    body = text[text.index("typedef struct {", text.index("grav_survey;")):text.index("} grav_options;")]
    fields = re.findall(r"^\s+(int|double)\s+(\w+);", body, re.M)
    py = [(n, t) for n, t in g.grav_options._fields_]
    assert [n.rstrip("_") for n, _ in py] == [n for _, n in fields]
    ctypes_of = {"int": ctypes.c_int, "double": ctypes.c_double}
    assert [t for _, t in py] == [ctypes_of[t] for t, _ in fields]
    o = g.grav_options()
    ctypes.memset(ctypes.byref(o), 0xFF, ctypes.sizeof(o))
    g._lib.grav_options_default(ctypes.byref(o))
    assert (o.refine, o.near_fp64, o.diag_fp64, o.nys_coarsen) == (0, 0, 0, 0)
    assert o.timeout_s == 3600.0 and o.inner_max == 20
