"""The C-ABI library builds, loads without a GPU and exports every entry point of include/psp.h."""
import ctypes
import os

import pytest

from paper_1204_0111_gb300 import build as B
from paper_1204_0111_gb300 import psp


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(B.LIB):
        B.build()
    return psp.lib()


def test_every_declared_symbol_is_exported(L):
    names = psp.header_functions()
    assert len(names) >= 11
    for n in names:
        assert hasattr(L, n), n


def test_defaults_and_status_strings(L):
    o = psp.Options()
    L.psp_default_options(ctypes.byref(o))
    assert o.pml_C == 4.0 and abs(o.alpha - 2 * 3.141592653589793) < 1e-15
    assert o.pad_depth == -1 and o.leaf_size == 64 and o.pml_faces == 63
    assert o.precision == psp.PREC_C128 and o.aux_mode == psp.AUX_MOVING_PML
    assert L.psp_status_string(4) == b"zero pivot"
    assert L.psp_status_string(5) == b"not converged"


def test_bad_arguments_are_rejected_before_any_device_call(L):
    h = ctypes.c_void_p()
    g = psp.Grid(0, 4, 4, 0.2)
    c = (ctypes.c_double * 16)()
    st = L.psp_setup(ctypes.byref(g), ctypes.cast(c, ctypes.c_void_p), 1.0, 2, 2, None, None, ctypes.byref(h))
    assert st == 1 and h.value is None
    assert b"grid" in L.psp_last_error()
    g = psp.Grid(4, 4, 4, 0.2)
    st = L.psp_setup(ctypes.byref(g), ctypes.cast(c, ctypes.c_void_p), -1.0, 2, 2, None, None, ctypes.byref(h))
    assert st == 1
    st = L.psp_setup(ctypes.byref(g), ctypes.cast(c, ctypes.c_void_p), 1.0, 2, 0, None, None, ctypes.byref(h))
    assert st == 1
    o = psp.Options()
    L.psp_default_options(ctypes.byref(o))
    o.precision = 7
    st = L.psp_setup(ctypes.byref(g), ctypes.cast(c, ctypes.c_void_p), 1.0, 2, 2, ctypes.byref(o), None, ctypes.byref(h))
    assert st == 1
    L.psp_default_options(ctypes.byref(o))
    o.sweep_claim_ahead = 3
    st = L.psp_setup(ctypes.byref(g), ctypes.cast(c, ctypes.c_void_p), 1.0, 2, 2, ctypes.byref(o), None, ctypes.byref(h))
    assert st == 1 and b"options" in L.psp_last_error()
    assert L.psp_apply(None, None, None, 1, None) == 1
    assert L.psp_destroy(None) == 0


def test_batch_arguments_are_rejected_before_any_device_call(L):
    h = ctypes.c_void_p()
    grids = (psp.Grid * 2)(psp.Grid(4, 4, 4, 0.2), psp.Grid(4, 0, 4, 0.2))
    c = (ctypes.c_double * 64)()
    cs = (ctypes.c_void_p * 2)(ctypes.cast(c, ctypes.c_void_p), ctypes.cast(c, ctypes.c_void_p))
    om = (ctypes.c_double * 2)(1.0, 1.0)
    ga = (ctypes.c_int * 2)(2, 2)
    de = (ctypes.c_int * 2)(2, 2)
    assert L.psp_setup_batch(0, grids, cs, om, ga, de, None, None, ctypes.byref(h)) == 1 and h.value is None
    assert L.psp_setup_batch(2, grids, cs, om, ga, de, None, None, ctypes.byref(h)) == 1   # second grid is empty
    assert b"grid" in L.psp_last_error()
    grids[1] = psp.Grid(4, 4, 4, 0.2)
    de[1] = 0
    assert L.psp_setup_batch(2, grids, cs, om, ga, de, None, None, ctypes.byref(h)) == 1
    assert L.psp_setup_batch(2, grids, None, om, ga, de, None, None, ctypes.byref(h)) == 1
    n = ctypes.c_int()
    assert L.psp_batch_layout(None, ctypes.byref(n), None, 0) == 1


def test_tune_sweep_rejects_bad_arguments(L):
    assert L.psp_tune_sweep(None, 1, 1, None, None) == 1


def _c_struct_fields(name):
    """Field names, in order, of `typedef struct { ... } name;` in include/psp.h."""
    import re
    text = open(psp.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text, flags=re.S)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        fp = re.match(r".*\(\s*\*\s*(\w+)\s*\)\s*\(.*\)$", decl, flags=re.S)   # function pointer
        if fp:
            fields.append(fp.group(1))
            continue
        names = decl.split(None, 1)[1] if " " in decl else decl
        for nm in names.split(","):
            nm = nm.strip().lstrip("*").strip()
            fields.append(re.sub(r"\[.*\]", "", nm))
    return fields


@pytest.mark.parametrize("cname,py", [("psp_options", psp.Options), ("psp_solve_info", psp.SolveInfo),
                                      ("psp_kernel_stat", psp.KernelStat), ("psp_sweep_tuning", psp.SweepTuning),
                                      ("psp_setup_tuning", psp.SetupTuning), ("psp_grid", psp.Grid)])
def test_binding_structs_match_the_header(cname, py):
    # the ctypes mirrors must list the C fields in the same order (a shifted field would silently
    # pass the wrong option)
    assert [f for f, _ in py._fields_] == _c_struct_fields(cname)
