"""The C-ABI library loads on a machine without a GPU and exports every symbol
the header declares.  No compute call is made here."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "abilu.h")


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g._build_ext().build()
    import paper_1912_00539_gb300.abilu as ab
    return ab


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(\w+)\s*\(", text, flags=re.M)) -
                  {"if", "while"})


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("abilu_build", "abilu_apply", "bsr_spmv", "fgmres_solve"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    for nm in names:
        assert hasattr(lib._lib, nm), nm
    assert set(names) == set(lib.EXPORTS)


def test_version_and_default_opts(lib):
    assert lib.version().startswith("abilu-gb300")
    o = lib.default_opts()
    assert (o.restart, o.max_iters, o.rtol) == (30, 2500, 1e-6)
    assert (o.build_sweeps, o.apply_sweeps_lower, o.apply_sweeps_upper) == (1, 3, 3)


def test_argument_errors_before_any_device_work(lib):
    h = C.c_void_p()
    st = lib._lib.abilu_pattern_create(0, 0, None, None, None, C.byref(h))
    assert st == lib.EINVAL and not h.value
    assert b"n >= 1" in lib._lib.abilu_last_error()
    assert lib._lib.abilu_pattern_create(4, 2, None, None, None, C.byref(h)) == lib.EINVAL
    assert lib._lib.abilu_build(None, None, 1, 0, 0, None) == lib.EINVAL
    assert lib._lib.abilu_apply(None, None, None, 1, 1, 0, None) == lib.EINVAL
    assert lib._lib.bsr_spmv(None, None, 1.0, None, 0.0, None, None) == lib.EINVAL
    r = lib.FgmresResult()
    o = lib.default_opts()
    assert lib._lib.fgmres_solve(None, None, None, None, None, C.byref(o), C.byref(r), None) == lib.EINVAL


def test_multigrid_defaults_and_argument_errors(lib):
    o = lib.MgOpts()
    lib._lib.abilu_mg_default_opts(C.byref(o))
    assert (o.max_levels, o.min_coarse, o.theta) == (10, 512, 0.25)
    assert (o.factor_dtype, o.build_sweeps, o.apply_sweeps_lower, o.apply_sweeps_upper) == (1, 4, 2, 2)
    assert (o.pre_smooth, o.post_smooth, o.coarse_smooth, o.mode, o.init) == (1, 1, 2, 0, 0)
    h = C.c_void_p()
    assert lib._lib.abilu_mg_create(None, None, C.byref(o), None, C.byref(h)) == lib.EINVAL
    assert not h.value
    assert lib._lib.abilu_mg_setup(None, None, None) == lib.EINVAL
    assert lib._lib.abilu_mg_apply(None, None, None, None) == lib.EINVAL
    out = (C.c_int64 * 33)()
    assert lib._lib.abilu_mg_levels(None, out) == lib.EINVAL
    r = lib.FgmresResult()
    fo = lib.default_opts()
    assert lib._lib.fgmres_solve_mg(None, None, None, None, C.byref(fo), C.byref(r), None) == lib.EINVAL
