"""The C-ABI library loads and exports every entry point of include/ghsvd.h
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ghsvd.h")


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ghsvd_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_08560_gb300 import build, ghsvd
    build.build()
    return ghsvd.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("ghsvd_create", "ghsvd_solve", "ghsvd_solve_from", "ghsvd_solve_host",
              "ghsvd_get_factors", "ghsvd_get_stats", "ghsvd_destroy", "ghsvd_status_string",
              "ghsvd_default_opts"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_default_opts_and_status_strings(lib):
    from paper_1907_08560_gb300 import ghsvd
    o = ghsvd.ghsvd_default_opts()
    assert (o.block_width, o.inner_sweeps, o.max_sweeps, o.crit_mode, o.precision) == (32, 1, 30, 0, 0)
    for s in range(10):
        assert ghsvd.status_string(s) != "unknown status"
    assert (o.ordering, o.tol_scale, o.timeout_ms, o.shorten) == (0, 1.0, 0, 0)
    assert ghsvd.status_string(99) == "unknown status"


def test_create_rejects_bad_options(lib):
    from paper_1907_08560_gb300 import ghsvd
    for bad in (dict(block_width=0), dict(block_width=33), dict(inner_sweeps=0),
                dict(max_sweeps=0), dict(crit_mode=2), dict(precision=5), dict(shorten=2),
                dict(ordering=1), dict(tol_scale=0.0), dict(tol_scale=-1.0), dict(timeout_ms=-1)):
        o = ghsvd.ghsvd_default_opts(**bad)
        h = ctypes.c_void_p()
        s = lib.ghsvd_create(ctypes.byref(h), 0, ctypes.byref(o))
        assert s == ghsvd.GHSVD_ERR_INVALID_ARG and not h.value


def test_null_arguments_are_rejected(lib):
    from paper_1907_08560_gb300 import ghsvd
    assert lib.ghsvd_create(None, 0, None) == ghsvd.GHSVD_ERR_INVALID_ARG
    assert lib.ghsvd_default_opts(None) == ghsvd.GHSVD_ERR_INVALID_ARG
    assert lib.ghsvd_get_stats(None, None) == ghsvd.GHSVD_ERR_INVALID_ARG
    lib.ghsvd_destroy(None)
    s = lib.ghsvd_solve(None, 4, 4, 4, None, 4, None, 0, None, 4, None, None, 4, None, None)
    assert s == ghsvd.GHSVD_ERR_INVALID_ARG
    s = lib.ghsvd_urv(6, 6, 4, None, 6, None, 3, None, 6, None, 4, None, None, 4, None, None, None)
    assert s == ghsvd.GHSVD_ERR_INVALID_ARG
    assert lib.ghsvd_inverse(4, None, 4, None, 4, None) == ghsvd.GHSVD_ERR_INVALID_ARG
    assert lib.ghsvd_inverse(0, None, 4, None, 4, None) == ghsvd.GHSVD_ERR_INVALID_ARG
    assert lib.ghsvd_phase4(None, None, None, None, 4, None) == ghsvd.GHSVD_ERR_INVALID_ARG
    s = lib.ghsvd_decomposition_errors(None, None, 4, None, 4, None, 4, None, None, None)
    assert s == ghsvd.GHSVD_ERR_INVALID_ARG


def test_binding_has_the_same_names(lib):
    from paper_1907_08560_gb300 import ghsvd
    for name in declared_functions():
        if name in ("ghsvd_status_string",):
            continue
        assert hasattr(ghsvd, name), name
