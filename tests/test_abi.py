"""The C-ABI library builds, loads without a GPU and exports every entry point include/cans.h declares."""
import ctypes
import os
import re

import pytest

from paper_2001_05234_b300 import build_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(cans_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def cans():
    build_lib.build()
    import paper_2001_05234_b300 as P

    return P


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("cans_poisson_plan", "cans_poisson_solve", "cans_poisson_workspace_size", "cans_plan_destroy",
                 "cans_status_string", "cans_poisson_solve_batched", "cans_poisson_solve_adjoint"):
        assert must in names


def test_library_exports_every_declared_symbol(cans):
    L = cans.lib()
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings(cans):
    for code in range(-7, 1):
        s = cans.cans_status_string(code)
        assert s and s != "unknown status"
    assert cans.cans_status_string(42) == "unknown status"


def test_opts_defaults(cans):
    o = cans.cans_opts_default()
    assert o.prec == cans.CANS_FP64 and o.max_sweeps == 2 and o.tol == 1e-12 and abs(o.fp64_mode_fraction - 0.01) < 1e-15
    assert o.verify == 0


def test_plan_status_rejects_null_arguments(cans):
    import ctypes

    word = ctypes.c_int(5)
    assert cans.lib().cans_plan_status(None, ctypes.byref(word)) == cans.CANS_ERR_ARG
    assert cans.lib().cans_plan_status(None, None) == cans.CANS_ERR_ARG


def test_bounded_wait_check_rejects_bad_arguments(cans):
    """Refused before any launch: a NULL plan, no polls, more than 2^20 polls."""
    assert cans.lib().cans_check_bounded_wait(None, 100, 0, None) == cans.CANS_ERR_ARG
    fake = 1  # never dereferenced: the poll count is checked first
    assert cans.lib().cans_check_bounded_wait(fake, 0, 0, None) == cans.CANS_ERR_ARG
    assert cans.lib().cans_check_bounded_wait(fake, (1 << 20) + 1, 0, None) == cans.CANS_ERR_ARG


@pytest.mark.parametrize(
    "n,L,bc,dzf,want",
    [
        ((0, 8, 8), (1, 1), (0, 0, 1), None, -1),  # empty dimension
        ((8, 8, 8), (1, -1), (0, 0, 1), None, -1),  # bad length
        ((8, 8, 8), (1, 1), (0, 5, 1), None, -1),  # bad boundary condition
        ((8, 8, 4), (1, 1), (0, 0, 1), [0.25, 0.25, -0.1, 0.6], -1),  # negative cell width
        ((8, 8, 4), (1, 1), (0, 0, 1), [0.25, 0.25, float("nan"), 0.5], -1),  # non-finite cell width
        ((8, 8, 4), (1, 1), (0, 0, 0), [0.2, 0.3, 0.25, 0.25], -1),  # periodic z must be uniform
        ((8, 8, 5), (1, 1), (0, 0, 0), None, -2),  # odd periodic Nz
        ((7, 8, 4), (1, 1), (0, 0, 1), None, -2),  # odd periodic N
        ((8, 10, 4), (1, 1), (0, 1, 1), None, -2),  # N/2 = 5 does not factor into 2s and 3s
        ((8, 8, 600), (1, 1), (0, 0, 1), None, -2),  # Nz above 512
        ((8, 8, 8), (1, 1), (0, 0, 6), None, -1),  # no such boundary condition
        ((7, 8, 8), (1, 1), (3, 0, 1), None, -2),  # odd N along a quarter-wave direction
    ],
)
def test_plan_rejects_bad_arguments_on_the_host(cans, n, L, bc, dzf, want):
    st, h = cans.cans_poisson_plan(n, L, bc, dzf, None, check=False)
    assert st == want
    assert not h.value


def test_null_arguments(cans):
    L = cans.lib()
    assert L.cans_poisson_plan(None, None, None, None, None, None) == -1
    assert L.cans_poisson_solve(None, None, None, None, None, None) == -1
    assert L.cans_plan_destroy(None) == -1
    assert L.cans_poisson_workspace_size(None, None) == -1


@pytest.mark.parametrize("field,value,bc", [("shift", 1.0, (0, 0, 2)), ("shift", float("inf"), (0, 0, 2)),
                                            ("z_grid", 2, (0, 0, 2)), ("z_grid", 1, (0, 0, 1)),
                                            ("z_grid", 1, (0, 0, 3))])
def test_plan_rejects_bad_helmholtz_options_on_the_host(cans, field, value, bc):
    """A positive or non-finite shift, an unknown z grid, and the face grid without Dirichlet walls at
    both ends are refused before any device work."""
    o = cans.cans_opts_default()
    setattr(o, field, value)
    st, h = cans.cans_poisson_plan((8, 8, 8), (1, 1), bc, None, o, check=False)
    assert st == -1 and not h.value
