"""C-ABI library: loads, exports every symbol of include/rh.h, and its host
symbolic phase matches the oracle's independent one bit for bit (no GPU needed:
a grid created with device < 0 runs the symbolic phase only)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import OracleGrid
from paper_2201_00241_gb300 import gridgen as gg
from paper_2201_00241_gb300 import rh

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "rh.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rh_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = rh.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(rh.EXPORTS) == names


def host_grid(g):
    """rh_grid_create with device = -1 (symbolic phase only)."""
    lib = rh.load()
    keep = [np.ascontiguousarray(g.fr, np.int32), np.ascontiguousarray(g.to, np.int32),
            np.ascontiguousarray(g.r, float), np.ascontiguousarray(g.x, float), np.ascontiguousarray(g.b, float),
            np.ascontiguousarray(g.bus_type, np.int8), np.ascontiguousarray(g.c2, float),
            np.ascontiguousarray(g.c1, float)]
    d = rh._Desc(g.n_bus, g.n_branch, *[rh._ptr(a) for a in keep], g.base_mva, g.order_level_cost)
    h = C.c_void_p(0)
    st = lib.rh_grid_create(C.byref(d), -1, C.byref(h))
    return st, h, keep


@pytest.mark.parametrize("case,level_cost", [("tiny9", None), ("tiny30", None), ("case118", None),
                                             ("case1354", None), ("case2869", None), ("case9241", None),
                                             ("case118", 0), ("case1354", 0), ("case1354", 10**12)])
def test_symbolic_bit_exact_against_oracle(case, level_cost):
    """Order, patterns and levels equal the oracle's, bit for bit; also with other
    values of the level weight that both sides take from the grid record."""
    import dataclasses
    g = gg.make_grid(9, 12, 3, 2) if case == "tiny9" else gg.make_grid(30, 41, 6, 4) if case == "tiny30" \
        else gg.make_case(case)
    if level_cost is not None:
        g = dataclasses.replace(g, order_level_cost=level_cost)
    lib = rh.load()
    st, h, keep = host_grid(g)
    assert st == 0, lib.rh_last_error()
    try:
        dm = rh.Dims()
        assert lib.rh_grid_dims(h, C.byref(dm)) == 0
        nx = dm.n_x
        out = dict(perm=np.empty(nx, np.int32), bus_order=np.empty(g.n_bus - 1, np.int32),
                   level=np.empty(g.n_bus - 1, np.int32), Lp=np.empty(nx + 1, np.int32),
                   Lj=np.empty(dm.nnz_l, np.int32), Up=np.empty(nx + 1, np.int32), Uj=np.empty(dm.nnz_u, np.int32))
        assert lib.rh_grid_symbolic(h, *[rh._ptr(out[k]) for k in ("perm", "bus_order", "level", "Lp", "Lj", "Up",
                                                                   "Uj")]) == 0
        # a device call on a symbolic-only grid is refused, not attempted
        assert lib.rh_adjoint(h, None, None, None) == rh.RH_ESTATE
    finally:
        lib.rh_grid_destroy(h)
    ref = OracleGrid(g).symbolic()
    assert (dm.n_x, dm.n_p) == (OracleGrid(g).n_x, OracleGrid(g).n_p)
    for k in ("perm", "bus_order", "level", "Lp", "Lj", "Up", "Uj"):
        assert np.array_equal(out[k], ref[k]), k


def test_invalid_grids_are_rejected():
    g = gg.make_grid(9, 12, 3, 2)
    lib = rh.load()
    bad = gg.make_grid(9, 12, 3, 2)
    bad.bus_type = bad.bus_type.copy()
    bad.bus_type[bad.bus_type == 1] = 0          # several slack buses
    st, h, _ = host_grid(bad)
    assert st == rh.RH_EINVAL and b"slack" in lib.rh_last_error()
    bad = gg.make_grid(9, 12, 3, 2)
    bad.to = bad.to.copy()
    bad.to[0] = bad.fr[0]                         # self loop
    st, h, _ = host_grid(bad)
    assert st == rh.RH_EINVAL
    bad = gg.make_grid(9, 12, 3, 2)
    bad.r = np.zeros_like(bad.r)
    bad.x = np.zeros_like(bad.x)                  # zero impedance
    st, h, _ = host_grid(bad)
    assert st == rh.RH_EINVAL
    import dataclasses
    st, h, _ = host_grid(dataclasses.replace(g, order_level_cost=-1))   # negative level weight
    assert st == rh.RH_EINVAL and b"order_level_cost" in lib.rh_last_error()
    st, h, _ = host_grid(g)
    assert st == 0
    lib.rh_grid_destroy(h)


@pytest.mark.parametrize("case", ["tiny9", "tiny30", "case118", "case1354", "case2869", "case9241"])
def test_coloring_bit_exact_against_oracle(case):
    """The library's column colouring (host symbolic phase) equals the oracle's
    independent greedy colouring, colour for colour."""
    g = gg.make_grid(9, 12, 3, 2) if case == "tiny9" else gg.make_grid(30, 41, 6, 4) if case == "tiny30" \
        else gg.make_case(case)
    lib = rh.load()
    st, h, keep = host_grid(g)
    assert st == 0, lib.rh_last_error()
    try:
        o = OracleGrid(g)
        cx, cp = np.empty(o.n_x, np.int32), np.empty(o.n_p, np.int32)
        ncx, ncp = C.c_int32(0), C.c_int32(0)
        assert lib.rh_grid_coloring(h, rh._ptr(cx), rh._ptr(cp), C.byref(ncx), C.byref(ncp)) == 0
        assert lib.rh_jacobian(h, 1, None, None, None, None, None, None) == rh.RH_ESTATE
    finally:
        lib.rh_grid_destroy(h)
    ref_x, ref_p, ref_ncx, ref_ncp = o.coloring()
    assert (ncx.value, ncp.value) == (ref_ncx, ref_ncp)
    assert np.array_equal(cx, ref_x) and np.array_equal(cp, ref_p)
