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
    return sorted(set(re.findall(r"\b(rh_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = rh.load()
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(rh.EXPORTS) == names


def host_grid(g, max_tail=0):
    """rh_grid_create with device = -1 (symbolic phase only)."""
    lib = rh.load()
    keep = [np.ascontiguousarray(g.fr, np.int32), np.ascontiguousarray(g.to, np.int32),
            np.ascontiguousarray(g.r, float), np.ascontiguousarray(g.x, float), np.ascontiguousarray(g.b, float),
            np.ascontiguousarray(g.bus_type, np.int8), np.ascontiguousarray(g.c2, float),
            np.ascontiguousarray(g.c1, float)]
    d = rh._Desc(g.n_bus, g.n_branch, *[rh._ptr(a) for a in keep], g.base_mva, g.order_level_cost, max_tail)
    h = C.c_void_p(0)
    st = lib.rh_grid_create(C.byref(d), -1, C.byref(h))
    return st, h, keep


@pytest.mark.parametrize("case,level_cost,max_tail", [
    ("tiny9", None, 0), ("tiny30", None, 0), ("case118", None, 0), ("case1354", None, 0), ("case2869", None, 0),
    ("case9241", None, 0), ("case118", 0, 0), ("case1354", 0, 0), ("case1354", 10**12, 0),
    ("case1354", None, 2), ("case1354", None, 512), ("case9241", None, 64)])
def test_symbolic_bit_exact_against_oracle(case, level_cost, max_tail):
    """Order, patterns and levels equal the oracle's, bit for bit; also with other
    values of the level weight that both sides take from the grid record, and with
    other dense-tail bounds (the tail is a storage choice of the library: it changes
    neither the order nor the patterns)."""
    import dataclasses
    g = gg.make_grid(9, 12, 3, 2) if case == "tiny9" else gg.make_grid(30, 41, 6, 4) if case == "tiny30" \
        else gg.make_case(case)
    if level_cost is not None:
        g = dataclasses.replace(g, order_level_cost=level_cost)
    lib = rh.load()
    st, h, keep = host_grid(g, max_tail)
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
    for t in (-1, 1, 513):                                               # dense-tail bound out of range
        st, h, _ = host_grid(g, t)
        assert st == rh.RH_EINVAL and b"max_tail" in lib.rh_last_error()
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


@pytest.mark.parametrize("case,n_sm", [("tiny30", 4), ("case1354", 152), ("case9241", 152), ("case9241", 148)])
def test_reduced_hessian_flop_counts(case, n_sm):
    """rh_reduced_hessian_flops against a count made here from the symbolic data the
    library exports (order, L and U patterns) and the oracle's J_p pattern: the
    algorithmic count of Algorithm 2 for n_p dense directions, and the work the two
    direction launches issue (each CTA's forward sweep over its reach, the last L^T
    sweep over the rows SpMulAdd reads)."""
    g = gg.make_grid(30, 41, 6, 4) if case == "tiny30" else gg.make_case(case)
    lib = rh.load()
    st, h, keep = host_grid(g)
    assert st == 0
    try:
        dm = rh.Dims()
        assert lib.rh_grid_dims(h, C.byref(dm)) == 0
        nx = dm.n_x
        sym = dict(perm=np.empty(nx, np.int32), bus_order=np.empty(g.n_bus - 1, np.int32),
                   level=np.empty(g.n_bus - 1, np.int32), Lp=np.empty(nx + 1, np.int32),
                   Lj=np.empty(dm.nnz_l, np.int32), Up=np.empty(nx + 1, np.int32), Uj=np.empty(dm.nnz_u, np.int32))
        assert lib.rh_grid_symbolic(h, *[rh._ptr(sym[k]) for k in ("perm", "bus_order", "level", "Lp", "Lj", "Up",
                                                                   "Uj")]) == 0
        a, e = C.c_double(), C.c_double()
        assert lib.rh_reduced_hessian_flops(h, n_sm, C.byref(a), C.byref(e)) == 0
        assert lib.rh_reduced_hessian_flops(h, 0, C.byref(a), C.byref(e)) == rh.RH_EINVAL   # no device to ask
        assert lib.rh_reduced_hessian_flops(h, n_sm, C.byref(a), C.byref(e)) == 0
    finally:
        lib.rh_grid_destroy(h)
    np_, n_bus = dm.n_p, g.n_bus
    Lp, Up, Uj = sym["Lp"], sym["Up"], sym["Uj"]
    order = sym["bus_order"]
    nv = np.array([2 if g.bus_type[b] == 2 else 1 for b in order])
    q0 = np.concatenate([[0], np.cumsum(nv)[:-1]])
    n_el = len(order)
    pos_of_q = np.repeat(np.arange(n_el), nv)
    fwd = nv * (Lp[q0 + 1] - Lp[q0]) + (nv == 2)
    bwd = nv * (Up[q0 + 1] - Up[q0] - nv) + (nv == 2)
    parent = np.array([pos_of_q[Uj[Up[q] + nv[k]]] if Up[q + 1] - Up[q] > nv[k] else -1
                       for k, q in enumerate(q0)])
    # the dense tail: the longest suffix of buses with at most dm.max_tail variables
    t_bus0 = n_el
    while t_bus0 > 0 and nx - q0[t_bus0 - 1] <= dm.max_tail:
        t_bus0 -= 1
    t0 = q0[t_bus0] if t_bus0 < n_el else nx
    T = nx - t0
    # incidences, J_p pattern (internal rows) by p column
    pairs = {(min(a_, b_), max(a_, b_)) for a_, b_ in zip(g.fr, g.to)}
    n_inc = 2 * len(pairs)
    ref = int(np.flatnonzero(g.bus_type == 0)[0])
    deg_ref = sum(1 for a_, b_ in pairs if ref in (a_, b_))
    n_gref = 1 + 2 * deg_ref
    o = OracleGrid(g)
    so = o.plant()
    _, Jp = o.jacobians_csc(so.x, so.p)
    iperm = np.empty(nx, np.int64)
    iperm[sym["perm"]] = np.arange(nx)
    jp_rows = [iperm[Jp.indices[Jp.indptr[j]:Jp.indptr[j + 1]]] for j in range(np_)]
    nnz_jp = Jp.nnz
    n_pv = int((g.bus_type == 1).sum())
    algorithmic = np_ * (4.0 * nnz_jp + 2 * (2 * dm.nnz_l + 2 * (dm.nnz_u - nx)) + 8 * n_inc + 8 * n_bus +
                         4 * n_gref + n_pv)
    assert a.value == algorithmic
    # CTA split of the two launches: 2 CTAs per SM, the first launch one slot short
    slots = 2 * n_sm
    n2 = max(min(np_, slots), -(-np_ // 256), 1)
    per = (np_ + slots - 2) // (slots - 1)
    n1 = min(n2, max(1, -(-np_ // per)))
    tailed = T > 1 and T * -(-np_ // n1) <= 4096 and T * -(-np_ // n2) <= 4096
    assert tailed
    ext = sum(nv[k] * int(np.count_nonzero(sym["Lj"][Lp[q0[k]]:Lp[q0[k] + 1]] < t0)) for k in range(t_bus0, n_el))
    tail = T * (T - 1) // 2
    need = np.zeros(n_el, bool)
    for rows in jp_rows:
        need[pos_of_q[rows]] = True
    for k in range(n_el):               # ancestors of needed buses (parents come later)
        if need[k] and parent[k] >= 0:
            need[parent[k]] = True
    sp = np.arange(t_bus0)
    lev0_pq = int(((sym["level"][:t_bus0] == 0) & (nv[:t_bus0] == 2)).sum())
    ut = int(fwd[sp][sym["level"][:t_bus0] > 0].sum())
    lt = int(bwd[sp][need[:t_bus0]].sum())
    proj = 6 * n_bus + 8 * n_inc + 4 * (1 + deg_ref) + 2 * n_gref + 1 + n_pv + 2 * lev0_pq
    l2 = proj + 2 * (ut + ext + 2 * tail + lt) + 2 * nnz_jp
    # the launches take the identity columns in the order of the lowest elimination-tree
    # postorder among each column's J_p buses (children and roots in ascending position)
    kids = [[] for _ in range(n_el)]
    roots = []
    for k in range(n_el):
        (kids[parent[k]] if parent[k] >= 0 else roots).append(k)
    post = np.zeros(n_el, np.int64)
    count = 0

    def visit(k):
        nonlocal count
        stack = [(k, 0)]
        while stack:
            b, i = stack.pop()
            if i < len(kids[b]):
                stack.append((b, i + 1))
                stack.append((kids[b][i], 0))
            else:
                post[b] = count
                count += 1
    for r in roots:
        visit(r)
    anchor = [min(post[pos_of_q[r]] for r in rows) if len(rows) else n_el for rows in jp_rows]
    order = sorted(range(np_), key=lambda j: anchor[j])
    l1 = 0.0
    for c in range(n1):
        c0, c1 = c * np_ // n1, (c + 1) * np_ // n1
        reach = np.zeros(n_el, bool)
        for j in range(c0, c1):
            reach[pos_of_q[jp_rows[order[j]]]] = True
        for k in range(t_bus0):
            if reach[k] and 0 <= parent[k] < t_bus0:
                reach[parent[k]] = True
        l = int(fwd[:t_bus0][reach[:t_bus0]].sum())
        l1 += (c1 - c0) * 2.0 * (l + ext + 2 * tail + int(bwd[sp].sum()))
    assert e.value == pytest.approx(l1 + np_ * l2, rel=1e-15)
    if case == "case9241":      # the reach and the skipped rows outweigh the dense tail
        assert e.value < a.value


def test_batch_config_is_checked_before_anything_else():
    """rh_batch_hessvec_cfg refuses a configuration outside the compiled shapes and
    the k-split caps even with no items; the defaults and every compiled value pass."""
    lib = rh.load()
    bad = [(-1, 0, 0), (0, 64, 0), (0, 320, 0), (0, 512, 0), (0, 0, 3), (0, 0, 64), (0, 0, -2)]
    for w, t, k in bad:
        cfg = rh.HvConfig(w, t, k)
        assert lib.rh_batch_hessvec_cfg(0, None, C.byref(cfg), None) == rh.RH_EINVAL, (w, t, k)
    assert lib.rh_batch_hessvec_cfg(0, None, None, None) == rh.RH_EINVAL
    for t in (0, 128, 192, 256, 384):
        for k in (0, 1, 2, 4, 8, 16, 32):
            cfg = rh.HvConfig(4, t, k)
            assert lib.rh_batch_hessvec_cfg(0, None, C.byref(cfg), None) == rh.RH_OK, (t, k)
    assert lib.rh_batch_hessvec(0, None, -1, None) == rh.RH_EINVAL
    assert lib.rh_batch_hessvec(0, None, 8, None) == rh.RH_OK


@pytest.mark.parametrize("case", ["tiny9", "tiny30", "case118", "case1354", "case2869", "case9241"])
def test_default_dense_tail_bound(case):
    """max_tail = 0 takes 16 * max(1, round(sqrt(n_x) / 16)) (about the top separator of a
    near-planar grid, in whole 16-column tiles); an explicit bound is kept; the tail holds
    at most that many variables, and the symbolic data do not depend on it."""
    import math
    g = gg.make_grid(9, 12, 3, 2) if case == "tiny9" else gg.make_grid(30, 41, 6, 4) if case == "tiny30" \
        else gg.make_case(case)
    lib = rh.load()
    for bound in (0, 40):
        st, h, keep = host_grid(g, bound)
        assert st == 0, lib.rh_last_error()
        try:
            dm = rh.Dims()
            assert lib.rh_grid_dims(h, C.byref(dm)) == 0
            want = bound or 16 * max(1, int(math.floor(math.sqrt(dm.n_x) / 16.0 + 0.5)))
            assert dm.max_tail == want
            assert 0 <= dm.tail_vars <= want
        finally:
            lib.rh_grid_destroy(h)
