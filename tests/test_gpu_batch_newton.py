"""Batched Newton power flow (rh_batch_powerflow): load scenarios of one topology
re-solved together, one host synchronisation per iteration for all of them.

* Eight scenarios of the 1354-bus grid (per-bus loads x U[0.9, 1.1], the reading
  R20): every item's x matches the oracle's Newton on the same loads at 1e-11,
  and the batched refactorisation and solves give the same x, bit for bit, as
  rh_powerflow on each grid alone.
* From a flat start on the 118-bus grid with max_iter = 1, every item stops with
  RH_ENOCONV after one step; a second call continues and converges.
* Grids of another topology, a repeated grid or more than 32 items are refused.
"""
import numpy as np
import pytest

from oracle import OracleGrid
from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu


def scenario_grids(name, n):
    from paper_2201_00241_gb300 import rh
    g = gg.make_case(name)
    scales = gg.load_scales(g.n_bus, n, g.seed)
    grids, loads = [], []
    for k in range(n):
        lg = rh.Grid(g, device=0)
        st = lg.plant()
        pd, qd = st.pd * scales[k], st.qd * scales[k]
        lg.set_state(st.p, pd, qd)
        grids.append(lg)
        loads.append((st, pd, qd))
    return g, grids, loads, scales


def test_eight_scenarios_match_oracle_and_single_solves():
    from paper_2201_00241_gb300 import rh
    g, grids, loads, scales = scenario_grids("case1354", 8)
    xs, iters, resid, status = rh.batch_powerflow(grids, x0=[st.x for st, _, _ in loads])
    assert (status == rh.RH_OK).all() and (resid <= 1e-12).all() and (iters >= 2).all()
    o = OracleGrid(g)
    so = o.plant()          # the oracle plants its own loads; both sides scale them alike
    xo_all = []
    for k in range(8):
        xo, s, _, _ = o.newton(so.p, so.pd * scales[k], so.qd * scales[k], so.x)
        assert s == 0
        xo_all.append(xo)
        assert np.abs(xs[k] - xo).max() <= 1e-11 * np.abs(xo).max()
    # the same grids, each alone
    _, grids2, loads2, _ = scenario_grids("case1354", 8)
    for k, lg in enumerate(grids2):
        x1, it1, res1, _ = lg.powerflow(loads2[k][0].x)
        assert it1 == iters[k] and np.array_equal(x1, xs[k])
    # the grid state after the batch is ready for the adjoint and HW
    lam, grad, F = grids[3].adjoint()
    W = gg.random_directions(grids[3].n_p, 4, 3)
    HW = grids[3].hessvec(W)
    HWo = o.hessvec(xo_all[3], so.p, so.pd * scales[3], so.qd * scales[3], W)
    assert np.abs(HW - HWo).max() <= 1e-10 * np.abs(HWo).max()


def test_flat_start_one_step_then_resume():
    from paper_2201_00241_gb300 import rh
    _, grids, loads, _ = scenario_grids("case118", 5)
    xs, iters, resid, status = rh.batch_powerflow(grids, x0=None, max_iter=1)
    assert (status == rh.RH_ENOCONV).all() and (iters == 1).all() and (resid > 1e-12).all()
    xs, iters, resid, status = rh.batch_powerflow(grids, x0=None, max_iter=20)
    assert (status == rh.RH_OK).all() and (resid <= 1e-12).all()
    for k in range(5):
        lg = rh.Grid(gg.make_case("case118"), device=0)
        lg.set_state(loads[k][0].p, loads[k][1], loads[k][2])
        x1, _, _, _ = lg.powerflow(None)
        assert np.abs(x1 - xs[k]).max() <= 1e-11


def test_refused_batches():
    import ctypes as C
    from paper_2201_00241_gb300 import rh
    _, grids, _, _ = scenario_grids("case118", 2)
    other = rh.Grid(gg.make_grid(30, 41, 6, 4), device=0)
    lib = rh.load()
    hs = (C.c_void_p * 2)(grids[0]._h.value, other._h.value)
    assert lib.rh_batch_powerflow(2, hs, None, 1e-12, 5, None, None, None, None) == rh.RH_EINVAL
    hs = (C.c_void_p * 2)(grids[0]._h.value, grids[0]._h.value)
    assert lib.rh_batch_powerflow(2, hs, None, 1e-12, 5, None, None, None, None) == rh.RH_EINVAL
    hs = (C.c_void_p * 33)(*([grids[0]._h.value] * 33))
    assert lib.rh_batch_powerflow(33, hs, None, 1e-12, 5, None, None, None, None) == rh.RH_EINVAL
    assert lib.rh_batch_powerflow(0, None, None, 1e-12, 5, None, None, None, None) == rh.RH_OK
