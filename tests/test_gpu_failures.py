"""Failure statuses of the library, each made on the host (no GPU fault, no trap).

* A PQ bus with no branch has an exactly zero 2x2 block in J_x (Y_ii = 0, no
  shunt): the static pivot check of the refactorisation sets its device flag and
  rh_adjoint, rh_powerflow and rh_reduced_hessian return RH_ESINGULAR; the grid
  then refuses rh_hessvec with RH_ESTATE.
* Newton from a flat start with max_iter = 1 returns RH_ENOCONV after one step
  and keeps its iterate: a second call continues from it and converges.
* A NaN or an infinity in column j of W stays in column j of HW: every other
  column is bit for bit what it is without it (directions are independent).
"""
import dataclasses

import numpy as np
import pytest

from oracle import OracleGrid
from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu


def isolated_bus_grid():
    g = gg.make_grid(30, 41, 6, 4)
    return dataclasses.replace(g, n_bus=31, bus_type=np.append(g.bus_type, 2).astype(np.int8),
                               v_star=np.append(g.v_star, 1.0), theta_star=np.append(g.theta_star, 0.0),
                               c2=np.append(g.c2, 0.0), c1=np.append(g.c1, 0.0))


def test_zero_pivot_gives_esingular():
    from paper_2201_00241_gb300 import rh
    lg = rh.Grid(isolated_bus_grid(), device=0)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    with pytest.raises(rh.RHError) as e:
        lg.adjoint()
    assert e.value.status == rh.RH_ESINGULAR
    with pytest.raises(rh.RHError) as e:
        lg.hessvec(np.eye(lg.n_p)[:, :2].copy(order="F"))
    assert e.value.status == rh.RH_ESTATE
    with pytest.raises(rh.RHError) as e:
        lg.reduced_hessian()
    assert e.value.status == rh.RH_ESINGULAR
    x0 = st.x.copy()
    x0[0] += 0.01                                   # a residual, so Newton has to factor
    lib = rh.load()
    x0 = np.ascontiguousarray(x0)
    s = lib.rh_powerflow(lg._h, rh._ptr(x0), 1e-12, 5, None, None, None)
    assert s == rh.RH_ESINGULAR and b"pivot" in lib.rh_last_error()
    # the same topology without the isolated bus factors fine
    ok = rh.Grid(gg.make_grid(30, 41, 6, 4), device=0)
    so = ok.plant()
    ok.set_state(so.p, so.pd, so.qd)
    ok.powerflow(so.x)
    ok.adjoint()


def test_one_newton_step_from_flat_start_is_enoconv_and_resumable():
    from paper_2201_00241_gb300 import rh
    lg = rh.Grid(gg.make_case("case118"), device=0)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    x1, it, res, status = lg.powerflow(None, tol=1e-12, max_iter=1, raise_on_noconv=False)
    assert status == rh.RH_ENOCONV and it == 1 and res > 1e-12
    with pytest.raises(rh.RHError) as e:
        lg.powerflow(None, tol=1e-12, max_iter=0)
    assert e.value.status == rh.RH_ENOCONV
    x, it, res, status = lg.powerflow(None, tol=1e-12, max_iter=20)      # continues from the iterate
    assert status == rh.RH_OK and res <= 1e-12
    assert np.abs(x - st.x).max() <= 1e-8


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_nonfinite_direction_stays_in_its_column(bad):
    from paper_2201_00241_gb300 import rh
    lg = rh.Grid(gg.make_case("case1354"), device=0)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x)
    lg.adjoint()
    W = gg.random_directions(lg.n_p, 24, 9)
    clean = lg.hessvec(W)
    Wb = W.copy(order="F")
    Wb[17, 5] = bad
    HW = lg.hessvec(Wb)
    others = [j for j in range(24) if j != 5]
    assert np.array_equal(HW[:, others], clean[:, others])
    assert not np.isfinite(HW[:, 5]).all()


def test_hessian_columns_ranges():
    """rh_hessian_columns (one launch per column block: the unit of a column partition of
    H over several GPUs) against the oracle's columns and the concurrent full H."""
    from paper_2201_00241_gb300 import rh
    from paper_2201_00241_gb300 import shard
    g = gg.make_case("case1354")
    lg = rh.Grid(g, device=0)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x)
    with pytest.raises(rh.RHError) as e:
        lg.hessian_columns(0, 3)
    assert e.value.status == rh.RH_ESTATE
    lg.adjoint()
    H = lg.hessian(block_n=256, concurrent=True)
    o = OracleGrid(g)
    so = o.plant()
    for c0, n in [(0, 100), (100, 419), (518, 1)] + [shard.column_range(lg.n_p, 3, r) for r in range(3)]:
        B = lg.hessian_columns(c0, n)
        assert np.abs(B - H[:, c0:c0 + n]).max() <= 1e-12 * np.abs(H).max()
        E = np.zeros((lg.n_p, n))
        E[c0 + np.arange(n), np.arange(n)] = 1.0
        Ho = o.hessvec(so.x, so.p, so.pd, so.qd, E)
        assert np.abs(B - Ho).max() <= 1e-10 * np.abs(Ho).max()
    assert lg.hessian_columns(5, 0).shape == (lg.n_p, 0)
    lib = rh.load()
    out = np.empty((lg.n_p, 2), order="F")
    assert lib.rh_hessian_columns(lg._h, lg.n_p - 1, 2, rh._ptr(out), lg.n_p, None, 0) == rh.RH_EINVAL
    assert lib.rh_hessian_columns(lg._h, -1, 2, rh._ptr(out), lg.n_p, None, 0) == rh.RH_EINVAL
    assert lib.rh_hessian_columns(lg._h, 0, 2, rh._ptr(out), lg.n_p - 1, None, 0) == rh.RH_EINVAL
