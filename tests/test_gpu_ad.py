"""GPU parity of the coloured forward-mode Jacobian (section 4.2.2, Fig. 2) through the C ABI.

* rh_jacobian(RH_JAC_COLORED_AD): the structural pattern of J_x and J_p equals
  the oracle's (bit-exact integers) and every value agrees with the oracle's
  analytic Jacobian, which its own tests pin by central differences, up to
  1e-13 of max|J|.  The AD sums a row's derivative over the admittance row
  where the analytic formula uses P_i or Q_i, so the two differ by rounding
  of at most (row length) * eps * max|J|; 1e-13 leaves a wide margin.  Cases:
  30 to 9241 buses, at the planted point and at scaled loads.
* the whole path with AD assembly: Newton power flow from a flat start, lambda,
  grad F and HW against the oracle, and switching the method back restores the
  analytic results bit for bit.
"""
import numpy as np
import pytest

from oracle import OracleGrid
from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL_J = 1e-13
TOL_HW = 1e-10


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def grid_of(case):
    return gg.make_grid(30, 41, 6, 4) if case == "tiny30" else gg.make_case(case)


def sorted_triplets(rows, cols, vals, n_cols):
    order = np.lexsort((cols, rows))
    return rows[order], cols[order], vals[order]


@pytest.mark.parametrize("case,scale", [("tiny30", 1.0), ("case118", 1.0), ("case1354", 1.05), ("case9241", 1.0)])
def test_ad_jacobian_matches_oracle(case, scale):
    from paper_2201_00241_gb300 import rh
    g = grid_of(case)
    o = OracleGrid(g)
    st = o.plant()
    pd, qd = scale * st.pd, scale * st.qd
    x, s, _, _ = o.newton(st.p, pd, qd, st.x)
    assert s == 0
    lg = rh.Grid(g, device=0)
    lg.set_state(st.p, pd, qd)
    lg.powerflow(st.x)
    (xr, xc, xv), (pr, pc, pv) = lg.jacobian("ad")
    Jx, Jp = o.jacobians_csc(x, st.p)
    for (r, c, v), J in (((xr, xc, xv), Jx), ((pr, pc, pv), Jp)):
        coo = J.tocoo()
        rr, cr, vr = sorted_triplets(coo.row.astype(np.int32), coo.col.astype(np.int32), coo.data, J.shape[1])
        r, c, v = sorted_triplets(r, c, v, J.shape[1])
        assert np.array_equal(r, rr) and np.array_equal(c, cr)          # the structural pattern
        assert np.abs(v - vr).max() <= TOL_J * np.abs(vr).max()
    # the analytic assembly of the library agrees as well
    (_, _, xa), (_, _, pa) = lg.jacobian("analytic")
    assert np.abs(xa - xv).max() <= TOL_J * np.abs(xa).max()
    assert np.abs(pa - pv).max() <= TOL_J * np.abs(pa).max()


def test_path_with_ad_assembly_matches_oracle_and_switches_back():
    from paper_2201_00241_gb300 import rh
    g = gg.make_case("case1354")
    o = OracleGrid(g)
    st = o.plant()
    s = gg.load_scales(g.n_bus, 1, g.seed)[0]
    pd, qd = st.pd * s, st.qd * s
    W = gg.random_directions(o.n_p, 16, 77)

    lg = rh.Grid(g, device=0)
    lg.set_state(st.p, pd, qd)
    x_an, it_an, _, _ = lg.powerflow(st.x)
    lam_an, grad_an, F_an = lg.adjoint()
    hw_an = lg.hessvec(W)

    lg.set_jacobian_method("ad")
    with pytest.raises(rh.RHError):
        lg.hessvec(W)                                   # the adjoint was invalidated
    x_ad, it_ad, res, _ = lg.powerflow(st.x)
    lam_ad, grad_ad, F_ad = lg.adjoint()
    hw_ad = lg.hessvec(W)

    xo, so, _, _ = o.newton(st.p, pd, qd, st.x)
    lam_o, grad_o, F_o = o.adjoint(xo, st.p, pd, qd)
    hw_o = o.hessvec(xo, st.p, pd, qd, W)
    assert so == 0 and it_ad == it_an and res <= 1e-12
    assert rel(x_ad, xo) <= 1e-12 and rel(lam_ad, lam_o) <= 1e-10 and rel(grad_ad, grad_o) <= 1e-10
    assert F_ad == pytest.approx(F_o, rel=1e-12)
    assert rel(hw_ad, hw_o) <= TOL_HW

    lg.set_jacobian_method("analytic")
    lg.powerflow(st.x)
    lam2, grad2, F2 = lg.adjoint()
    hw2 = lg.hessvec(W)
    assert np.array_equal(lam2, lam_an) and np.array_equal(grad2, grad_an) and F2 == F_an
    assert np.array_equal(hw2, hw_an)


def test_ad_newton_from_flat_start():
    from paper_2201_00241_gb300 import rh
    g = gg.make_case("case118")
    o = OracleGrid(g)
    st = o.plant()
    lg = rh.Grid(g, device=0)
    lg.set_jacobian_method("ad")
    lg.set_state(st.p, st.pd, st.qd)
    ix_th, ix_v, _, _ = o.index_maps()
    x0 = np.zeros(o.n_x)
    x0[ix_v[ix_v >= 0]] = 1.0
    x, it, res, _ = lg.powerflow(x0)
    assert res <= 1e-12 and it <= 8
    assert rel(x, st.x) <= 1e-10


def test_unknown_jacobian_method_is_rejected():
    from paper_2201_00241_gb300 import rh
    lg = rh.Grid(gg.make_case("case118"), device=0)
    assert rh.load().rh_set_jacobian_method(lg._h, 7) == rh.RH_EINVAL
