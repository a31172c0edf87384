"""GPU parity on a grid whose x does not fit in shared memory (n_x = 28 599 for
15 500 buses): every single solve then runs through the direction kernel on the
unit-diagonal factors J_x = D L'' U', with the right-hand side scaled by D^-1 for
J_x z = b (the Newton steps) and the result scaled by D^-1 for J_x^T psi = r (the
adjoint).  Newton from the planted point at scaled loads, lambda, grad F, two
HVPs and two sampled columns of the full reduced Hessian against the oracle at
1e-10 of their maximum (the HW tolerance of every parity test).
"""
import numpy as np
import pytest

from oracle import OracleGrid
from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def test_grid_beyond_shared_memory_solves():
    from paper_2201_00241_gb300 import rh
    g = gg.make_grid(15500, 26900, 2400, 77)
    o = OracleGrid(g)
    st = o.plant()
    pd, qd = 1.02 * st.pd, 1.02 * st.qd
    xo, s, _, _ = o.newton(st.p, pd, qd, st.x)
    assert s == 0
    lam_o, grad_o, F_o = o.adjoint(xo, st.p, pd, qd)

    lg = rh.Grid(g, device=0)
    assert lg.n_x > 28000            # beyond the single-CTA shared-memory solve
    lg.set_state(st.p, pd, qd)
    x, iters, res, _ = lg.powerflow(st.x)
    assert res <= 1e-12 and rel(x, xo) <= TOL
    lam, grad, F = lg.adjoint()
    assert rel(lam, lam_o) <= TOL and rel(grad, grad_o) <= TOL and F == pytest.approx(F_o, rel=1e-12)

    W = gg.random_directions(lg.n_p, 2, 15500)
    hw_o = o.hessvec(xo, st.p, pd, qd, W)
    assert rel(lg.hessvec(W), hw_o) <= TOL

    cols = np.array([7, lg.n_p - 3])
    E = np.zeros((lg.n_p, 2))
    E[cols, [0, 1]] = 1.0
    H, grad_f, F_f = lg.reduced_hessian()
    assert rel(H[:, cols], o.hessvec(xo, st.p, pd, qd, E)) <= TOL
    assert rel(grad_f, grad_o) <= TOL
