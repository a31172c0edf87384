"""GPU parity of rh_reduced_hessian: Jacobians, refactorisation, adjoint (eq. 7) and
the full reduced Hessian (Algorithm 2 with W = I) in one call, with the adjoint's
transposed solve running beside the first direction sweeps.

* H against the oracle's Hessian (all columns, on every grid up to the 9241-bus
  benchmark grid) at 1e-10 of max|H|, the tolerance of every HW parity test;
* on a lossless 9241-bus grid, H against the closed form that the reduced
  formulation fixes (eq. 5, eq. 10): H[Pg_k, Pg_l] = c''_k delta_kl + c''_slack,
  zero rows and columns for v, through the reach-restricted first launch and
  the CTA split of the benchmark;
* F, grad F against the oracle and against rh_adjoint (the single solve of the
  fused call runs in another thread shape, so its sums may round differently:
  1e-12);
* H against the separate rh_adjoint + rh_hessian calls at 1e-12 (the first
  direction launch has fewer CTAs, which may change how a narrow level's rows
  are split);
* the grid is left ready for rh_hessvec, device outputs, re-capture for a new
  output buffer, the kernel count and the timing query, argument errors.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import OracleGrid
from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL_HW = 1e-10


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def ready(case, scale=1.0):
    from paper_2201_00241_gb300 import rh
    g = gg.make_grid(30, 41, 6, 4) if case == "tiny30" else gg.make_case(case)
    o = OracleGrid(g)
    st = o.plant()
    pd, qd = scale * st.pd, scale * st.qd
    xo, s, _, _ = o.newton(st.p, pd, qd, st.x)
    assert s == 0
    lg = rh.Grid(g, device=0)
    lg.set_state(st.p, pd, qd)
    lg.powerflow(st.x)
    return o, st, pd, qd, xo, lg


@pytest.mark.parametrize("case,scale", [("tiny30", 1.0), ("case118", 1.0), ("case1354", 1.05)])
def test_reduced_hessian_matches_oracle(case, scale):
    o, st, pd, qd, xo, lg = ready(case, scale)
    H, grad, F = lg.reduced_hessian()
    _, grad_o, F_o = o.adjoint(xo, st.p, pd, qd)
    Ho = o.hessvec(xo, st.p, pd, qd, np.eye(lg.n_p))
    assert rel(H, Ho) <= TOL_HW
    assert rel(grad, grad_o) <= 1e-10 and F == pytest.approx(F_o, rel=1e-12)


def test_reduced_hessian_equals_separate_calls_case9241():
    """The benchmark workload: the fused call (the launch configuration the benchmark
    times) against the oracle on all 2889 columns, against rh_adjoint + rh_hessian on
    the same state, and rh_hessvec afterwards."""
    o, st, pd, qd, xo, lg = ready("case9241")
    H, grad, F = lg.reduced_hessian()
    Ho = o.hessvec(xo, st.p, pd, qd, np.eye(lg.n_p))
    assert rel(H, Ho) <= TOL_HW
    _, grad_o, F_o = o.adjoint(xo, st.p, pd, qd)
    assert rel(grad, grad_o) <= 1e-10 and F == pytest.approx(F_o, rel=1e-12)
    lam2, grad2, F2 = lg.adjoint()
    H2 = lg.hessian(block_n=256, concurrent=True)
    assert rel(H, H2) <= 1e-12
    assert rel(grad, grad2) <= 1e-12 and F == pytest.approx(F2, rel=1e-14)
    # again, after the grid's own adjoint graph ran: the fused graph is reused
    H3, _, _ = lg.reduced_hessian()
    assert rel(H3, H) <= 1e-12
    W = gg.random_directions(lg.n_p, 4, 5)
    assert rel(lg.hessvec(W), H @ W) <= 1e-11


def test_reduced_hessian_lossless_closed_form_case9241():
    """With every r = 0 the losses vanish and F(p) = sum_PV c_k(Pg_k) + c_slack(sum Pd -
    sum_PV Pg_k) exactly, so H[Pg_k, Pg_l] = c''_k delta_kl + c''_slack and every v row
    and column of H is zero, although lambda, the Lagrangian Hessian, Z and Psi are
    not.  Checked through rh_reduced_hessian at the benchmark size, so the reach
    restriction and the CTA split of both direction launches are pinned by a fact of
    the reduced formulation, not by the oracle."""
    g = gg.make_case("case9241", lossless=True)
    from paper_2201_00241_gb300 import rh
    lg = rh.Grid(g, device=0)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x)
    H, _, _ = lg.reduced_hessian()
    _, _, ip_v, ip_pg = lg.index_maps()
    S = g.base_mva
    ref = int(np.flatnonzero(g.bus_type == 0)[0])
    pv = np.flatnonzero(ip_pg >= 0)
    ng = int((ip_v >= 0).sum())
    expect = np.zeros((lg.n_p, lg.n_p))
    expect[ng:, ng:] = 2 * g.c2[ref] * S * S
    expect[ip_pg[pv], ip_pg[pv]] += 2 * g.c2[pv] * S * S
    assert rel(H, expect) <= 1e-9


def test_device_output_recapture_counts_and_timing():
    from paper_2201_00241_gb300 import rh
    o, st, pd, qd, xo, lg = ready("case1354", 0.97)
    lib = rh.load()
    assert lib.rh_reduced_hessian_times(lg._h, (C.c_float * 3)()) == rh.RH_ESTATE
    dm = rh.Dims()
    assert lib.rh_grid_dims(lg._h, C.byref(dm)) == 0 and dm.hessian_kernels == 0
    Hh, _, _ = lg.reduced_hessian()
    n = lg.n_p
    outs = [torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda:0").t() for _ in range(2)]
    for out in outs:                      # a new output pointer: captured again
        lg.reduced_hessian(out=out)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), Hh) <= 1e-12
    lg.adjoint()
    assert lib.rh_grid_dims(lg._h, C.byref(dm)) == 0
    # + the two direction launches and the rescaling of the adjoint solve (run as a direction CTA
    # on the unit-diagonal factors, it yields D lambda)
    assert dm.setup_kernels > 2 and dm.hessian_kernels == dm.setup_kernels + 3
    total, first, adj = lg.reduced_hessian_times()
    assert 0.0 < first < total < 1e4 and 0.0 < adj < total
    # a wider rh_hessvec grows (reallocates) the workspace: the graph is captured again
    W = gg.random_directions(n, 2 * n + 3, 11)
    HW = lg.hessvec(W)
    assert rel(HW, Hh @ W) <= 1e-11
    H2, _, _ = lg.reduced_hessian()
    assert rel(H2, Hh) <= 1e-12
    # a padded leading dimension
    Hp = torch.zeros((n + 5) * n, dtype=torch.float64, device="cuda:0")
    st_ptr = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rh._check(lib.rh_reduced_hessian(lg._h, C.c_void_p(Hp.data_ptr()), n + 5, None, None, st_ptr,
                                     rh.RH_DEVICE_PTRS))
    torch.cuda.synchronize()
    Hpad = Hp.view(n, n + 5).cpu().numpy().T[:n, :]
    assert rel(Hpad, Hh) <= 1e-12


def test_reduced_hessian_argument_errors():
    from paper_2201_00241_gb300 import rh
    o, st, pd, qd, xo, lg = ready("case118")
    lib = rh.load()
    H = np.empty((lg.n_p, lg.n_p), order="F")
    assert lib.rh_reduced_hessian(None, rh._ptr(H), lg.n_p, None, None, None, 0) == rh.RH_EINVAL
    assert lib.rh_reduced_hessian(lg._h, None, lg.n_p, None, None, None, 0) == rh.RH_EINVAL
    assert lib.rh_reduced_hessian(lg._h, rh._ptr(H), lg.n_p - 1, None, None, None, 0) == rh.RH_EINVAL
    assert lib.rh_reduced_hessian_times(lg._h, None) == rh.RH_EINVAL
    # the refused calls changed nothing: without an adjoint the grid still refuses rh_hessvec
    W = np.eye(lg.n_p)[:, :2].copy(order="F")
    with pytest.raises(rh.RHError):
        lg.hessvec(W)
