"""GPU parity of the real-time tracking step (section 6.3, eq. 18-19) through the C ABI.

* rh_potrf against the oracle's Cholesky on seeded SPD matrices whose sizes
  span one tile, several tiles and ragged tails of both tile widths (16 up to
  n = 2048, 32 above), with padded leading dimensions; the strictly upper
  triangle must come back untouched (bit-exact); the first bad pivot of an
  indefinite matrix must be the oracle's (bit-exact integer); matrices scaled
  by powers of two far beyond the square root of the FP64 range factor to the
  scaled oracle factor.
* rh_potrs against the oracle's solve for 1 to 17 right-hand sides.
* rh_rto_step on the 1354-bus grid (the paper's Table 3 workload) against the
  oracle's tracking step, the applied form against rh_set_state with the same
  parameters, and the refusal of an indefinite reduced Hessian.

Tolerances follow from the arithmetic: a Cholesky factor computed in another
summation order differs by about n * eps * cond(A) relative to max|L|; the
test allows 8 n eps cond(A).  The step d = -H^{-1} g inherits the relative
difference of the two reduced Hessians (1e-10, the Hessian-vector parity
bound) times cond(H).
"""
import numpy as np
import pytest

from oracle import OracleGrid, cholesky, cholesky_solve
from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
EPS = np.finfo(float).eps
TOL_HW = 1e-10


def spd(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    return A @ A.T / max(n, 1) + np.eye(n)


def to_device(M, ld=None):
    """Column-major device copy of M with leading dimension ld (>= rows)."""
    n, m = M.shape
    ld = ld or max(n, 1)
    buf = torch.full((m, ld), 7.0, dtype=torch.float64, device="cuda")
    buf[:, :n] = torch.from_numpy(np.ascontiguousarray(M.T))
    return buf.t()[:n, :], buf


@pytest.mark.parametrize("n,pad", [(1, 0), (2, 0), (15, 0), (16, 0), (17, 3), (100, 0), (519, 0), (1000, 5),
                                   (2049, 0), (2889, 7)])
def test_potrf_matches_oracle(n, pad):
    from paper_2201_00241_gb300 import rh
    H = spd(n, 1000 + n)
    A = H + np.triu(np.full((n, n), 3.25), 1)           # upper triangle: a sentinel the call must not touch
    Ad, buf = to_device(A, n + pad)
    info = rh.potrf(Ad)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    got = Ad.cpu().numpy()
    L_ref, info_ref = cholesky(H)
    assert info_ref == 0
    assert np.array_equal(np.triu(got, 1), np.triu(A, 1))
    if pad:
        assert bool((buf[:, n:] == 7.0).all())              # padding rows of every column untouched
    tol = 8 * n * EPS * np.linalg.cond(H)
    assert np.abs(np.tril(got) - L_ref).max() <= tol * np.abs(L_ref).max()


@pytest.mark.parametrize("n,spread", [(100, 0), (519, 1000), (2100, 600)])
def test_potrf_under_extreme_power_of_two_scaling(n, spread):
    # P H P with P = diag(2^k): L = P L(H) up to rounding.  Uniform 2^450 puts the
    # entries near 2^900, whose products leave the FP64 range; the spreads put the
    # diagonal between 2^-spread and 2^spread.  The kernels equilibrate each
    # diagonal tile by powers of two before their cross-multiplied eliminations.
    from paper_2201_00241_gb300 import rh
    H = spd(n, 500 + n)
    rng = np.random.default_rng(n)
    k = rng.integers(-spread // 2, spread // 2 + 1, n) if spread else np.full(n, 450)
    P = np.ldexp(1.0, k)
    Ad, _ = to_device(H * P[:, None] * P[None, :])
    info = rh.potrf(Ad)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    got = np.tril(Ad.cpu().numpy())
    assert np.all(np.isfinite(got))
    L_ref, _ = cholesky(H)
    tol = 8 * n * EPS * np.linalg.cond(H)
    assert np.abs(got / P[:, None] - L_ref).max() <= tol * np.abs(L_ref).max()


@pytest.mark.parametrize("n,bad", [(4, 2), (50, 37), (2100, 2050)])
def test_potrf_reports_the_oracles_first_bad_pivot(n, bad):
    from paper_2201_00241_gb300 import rh
    H = spd(n, 7 + n)
    H[bad, bad] = -100.0 * np.abs(H).max()               # Schur pivot at `bad` is strongly negative
    _, info_ref = cholesky(H)
    assert info_ref == bad + 1
    Ad, _ = to_device(H)
    info = rh.potrf(Ad)
    torch.cuda.synchronize()
    assert int(info.item()) == info_ref
    # columns before the bad pivot are a valid factor
    L_ref, _ = cholesky(H[:bad, :bad])
    got = np.tril(Ad.cpu().numpy()[:bad, :bad])
    assert np.abs(got - L_ref).max() <= 8 * n * EPS * np.linalg.cond(H[:bad, :bad]) * np.abs(L_ref).max()


def test_potrf_empty_matrix_sets_info_to_zero():
    from paper_2201_00241_gb300 import rh
    info = torch.full((1,), 5, dtype=torch.int32, device="cuda")
    A = torch.empty((0, 0), dtype=torch.float64, device="cuda")
    rh.potrf(A, info=info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0


@pytest.mark.parametrize("n,nrhs", [(1, 1), (17, 3), (519, 1), (519, 17), (2049, 2), (2889, 1)])
def test_potrs_matches_oracle(n, nrhs):
    from paper_2201_00241_gb300 import rh
    H = spd(n, 3000 + n)
    L_ref, _ = cholesky(H)
    B = np.random.default_rng(n).standard_normal((n, nrhs))
    X_ref = cholesky_solve(L_ref, B)
    Ld, _ = to_device(L_ref)
    Bd, _ = to_device(B, n + 2)
    rh.potrs(Ld, Bd)
    torch.cuda.synchronize()
    tol = 8 * n * EPS * np.linalg.cond(H)
    assert np.abs(Bd.cpu().numpy() - X_ref).max() <= tol * np.abs(X_ref).max()


def ready(case, scale=1.05):
    from paper_2201_00241_gb300 import rh
    g = gg.make_case(case) if isinstance(case, str) else gg.make_grid(*case)
    o = OracleGrid(g)
    st = o.plant()
    pd, qd = scale * st.pd, scale * st.qd
    lg = rh.Grid(g, device=0)
    lg.set_state(st.p, pd, qd)
    lg.powerflow(st.x)
    lg.adjoint()
    return g, o, st, pd, qd, lg


def test_rto_step_matches_oracle_on_1354_bus_grid():
    g, o, st, pd, qd, lg = ready("case1354")
    x_ref, s, _, _ = o.newton(st.p, pd, qd, st.x)
    assert s == 0
    ref = o.rto_step(x_ref, st.p, pd, qd)
    d, p_next, H, info = lg.rto_step()
    assert info == 0
    d, p_next, H = d.cpu().numpy(), p_next.cpu().numpy(), H.cpu().numpy()
    cond = np.linalg.cond(ref["H"])
    assert np.abs(d - ref["d"]).max() <= 2 * cond * TOL_HW * np.abs(ref["d"]).max()
    assert np.array_equal(p_next, st.p + d)                       # the same IEEE additions
    iu = np.triu_indices(lg.n_p, 1)
    assert np.abs(H[iu] - ref["H"][iu]).max() <= TOL_HW * np.abs(ref["H"]).max()   # upper triangle: H itself
    L_ref = ref["L"]
    assert np.abs(np.tril(H) - L_ref).max() <= 2 * cond * TOL_HW * np.abs(L_ref).max()


def test_rto_step_apply_equals_setting_the_parameters():
    """RH_RTO_APPLY must leave the grid exactly as rh_set_state(p_next) would:
    the residual ||g(x, p_next)|| at a fixed x (max_iter = 0: no Newton step,
    so no convergence is needed) and F, grad F there agree bit for bit."""
    from paper_2201_00241_gb300 import rh
    g, o, st, pd, qd, lg = ready("case118")
    x0, _, _, _ = lg.powerflow()
    lg.adjoint()
    d, p_next, _, info = lg.rto_step(apply=True)
    assert info == 0
    with pytest.raises(rh.RHError):
        lg.hessvec(np.eye(lg.n_p)[:, :1])          # the adjoint was invalidated
    other = rh.Grid(g, device=0)
    other.set_state(p_next.cpu().numpy(), pd, qd)

    def probe(grid):
        _, _, res, _ = grid.powerflow(x0, max_iter=0, raise_on_noconv=False)
        _, gr, F = grid.adjoint()
        return res, gr, F

    ra, ga, Fa = probe(lg)
    rb, gb, Fb = probe(other)
    assert ra == rb and Fa == Fb and np.array_equal(ga, gb)
    # the parameters before the step give a different residual
    before = rh.Grid(g, device=0)
    before.set_state(st.p, pd, qd)
    assert probe(before)[0] != ra
    # rh_set_state(p = NULL) keeps the applied parameters
    lg.set_state(None, pd, qd)
    rc, gc, Fc = probe(lg)
    assert rc == rb and Fc == Fb and np.array_equal(gc, gb)


def test_rto_step_refuses_an_indefinite_reduced_hessian_and_keeps_p():
    """30-bus seed-4 grid: H_00 < 0 at the planted point, so the first pivot fails
    (the oracle's answer too); with RH_RTO_APPLY the parameters stay as they were."""
    from paper_2201_00241_gb300 import rh
    g = gg.make_grid(30, 41, 6, 4)
    o = OracleGrid(g)
    st = o.plant()
    H_ref = o.hessvec(st.x, st.p, st.pd, st.qd, np.eye(o.n_p))
    assert cholesky(H_ref)[1] == 1
    lg = rh.Grid(g, device=0)
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x)
    _, g_before, _ = lg.adjoint()
    _, _, _, info = lg.rto_step(apply=True)
    assert info == 1
    lg.powerflow(st.x)
    _, g_after, _ = lg.adjoint()
    assert np.array_equal(g_before, g_after)
