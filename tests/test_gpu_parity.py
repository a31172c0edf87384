"""GPU parity: every step of the CUDA path against the CPU oracle, through the C ABI.

Tolerance (floating point): ||HW_gpu - HW_oracle||_max / ||HW_oracle||_max <= 1e-10,
normwise over the block; intermediate quantities are held to tighter bounds where
the arithmetic allows.  Integer/symbolic data is compared bit for bit
(tests/test_abi.py).  Both sides plant the loads with their own injection code.
"""
import numpy as np
import pytest

from oracle import OracleGrid
from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu

TOL_HW = 1e-10


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


_cache = {}


def setup_case(name, lossless=False, scale=None):
    key = (name, lossless, None if scale is None else scale.tobytes())
    if key in _cache:
        return _cache[key]
    from paper_2201_00241_gb300 import rh
    if name == "tiny30":
        g = gg.make_grid(30, 41, 6, 4, lossless=lossless)
    elif name == "tiny9":
        g = gg.make_grid(9, 12, 3, 2, lossless=lossless)
    else:
        c = gg.CASES[name]
        g = gg.make_grid(c["n_bus"], c["n_branch"], c["n_gen"], c["seed"], lossless=lossless)
    o = OracleGrid(g)
    so = o.plant()
    lg = rh.Grid(g, device=0)
    sl = lg.plant()
    pd_o, qd_o, pd_l, qd_l = so.pd, so.qd, sl.pd, sl.qd
    if scale is not None:
        pd_o, qd_o, pd_l, qd_l = pd_o * scale, qd_o * scale, pd_l * scale, qd_l * scale
    x_o, st, _, _ = o.newton(so.p, pd_o, qd_o, so.x)
    assert st == 0
    lg.set_state(sl.p, pd_l, qd_l)
    x_l, iters, res, _ = lg.powerflow(sl.x)
    lam, grad, F = lg.adjoint()
    d = dict(g=g, o=o, so=so, lg=lg, sl=sl, x_o=x_o, x_l=x_l, pd_o=pd_o, qd_o=qd_o, lam=lam, grad=grad, F=F)
    _cache[key] = d
    return d


def oracle_hv(d, W):
    return d["o"].hessvec(d["x_o"], d["so"].p, d["pd_o"], d["qd_o"], W)


# ---------------------------------------------------------------------------
# step by step
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["case118", "case1354"])
def test_injections(case):
    d = setup_case(case)
    rng = np.random.default_rng(1)
    vm = rng.uniform(0.9, 1.1, d["g"].n_bus)
    va = rng.normal(0, 0.2, d["g"].n_bus)
    P, Q = d["lg"].injections(vm, va)
    Po, Qo = d["o"].injections(vm, va)
    assert rel(P, Po) <= 1e-13 and rel(Q, Qo) <= 1e-13


def test_planted_loads_agree():
    d = setup_case("case1354")
    assert rel(d["sl"].pd, d["so"].pd) <= 1e-13 and rel(d["sl"].p, d["so"].p) <= 1e-13


def test_powerflow_flat_start_recovers_planted_point():
    from paper_2201_00241_gb300 import rh
    g = gg.make_case("case118")
    lg = rh.Grid(g)
    sl = lg.plant()
    lg.set_state(sl.p, sl.pd, sl.qd)
    x, iters, res, _ = lg.powerflow(None, tol=1e-12, max_iter=20)
    assert res <= 1e-12 and iters >= 3
    assert np.abs(x - sl.x).max() <= 1e-8


def test_powerflow_matches_oracle_on_scaled_loads():
    scale = gg.load_scales(1354, 1, 20220101)[0]
    d = setup_case("case1354", scale=scale)
    assert rel(d["x_l"], d["x_o"]) <= 1e-11


@pytest.mark.parametrize("case", ["tiny30", "case118"])
def test_refactor_reproduces_permuted_jacobian(case):
    d = setup_case(case)
    lg, o = d["lg"], d["o"]
    A = lg.refactor()
    sym = lg.symbolic()
    n = lg.n_x
    L = np.eye(n)
    U = np.zeros((n, n))
    la = ua = 0
    Lp, Lj, Up, Uj = sym["Lp"], sym["Lj"], sym["Up"], sym["Uj"]
    # A is stored row by row: L part then U part
    pos = 0
    for r in range(n):
        nl, nu = Lp[r + 1] - Lp[r], Up[r + 1] - Up[r]
        L[r, Lj[Lp[r]:Lp[r + 1]]] = A[pos:pos + nl]
        U[r, Uj[Up[r]:Up[r + 1]]] = A[pos + nl:pos + nl + nu]
        pos += nl + nu
    jx, _ = o.jacobians_dense(d["x_o"], d["so"].p)
    B = jx[np.ix_(sym["perm"], sym["perm"])]
    assert rel(L @ U, B) <= 1e-12
    lg.adjoint()  # restore the hessvec-ready state for later tests


@pytest.mark.parametrize("case", ["case1354", "case9241"])
def test_refactor_sparse_product_large(case):
    """Every level of the update schedule and the closing pivot launch on the larger
    grids: L U against the permuted J_x, as sparse matrices."""
    import scipy.sparse as sp
    d = setup_case(case)
    lg, o = d["lg"], d["o"]
    A = lg.refactor()
    sym = lg.symbolic()
    n = lg.n_x
    Lp, Lj, Up, Uj = (np.asarray(sym[k], dtype=np.int64) for k in ("Lp", "Lj", "Up", "Uj"))
    # row r of A holds its L part then its U part, from position Lp[r] + Up[r]
    rows_l = np.repeat(np.arange(n), np.diff(Lp))
    rows_u = np.repeat(np.arange(n), np.diff(Up))
    L = sp.csr_matrix((A[Up[rows_l] + np.arange(len(Lj))], Lj, Lp), shape=(n, n)) + sp.identity(n, format="csr")
    U = sp.csr_matrix((A[Lp[rows_u + 1] + np.arange(len(Uj))], Uj, Up), shape=(n, n))
    Jx, _ = o.jacobians_csc(d["x_o"], d["so"].p)
    perm = np.asarray(sym["perm"])
    B = sp.csr_matrix(Jx)[perm][:, perm]
    diff = (L @ U - B).tocoo()
    assert np.abs(diff.data).max(initial=0.0) <= 1e-12 * np.abs(B.data).max()
    lg.adjoint()  # restore the hessvec-ready state for later tests


@pytest.mark.parametrize("nrhs", [1, 3, 31, 32, 33, 64])
@pytest.mark.parametrize("trans", [False, True])
def test_batched_solves(nrhs, trans):
    d = setup_case("case1354")
    R = np.random.default_rng(nrhs).normal(size=(d["lg"].n_x, nrhs))
    X = d["lg"].solve(R, trans=trans)
    Xo = d["o"].solve(d["x_o"], d["so"].p, R, trans=trans)
    assert rel(X, Xo) <= 1e-11


@pytest.mark.parametrize("case", ["tiny30", "case118", "case1354"])
def test_adjoint_and_gradient(case):
    d = setup_case(case)
    lam_o, grad_o, F_o = d["o"].adjoint(d["x_o"], d["so"].p, d["pd_o"], d["qd_o"])
    assert rel(d["lam"], lam_o) <= 1e-10
    assert rel(d["grad"], grad_o) <= 1e-10
    assert d["F"] == pytest.approx(F_o, rel=1e-12)


@pytest.mark.parametrize("case", ["tiny30", "case118"])
def test_projection_matches_explicit_lagrangian_hessian(case):
    d = setup_case(case)
    lam_o, _, _ = d["o"].adjoint(d["x_o"], d["so"].p, d["pd_o"], d["qd_o"])
    K = d["o"].lagrangian_hessian_dense(d["x_o"], d["so"].p, d["pd_o"], lam_o)
    V = np.random.default_rng(3).normal(size=(K.shape[0], 5))
    Y = d["lg"].lagrangian_hessvec(V)
    assert rel(Y, K @ V) <= 1e-11


# ---------------------------------------------------------------------------
# the composed reduced-Hessian-vector product
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N", [1, 2, 3, 31, 32, 33, 64, 255, 256])
def test_hessvec_widths_case1354(N):
    d = setup_case("case1354")
    W = gg.random_directions(d["lg"].n_p, N, 1354 + N)
    HW = d["lg"].hessvec(W)
    assert rel(HW, oracle_hv(d, W)) <= TOL_HW


@pytest.mark.parametrize("case", ["tiny9", "tiny30", "case118"])
def test_full_hessian_blocks_and_concurrent(case):
    d = setup_case(case)
    Ho = oracle_hv(d, np.eye(d["lg"].n_p))
    Hc = d["lg"].hessian(block_n=16, concurrent=True)
    Hb = d["lg"].hessian(block_n=16, concurrent=False)
    assert rel(Hc, Ho) <= TOL_HW and rel(Hb, Ho) <= TOL_HW
    assert rel(Hc, Hc.T) <= 1e-11


def test_case9241_full_size_all_columns():
    """The benchmark workload: all 2889 columns of H in one concurrent launch (blocks of
    256), every column against the oracle, symmetry on the whole matrix."""
    d = setup_case("case9241")
    lg = d["lg"]
    H = lg.hessian(block_n=256, concurrent=True)
    Ho = oracle_hv(d, np.eye(lg.n_p))
    assert rel(H, Ho) <= TOL_HW
    assert rel(H, H.T) <= 1e-10
    # and a random block of N = 256 directions (sampled columns)
    W = gg.random_directions(lg.n_p, 256, 9241)
    HW = lg.hessvec(W)
    pick = [0, 1, 100, 255]
    assert rel(HW[:, pick], oracle_hv(d, W[:, pick])) <= TOL_HW
    # per-block launches agree with the concurrent launch
    Hb = lg.hessian(block_n=256, concurrent=False)
    assert rel(Hb, H) <= 1e-12


def test_lossless_closed_form_on_gpu():
    d = setup_case("case118", lossless=True)
    g, lg = d["g"], d["lg"]
    H = lg.hessian(block_n=16)
    _, _, ip_v, ip_pg = lg.index_maps()
    S = g.base_mva
    ref = int(np.flatnonzero(g.bus_type == 0)[0])
    pv = np.flatnonzero(ip_pg >= 0)
    ng = int((ip_v >= 0).sum())
    expect = np.zeros_like(H)
    expect[ng:, ng:] = 2 * g.c2[ref] * S * S
    expect[ip_pg[pv], ip_pg[pv]] += 2 * g.c2[pv] * S * S
    assert rel(H, expect) <= 1e-9


def test_deterministic_and_column_independent():
    d = setup_case("case1354")
    lg = d["lg"]
    W = gg.random_directions(lg.n_p, 64, 7)
    a = lg.hessvec(W)
    b = lg.hessvec(W)
    assert np.array_equal(a, b)
    for j in (0, 17, 63):
        single = lg.hessvec(W[:, j:j + 1])
        assert rel(single[:, 0], a[:, j]) <= 1e-13


def test_linearity():
    d = setup_case("case118")
    lg = d["lg"]
    W = gg.random_directions(lg.n_p, 2, 11)
    hw = lg.hessvec(W)
    comb = lg.hessvec((2.0 * W[:, 0] - 3.0 * W[:, 1])[:, None])
    assert rel(comb[:, 0], 2.0 * hw[:, 0] - 3.0 * hw[:, 1]) <= 1e-12


def test_errors_and_edge_cases():
    from paper_2201_00241_gb300 import rh
    d = setup_case("tiny30")
    lg = d["lg"]
    empty = lg.hessvec(np.zeros((lg.n_p, 0)))
    assert empty.shape == (lg.n_p, 0)
    g2 = rh.Grid(d["g"])
    with pytest.raises(rh.RHError) as e:
        g2.hessvec(np.eye(g2.n_p)[:, :2])
    assert e.value.status == rh.RH_ESTATE
    lib = rh.load()
    W = np.zeros((lg.n_p, 2), order="F")
    HW = np.zeros((lg.n_p, 2), order="F")
    st = lib.rh_hessvec(lg._h, rh._ptr(W), lg.n_p - 1, 2, rh._ptr(HW), lg.n_p, None, 0)
    assert st == rh.RH_EINVAL


def test_device_pointers_and_streams():
    torch = pytest.importorskip("torch")
    d = setup_case("case1354")
    lg = d["lg"]
    W = gg.random_directions(lg.n_p, 40, 5)
    Wt = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()   # column-major view
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        HWt = lg.hessvec(Wt)
    s.synchronize()
    assert rel(HWt.cpu().numpy(), lg.hessvec(W)) <= 1e-13


@pytest.mark.parametrize("k", [0, 5])
def test_load_scenarios_case1354(k):
    """Cross-scenario workload: loads scaled per bus by U[0.9, 1.1], power flow re-solved."""
    scale = gg.load_scales(1354, 8, 20220101)[k]
    d = setup_case("case1354", scale=scale)
    W = gg.random_directions(d["lg"].n_p, 64, 1000 + k)
    assert rel(d["lg"].hessvec(W), oracle_hv(d, W)) <= TOL_HW


def test_setup_kernel_count_is_reported_after_the_first_adjoint():
    """rh_dims.setup_kernels counts the kernels of rh_adjoint's captured graph: 0
    before the first call, then the same positive number on every call."""
    import ctypes as C
    from paper_2201_00241_gb300 import rh
    lg = rh.Grid(gg.make_case("case118"), device=0)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x)
    lib = rh.load()
    dm = rh.Dims()
    assert lib.rh_grid_dims(lg._h, C.byref(dm)) == 0 and dm.setup_kernels == 0
    lg.adjoint()
    assert lib.rh_grid_dims(lg._h, C.byref(dm)) == 0
    first = dm.setup_kernels
    assert first > 5
    lg.adjoint()
    assert lib.rh_grid_dims(lg._h, C.byref(dm)) == 0 and dm.setup_kernels == first
