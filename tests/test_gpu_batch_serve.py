"""GPU tests of the batched, differentiable and served forms (through the C ABI).

* rh_batch_hessvec: every item of a mixed batch (grids of different sizes, two
  load scenarios of one topology) equals rh_hessvec on its own, for several
  interleave widths, also when the launch is captured in a CUDA graph and
  replayed; one item against the oracle.
* ReducedObjective: backward = reduced gradient, double backward = HW,
  checked against central differences (step 1e-6) of the reduced gradient over
  32 random directions on the 1354-bus grid, and against rh_hessvec.
* RHServer: a request's result is the same alone and in a mix of concurrent
  requests; admission by memory budget defers requests without changing results.
"""
import numpy as np
import pytest

from oracle import OracleGrid
from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def ready(name, scale=None, seed_scale=0):
    from paper_2201_00241_gb300 import rh
    g = gg.make_case(name)
    lg = rh.Grid(g, device=0)
    st = lg.plant()
    pd, qd = st.pd, st.qd
    if scale is not None:
        s = gg.load_scales(g.n_bus, seed_scale + 1, g.seed)[seed_scale]
        pd, qd = pd * s, qd * s
    lg.set_state(st.p, pd, qd)
    lg.powerflow(st.x)
    lg.adjoint()
    return lg


def colmajor(W):
    return torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()


@pytest.fixture(scope="module")
def grids():
    return {"g118": ready("case118"), "g1354a": ready("case1354", scale=True, seed_scale=0),
            "g1354b": ready("case1354", scale=True, seed_scale=1), "g2869": ready("case2869"),
            "g9241": ready("case9241")}


@pytest.mark.parametrize("width", [0, 4, 16])
def test_batch_equals_individual(grids, width):
    from paper_2201_00241_gb300 import rh
    spec = [("g118", 5), ("g1354a", 64), ("g1354b", 64), ("g2869", 33), ("g1354a", 7)]
    items, refs, outs = [], [], []
    for k, (name, N) in enumerate(spec):
        lg = grids[name]
        W = gg.random_directions(lg.n_p, N, 50 + k)
        refs.append(lg.hessvec(W))
        HW = torch.empty((N, lg.n_p), dtype=torch.float64, device="cuda").t()
        work = torch.empty(rh.work_doubles(lg, N), dtype=torch.float64, device="cuda")
        items.append((lg, colmajor(W), HW, work))
        outs.append(HW)
    rh.batch_hessvec(items, width)
    torch.cuda.synchronize()
    for ref, out in zip(refs, outs):
        assert rel(out.cpu().numpy(), ref) <= 1e-12
    # two load scenarios really are different states
    assert rel(refs[1], refs[2]) > 1e-6


def test_batch_item_against_oracle(grids):
    from paper_2201_00241_gb300 import rh
    lg = grids["g1354b"]
    g = gg.make_case("case1354")
    o = OracleGrid(g)
    so = o.plant()
    s = gg.load_scales(g.n_bus, 2, g.seed)[1]
    xo, st, _, _ = o.newton(so.p, so.pd * s, so.qd * s, so.x)
    W = gg.random_directions(lg.n_p, 16, 99)
    HW = torch.empty((16, lg.n_p), dtype=torch.float64, device="cuda").t()
    rh.batch_hessvec([(lg, colmajor(W), HW, None)], 4)
    torch.cuda.synchronize()
    assert rel(HW.cpu().numpy(), o.hessvec(xo, so.p, so.pd * s, so.qd * s, W)) <= 1e-10


def test_batch_launch_captured_in_a_cuda_graph(grids):
    from paper_2201_00241_gb300 import rh
    lg_a, lg_b = grids["g1354a"], grids["g1354b"]
    Wa = colmajor(gg.random_directions(lg_a.n_p, 64, 1))
    Wb = colmajor(gg.random_directions(lg_b.n_p, 64, 2))
    HWa = torch.empty((64, lg_a.n_p), dtype=torch.float64, device="cuda").t()
    HWb = torch.empty((64, lg_b.n_p), dtype=torch.float64, device="cuda").t()
    wa = torch.empty(rh.work_doubles(lg_a, 64), dtype=torch.float64, device="cuda")
    wb = torch.empty(rh.work_doubles(lg_b, 64), dtype=torch.float64, device="cuda")
    items = [(lg_a, Wa, HWa, wa), (lg_b, Wb, HWb, wb)]
    rh.batch_hessvec(items, 8)                       # warm-up outside capture
    torch.cuda.synchronize()
    ref_a, ref_b = HWa.cpu().numpy(), HWb.cpu().numpy()
    graph = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(graph, stream=s):
            rh.batch_hessvec(items, 8, stream=rh.C.c_void_p(s.cuda_stream))
    HWa.zero_()
    HWb.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert np.array_equal(HWa.cpu().numpy(), ref_a) and np.array_equal(HWb.cpu().numpy(), ref_b)


def test_reduced_objective_autograd_against_finite_differences():
    from paper_2201_00241_gb300.autograd import reduced_objective, _ensure_state
    from paper_2201_00241_gb300 import rh
    g = gg.make_case("case1354")
    lg = rh.Grid(g)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x)
    lg._ad_x = st.x
    p0 = torch.tensor(st.p, dtype=torch.float64, requires_grad=True)
    F = reduced_objective(p0, lg)
    grad = torch.autograd.grad(F, p0, create_graph=True)[0]
    lam, grad_ref, F_ref = lg.adjoint()
    assert float(F.detach()) == pytest.approx(F_ref, rel=1e-14)
    assert rel(grad.detach().numpy(), grad_ref) <= 1e-14
    W = gg.random_directions(lg.n_p, 32, 1354)
    h = 1e-6
    worst_fd, worst_hv = 0.0, 0.0
    for j in range(32):
        w = torch.tensor(W[:, j])
        hv = torch.autograd.grad(grad, p0, grad_outputs=w, retain_graph=True)[0].numpy()
        hv_ref = lg.hessvec(W[:, j:j + 1])[:, 0] if j % 8 == 0 else None
        gp, gm = [], []
        for sign, out in ((1.0, gp), (-1.0, gm)):
            _ensure_state(lg, torch.tensor(st.p + sign * h * W[:, j]))
            out.append(lg._ad_grad.copy())
        fd = (gp[0] - gm[0]) / (2 * h)
        worst_fd = max(worst_fd, rel(hv, fd))
        if hv_ref is not None:
            worst_hv = max(worst_hv, rel(hv, hv_ref))
    assert worst_fd <= 1e-5
    assert worst_hv <= 1e-12


def test_autograd_on_the_device_and_in_blocks():
    # p on the GPU: the double backward runs rh_hessvec on device pointers; a block of
    # directions is one launch; both equal the host-buffer products
    from paper_2201_00241_gb300.autograd import reduced_objective, reduced_hessian_vector_products
    from paper_2201_00241_gb300 import rh
    g = gg.make_case("case1354")
    lg = rh.Grid(g)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x)
    lg._ad_x = st.x
    p0 = torch.tensor(st.p, dtype=torch.float64, device="cuda", requires_grad=True)
    F = reduced_objective(p0, lg)
    grad = torch.autograd.grad(F, p0, create_graph=True)[0]
    assert grad.is_cuda
    W = gg.random_directions(lg.n_p, 24, 2024)
    ref = lg.hessvec(W)                                       # host buffers, one call
    for j in (0, 7, 23):
        hv = torch.autograd.grad(grad, p0, grad_outputs=torch.tensor(W[:, j], device="cuda"),
                                 retain_graph=True)[0]
        assert hv.is_cuda
        assert rel(hv.cpu().numpy(), ref[:, j]) <= 1e-12
    HW = reduced_hessian_vector_products(p0, lg, torch.tensor(W, device="cuda"))
    assert HW.is_cuda and tuple(HW.shape) == (lg.n_p, 24)
    assert rel(HW.cpu().numpy(), ref) <= 1e-12


def test_server_result_alone_equals_in_the_mix(grids):
    from paper_2201_00241_gb300.server import RHServer
    srv = RHServer(device=0, budget_bytes=6 << 30, max_batch=8, n_streams=3)
    try:
        for k, v in grids.items():
            srv.register(k, v)
        probe_W = gg.random_directions(grids["g1354a"].n_p, 37, 4242)
        alone = srv.submit("g1354a", probe_W).result(timeout=120)
        probe9 = gg.random_directions(grids["g9241"].n_p, 50, 4343)
        alone9 = srv.submit("g9241", probe9).result(timeout=120)
        rng = np.random.default_rng(7)
        names = list(grids)
        futs, ws = [], []
        for i in range(40):
            name = names[rng.integers(len(names))]
            W = gg.random_directions(grids[name].n_p, int(rng.integers(1, 97)), 500 + i)
            futs.append((name, srv.submit(name, W)))
            ws.append(W)
            if i == 20:
                mixed = srv.submit("g1354a", probe_W)
                mixed9 = srv.submit("g9241", probe9)
        results = [(name, f.result(timeout=300)) for name, f in futs]
        in_mix = mixed.result(timeout=300)
        assert rel(in_mix, alone) <= 1e-12
        assert rel(mixed9.result(timeout=300), alone9) <= 1e-12
        for (name, hw), W in list(zip(results, ws))[::7]:
            assert rel(hw, grids[name].hessvec(W)) <= 1e-12
        st = srv.stats()
        assert st["requests"] == 44 and st["batches"] >= 2
    finally:
        srv.close()


def test_server_admission_budget_defers_without_changing_results(grids):
    from paper_2201_00241_gb300.server import RHServer
    from paper_2201_00241_gb300 import rh
    lg = grids["g2869"]
    N = 64
    one = 8 * (rh.work_doubles(lg, N) + 2 * lg.n_p * N)
    srv = RHServer(device=0, budget_bytes=int(2.5 * one), max_batch=8, n_streams=2)
    try:
        srv.register("g", lg)
        ws = [gg.random_directions(lg.n_p, N, 900 + i) for i in range(10)]
        futs = [srv.submit("g", W) for W in ws]
        for W, f in zip(ws, futs):
            assert rel(f.result(timeout=300), lg.hessvec(W)) <= 1e-12
        assert srv.stats()["waited_for_budget"] > 0
        # a request larger than an arena is refused on its future, and the server goes on
        big = srv.submit("g", gg.random_directions(lg.n_p, 4 * N, 999))
        with pytest.raises(ValueError):
            big.result(timeout=60)
        ok = srv.submit("g", ws[0])
        assert rel(ok.result(timeout=300), lg.hessvec(ws[0])) <= 1e-12
    finally:
        srv.close()
