"""Allocation-free reduced-Hessian-vector products (rh_hessvec_noalloc).

For callers that must not let the library allocate device memory once running
(an application that owns all device memory through its own pool, a real-time
loop that forbids allocation).  The entry point keeps its two direction buffers
in a fixed device array instead of calling cudaMalloc.  These tests call it
through the C ABI with device pointers and compare it with rh_hessvec, on two
calls in a row, so that a call that depended on what the previous call left in
the shared array would be caught; they also check that two calls on a grid
that never ran rh_hessvec leave the device's free memory unchanged, and that
padded leading dimensions read and write only the n_p rows of each column.
The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2201_00241_gb300 import gridgen as gg

pytestmark = pytest.mark.gpu

TOL_HW = 1e-10


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def ready_grid(name):
    from paper_2201_00241_gb300 import rh
    lg = rh.Grid(gg.make_case(name), device=0)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    lg.powerflow(st.x)
    lg.adjoint()
    return lg


def call_noalloc(lib, lg, Wd, N, torch):
    from paper_2201_00241_gb300 import rh
    HWd = torch.full((N, lg.n_p), float("nan"), dtype=torch.float64, device="cuda")   # column-major n_p x N
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.rh_hessvec_noalloc(lg._h, C.c_void_p(Wd.data_ptr()), lg.n_p, N, C.c_void_p(HWd.data_ptr()), lg.n_p,
                                stream)
    assert st == rh.RH_OK, lib.rh_last_error()
    torch.cuda.synchronize()
    return HWd.cpu().numpy().T


@pytest.mark.parametrize("name,N", [("case1354", 64), ("case9241", 48)])
def test_noalloc_matches_hessvec_on_two_calls(name, N):
    torch = pytest.importorskip("torch")
    from paper_2201_00241_gb300 import rh
    lib = rh.load()
    lg = ready_grid(name)
    for call in range(2):
        W = gg.random_directions(lg.n_p, N, 100 + call)
        expect = lg.hessvec(W)                                          # the existing entry point
        Wd = torch.from_numpy(np.ascontiguousarray(W.T)).cuda()           # column-major n_p x N
        got = call_noalloc(lib, lg, Wd, N, torch)
        assert np.isfinite(got).all()
        assert rel(got, expect) <= TOL_HW


def test_noalloc_allocates_nothing_on_a_fresh_grid():
    """A grid that never ran rh_hessvec has no direction workspace: two allocation-free
    calls on it must leave the device's free memory as it was, and still equal
    rh_hessvec (run only afterwards)."""
    torch = pytest.importorskip("torch")
    from paper_2201_00241_gb300 import rh
    lib = rh.load()
    # module loading and the one-time address lookup happen on another grid first
    warm = ready_grid("case118")
    Ww = torch.from_numpy(np.ascontiguousarray(gg.random_directions(warm.n_p, 4, 1).T)).cuda()
    call_noalloc(lib, warm, Ww, 4, torch)
    lg = ready_grid("case1354")
    # N = 320: a workspace rh_hessvec would allocate for it is 2 x 7.6 MB, well above the
    # granularity of the free-memory count
    N = 320
    Ws = [gg.random_directions(lg.n_p, N, 300 + k) for k in range(2)]
    Wd = [torch.from_numpy(np.ascontiguousarray(W.T)).cuda() for W in Ws]
    HWd = [torch.full((N, lg.n_p), float("nan"), dtype=torch.float64, device="cuda") for _ in Ws]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for w, h in zip(Wd, HWd):
        st = lib.rh_hessvec_noalloc(lg._h, C.c_void_p(w.data_ptr()), lg.n_p, N, C.c_void_p(h.data_ptr()), lg.n_p,
                                    stream)
        assert st == rh.RH_OK, lib.rh_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    for W, h in zip(Ws, HWd):
        assert rel(h.cpu().numpy().T, lg.hessvec(W)) <= TOL_HW


def test_noalloc_padded_leading_dimensions():
    """W and HW as the top n_p rows of wider column-major buffers (ldw = ldhw = n_p + 3):
    the padding rows, filled with NaN, are neither read nor written."""
    torch = pytest.importorskip("torch")
    from paper_2201_00241_gb300 import rh
    lib = rh.load()
    lg = ready_grid("case1354")
    N, ld = 24, lg.n_p + 3
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        W = gg.random_directions(lg.n_p, N, 500 + call)
        Wp = np.full((ld, N), np.nan, order="F")
        Wp[:lg.n_p] = W
        Wd = torch.from_numpy(np.ascontiguousarray(Wp.T)).cuda()        # column-major ld x N
        HWd = torch.full((N, ld), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.rh_hessvec_noalloc(lg._h, C.c_void_p(Wd.data_ptr()), ld, N, C.c_void_p(HWd.data_ptr()), ld, stream)
        assert st == rh.RH_OK, lib.rh_last_error()
        torch.cuda.synchronize()
        got = HWd.cpu().numpy().T
        assert np.isnan(got[lg.n_p:]).all()
        assert rel(got[:lg.n_p], lg.hessvec(W)) <= TOL_HW


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch():
    torch = pytest.importorskip("torch")
    from paper_2201_00241_gb300 import rh
    lib = rh.load()
    lg = ready_grid("case9241")
    N = 64                                                              # 64 * 19926 > 2^20 doubles
    Wd = torch.zeros((N, lg.n_p), dtype=torch.float64, device="cuda")
    HWd = torch.zeros((N, lg.n_p), dtype=torch.float64, device="cuda")
    st = lib.rh_hessvec_noalloc(lg._h, C.c_void_p(Wd.data_ptr()), lg.n_p, N, C.c_void_p(HWd.data_ptr()), lg.n_p,
                                C.c_void_p(0))
    assert st == rh.RH_EINVAL
    assert b"exceeds the fixed scratch" in lib.rh_last_error()
