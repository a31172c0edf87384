"""Allocation-free reduced-Hessian-vector products (rh_hessvec_noalloc).

For callers that must not let the library allocate device memory once running
(an application that owns all device memory through its own pool, a real-time
loop that forbids allocation).  The entry point keeps its two direction buffers
in a fixed device array instead of calling cudaMalloc.  These tests call it
through the C ABI with device pointers and compare it with rh_hessvec, on two
calls in a row, so that a call that depended on what the previous call left in
the shared array would be caught.  The file is named to be collected last.
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
