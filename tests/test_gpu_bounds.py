"""Index checks on the GPU: the whole path through the index-checking build.

librh_bounds.so (the same sources compiled with -DRH_BOUNDS) checks every row,
slot and position index its kernels read or write; a failed check sets an error
word on the device and skips the access.  A child process loads that build in
place of librh.so and runs every entry point on the 30- and 118-bus grids: power
flow from a flat start, adjoint, rh_hessvec at several widths (host and device
pointers), the full Hessian by blocks and at once, the fused call, column
blocks, both batched solves, the projection, a batched launch, the
allocation-free call, the coloured Jacobian and the tracking step.  The error
word must stay 0, and HW must still match the oracle.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys, ctypes as C
import numpy as np
sys.path.insert(0, ROOT)
from paper_2201_00241_gb300 import build as B
B.LIB = B.build(bounds=True)
import torch
from paper_2201_00241_gb300 import rh, gridgen as gg
from oracle import OracleGrid

lib = rh.load()
out = {}
en, err = C.c_int32(0), C.c_uint32(0)
assert lib.rh_bounds_check(0, C.byref(en), C.byref(err)) == 0
out["enabled"] = en.value
for name in ["tiny30", "case118"]:
    g = gg.make_grid(30, 41, 6, 4) if name == "tiny30" else gg.make_case(name)
    lg = rh.Grid(g, device=0)
    st = lg.plant()
    lg.set_state(st.p, st.pd, st.qd)
    x, it, res, _ = lg.powerflow(None)
    lam, grad, F = lg.adjoint()
    o = OracleGrid(g)
    so = o.plant()
    worst = 0.0
    for N in (1, 3, 33, 64):
        W = gg.random_directions(lg.n_p, N, N)
        HW = lg.hessvec(W)
        Ho = o.hessvec(so.x, so.p, so.pd, so.qd, W)
        worst = max(worst, float(np.abs(HW - Ho).max() / np.abs(Ho).max()))
        Wd = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
        lg.hessvec(Wd)
    Hc = lg.hessian(block_n=16, concurrent=True)
    Hb = lg.hessian(block_n=16, concurrent=False)
    Hf, _, _ = lg.reduced_hessian()
    lg.hessian_columns(3, 7)
    R = np.random.default_rng(0).normal(size=(lg.n_x, 5))
    lg.solve(R, trans=False)
    lg.solve(R, trans=True)
    lg.lagrangian_hessvec(np.random.default_rng(1).normal(size=(lg.n_x + lg.n_p, 3)))
    W = gg.random_directions(lg.n_p, 8, 2)
    Wd = torch.from_numpy(np.ascontiguousarray(W.T)).cuda().t()
    HWd = torch.empty((8, lg.n_p), dtype=torch.float64, device="cuda").t()
    work = torch.empty(rh.work_doubles(lg, 8), dtype=torch.float64, device="cuda")
    rh.batch_hessvec([(lg, Wd, HWd, work)], 2)
    torch.cuda.synchronize()
    Wc = torch.from_numpy(np.ascontiguousarray(W.T)).cuda()
    HWc = torch.empty((8, lg.n_p), dtype=torch.float64, device="cuda")
    assert lib.rh_hessvec_noalloc(lg._h, C.c_void_p(Wc.data_ptr()), lg.n_p, 8, C.c_void_p(HWc.data_ptr()), lg.n_p,
                                  C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    lg.set_jacobian_method("ad")
    lg.adjoint()
    lg.set_jacobian_method("analytic")
    lg.adjoint()
    n = lg.n_p
    H = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    rh._check(lib.rh_rto_step(lg._h, rh._ptr(H), n, rh._ptr(d), None, rh._ptr(info),
                              C.c_void_p(torch.cuda.current_stream().cuda_stream), 0))
    torch.cuda.synchronize()
    Ho = o.hessvec(so.x, so.p, so.pd, so.qd, np.eye(n))
    worst = max(worst, float(np.abs(Hf - Ho).max() / np.abs(Ho).max()),
                float(np.abs(Hc - Ho).max() / np.abs(Ho).max()), float(np.abs(Hb - Ho).max() / np.abs(Ho).max()))
    assert lib.rh_bounds_check(0, C.byref(en), C.byref(err)) == 0
    out[name] = {"errors": int(err.value), "worst_rel": worst, "newton_iters": it, "resid": res}
print(json.dumps(out))
"""


def test_index_checking_build_reports_no_index_outside_its_array():
    env = dict(os.environ)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["enabled"] == 1
    for name in ("tiny30", "case118"):
        assert res[name]["errors"] == 0, res
        assert res[name]["worst_rel"] <= 1e-10, res
        assert res[name]["resid"] <= 1e-12


def test_normal_build_reports_checks_off():
    import ctypes as C
    from paper_2201_00241_gb300 import rh
    lib = rh.load()
    en, err = C.c_int32(7), C.c_uint32(7)
    assert lib.rh_bounds_check(0, C.byref(en), C.byref(err)) == 0
    assert en.value == 0 and err.value == 0
