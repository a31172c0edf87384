"""Thin ctypes binding of librh (include/rh.h): argument marshalling only.

Every numerical step runs in the CUDA kernels of the library.  Arrays may be
numpy arrays (host pointers) or CUDA torch tensors (device pointers, used on
torch's current stream).  There is no CPU fallback: without the built library
or a CUDA device the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

RH_OK, RH_EINVAL, RH_ENOMEM, RH_ESINGULAR, RH_ENOCONV, RH_ETIMEOUT, RH_ECUDA, RH_ESTATE = range(8)
RH_HOST_PTRS, RH_DEVICE_PTRS, RH_HESSIAN_CONCURRENT, RH_RTO_APPLY = 0, 1, 2, 4
_NAMES = ["RH_OK", "RH_EINVAL", "RH_ENOMEM", "RH_ESINGULAR", "RH_ENOCONV", "RH_ETIMEOUT", "RH_ECUDA", "RH_ESTATE"]

# every symbol declared in include/rh.h
EXPORTS = ["rh_grid_create", "rh_grid_destroy", "rh_grid_dims", "rh_grid_symbolic", "rh_injections",
           "rh_set_state", "rh_powerflow", "rh_adjoint", "rh_hessvec", "rh_hessian", "rh_solve", "rh_refactor",
           "rh_lagrangian_hessvec", "rh_hessvec_noalloc", "rh_hv_work_doubles", "rh_batch_hessvec",
           "rh_potrf", "rh_potrs", "rh_rto_step", "rh_set_jacobian_method", "rh_grid_coloring", "rh_jacobian",
           "rh_reduced_hessian", "rh_reduced_hessian_times", "rh_reduced_hessian_flops", "rh_fp64_fma_rate",
           "rh_hessian_columns", "rh_bounds_check", "rh_batch_powerflow", "rh_batch_hessvec_cfg",
           "rh_last_error"]
RH_JAC_ANALYTIC, RH_JAC_COLORED_AD = 0, 1


class RHError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES[status] if 0 <= status < len(_NAMES) else status}: {msg}")
        self.status = status


class _Desc(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("from_", C.c_void_p), ("to", C.c_void_p),
                ("r", C.c_void_p), ("x", C.c_void_p), ("b", C.c_void_p), ("bus_type", C.c_void_p),
                ("c2", C.c_void_p), ("c1", C.c_void_p), ("base_mva", C.c_double),
                ("order_level_cost", C.c_int64), ("max_tail", C.c_int32)]


class HvConfig(C.Structure):
    """rh_hv_config: width (directions per CTA, 0 = spread over the SMs), threads
    (CTA shape 128, 192, 256 or 384; 0 = 384), split_lanes (narrow-level k-split
    cap, a power of two <= 32; 0 = 32)."""
    _fields_ = [("width", C.c_int32), ("threads", C.c_int32), ("split_lanes", C.c_int32)]


class HvItem(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("W", C.c_void_p), ("ldw", C.c_int64), ("N", C.c_int32),
                ("HW", C.c_void_p), ("ldhw", C.c_int64), ("work", C.c_void_p)]


class Dims(C.Structure):
    _fields_ = [("n_bus", C.c_int32), ("n_branch", C.c_int32), ("n_gen", C.c_int32), ("n_pv", C.c_int32),
                ("n_pq", C.c_int32), ("n_x", C.c_int32), ("n_p", C.c_int32), ("n_levels_fwd", C.c_int32),
                ("n_levels_bwd", C.c_int32), ("nnz_jx", C.c_int64), ("nnz_jp", C.c_int64), ("nnz_l", C.c_int64),
                ("nnz_u", C.c_int64), ("refactor_updates", C.c_int64), ("setup_kernels", C.c_int32),
                ("hessian_kernels", C.c_int32), ("max_tail", C.c_int32), ("tail_vars", C.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librh.so; builds it first when it is missing and nvcc is available."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"librh is not built ({path}); run __graft_entry__.build()")
        _build.build()
    lib = C.CDLL(path)
    P, I32, I64, D, U32 = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint32
    sig = {
        "rh_grid_create": ([P, I32, P], C.c_int),
        "rh_grid_destroy": ([P], None),
        "rh_grid_dims": ([P, P], C.c_int),
        "rh_grid_symbolic": ([P] + [P] * 7, C.c_int),
        "rh_injections": ([P, P, P, P, P], C.c_int),
        "rh_set_state": ([P, P, P, P], C.c_int),
        "rh_powerflow": ([P, P, D, I32, P, P, P], C.c_int),
        "rh_adjoint": ([P, P, P, P], C.c_int),
        "rh_hessvec": ([P, P, I64, I32, P, I64, P, U32], C.c_int),
        "rh_hessian": ([P, I32, P, I64, P, U32], C.c_int),
        "rh_hessian_columns": ([P, I32, I32, P, I64, P, U32], C.c_int),
        "rh_bounds_check": ([I32, P, P], C.c_int),
        "rh_batch_powerflow": ([I32, P, P, D, I32, P, P, P, P], C.c_int),
        "rh_solve": ([P, P, I64, I32, I32, P, U32], C.c_int),
        "rh_refactor": ([P, P], C.c_int),
        "rh_lagrangian_hessvec": ([P, P, I64, I32, P, I64, P, U32], C.c_int),
        "rh_hessvec_noalloc": ([P, P, I64, I32, P, I64, P], C.c_int),
        "rh_hv_work_doubles": ([P, I32], C.c_int64),
        "rh_batch_hessvec": ([I32, P, I32, P], C.c_int),
        "rh_batch_hessvec_cfg": ([I32, P, P, P], C.c_int),
        "rh_potrf": ([I32, P, I64, P, P], C.c_int),
        "rh_potrs": ([I32, P, I64, P, I64, I32, P, P], C.c_int),
        "rh_rto_step": ([P, P, I64, P, P, P, P, U32], C.c_int),
        "rh_set_jacobian_method": ([P, I32], C.c_int),
        "rh_grid_coloring": ([P, P, P, P, P], C.c_int),
        "rh_jacobian": ([P, I32, P, P, P, P, P, P], C.c_int),
        "rh_reduced_hessian": ([P, P, I64, P, P, P, U32], C.c_int),
        "rh_reduced_hessian_times": ([P, P], C.c_int),
        "rh_reduced_hessian_flops": ([P, I32, P, P], C.c_int),
        "rh_fp64_fma_rate": ([I32, I32, I32, I64, P, P], C.c_int),
        "rh_last_error": ([], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


def _check(st: int):
    if st != RH_OK:
        raise RHError(st, _lib.rh_last_error().decode())


def _ptr(a) -> C.c_void_p:
    if a is None:
        return C.c_void_p(0)
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())  # torch tensor


def _is_device(a) -> bool:
    return a is not None and not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def _stream_of(a):
    if _is_device(a):
        import torch
        return C.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)
    return C.c_void_p(0)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Planted:
    x: np.ndarray
    p: np.ndarray
    pd: np.ndarray
    qd: np.ndarray


class Grid:
    """One grid loaded on one GPU (rh_grid_create)."""

    def __init__(self, grid, device: int = 0, max_tail: int = 0):
        """max_tail: dense-tail bound of the factors (0: the library's default from n_x;
        rh_grid_desc.max_tail).  The bound in use is dims.max_tail."""
        lib = load()
        self.src = grid
        self.max_tail = int(max_tail)
        self._state = None            # (p, pd, qd) of the last set_state with host arrays
        self._x = None                # last power-flow solution
        self._keep = [np.ascontiguousarray(grid.fr, dtype=np.int32), np.ascontiguousarray(grid.to, dtype=np.int32),
                      _f64(grid.r), _f64(grid.x), _f64(grid.b), np.ascontiguousarray(grid.bus_type, dtype=np.int8),
                      _f64(grid.c2), _f64(grid.c1)]
        k = self._keep
        d = _Desc(int(grid.n_bus), int(grid.n_branch), *[_ptr(a) for a in k], float(grid.base_mva),
                  int(grid.order_level_cost), self.max_tail)
        h = C.c_void_p(0)
        _check(lib.rh_grid_create(C.byref(d), int(device), C.byref(h)))
        self._h = h
        self.device = device
        dm = Dims()
        _check(lib.rh_grid_dims(self._h, C.byref(dm)))
        self.dims = dm
        self.n_bus, self.n_x, self.n_p = dm.n_bus, dm.n_x, dm.n_p

    def close(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.rh_grid_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    # ---- symbolic ------------------------------------------------------------
    def symbolic(self) -> dict:
        dm, nx = self.dims, self.n_x
        out = dict(perm=np.empty(nx, np.int32), bus_order=np.empty(self.n_bus - 1, np.int32),
                   level=np.empty(self.n_bus - 1, np.int32), Lp=np.empty(nx + 1, np.int32),
                   Lj=np.empty(dm.nnz_l, np.int32), Up=np.empty(nx + 1, np.int32), Uj=np.empty(dm.nnz_u, np.int32))
        _check(_lib.rh_grid_symbolic(self._h, *[_ptr(out[k]) for k in ("perm", "bus_order", "level", "Lp", "Lj",
                                                                       "Up", "Uj")]))
        return out

    # ---- model ---------------------------------------------------------------
    def injections(self, vm, va):
        vm, va = _f64(vm), _f64(va)
        P = np.empty(self.n_bus)
        Q = np.empty(self.n_bus)
        _check(_lib.rh_injections(self._h, _ptr(vm), _ptr(va), _ptr(P), _ptr(Q)))
        return P, Q

    def set_state(self, p=None, pd=None, qd=None):
        """p None keeps the current parameters (for example those of a tracking step)."""
        p = None if p is None else _f64(p)
        pd = None if pd is None else _f64(pd)
        qd = None if qd is None else _f64(qd)
        _check(_lib.rh_set_state(self._h, _ptr(p), _ptr(pd), _ptr(qd)))
        if p is None:
            self._state = None        # parameters set on the device: not known here
        else:
            old = self._state or (None, None, None)
            self._state = (p.copy(), old[1] if pd is None else pd.copy(), old[2] if qd is None else qd.copy())
        self._x = None

    def clone(self, max_tail: int | None = None, device: int | None = None) -> "Grid":
        """The same grid record loaded again (another dense-tail bound or device), brought
        to this grid's state: set_state with its parameters and loads, power flow from its
        last solution, adjoint.  Needs a state set from the host and a power flow."""
        if self._state is None or self._x is None:
            raise RuntimeError("clone needs a state set from host arrays and a power-flow solution")
        g = Grid(self.src, self.device if device is None else device,
                 self.max_tail if max_tail is None else max_tail)
        p, pd, qd = self._state
        g.set_state(p, pd, qd)
        g.powerflow(self._x)
        g.adjoint()
        return g

    def powerflow(self, x0=None, tol=1e-12, max_iter=20, raise_on_noconv=True):
        x0 = None if x0 is None else _f64(x0)
        x = np.empty(self.n_x)
        it = C.c_int32(0)
        res = C.c_double(0.0)
        st = _lib.rh_powerflow(self._h, _ptr(x0), float(tol), int(max_iter), _ptr(x), C.byref(it), C.byref(res))
        if st != RH_ENOCONV or raise_on_noconv:
            _check(st)
        self._x = x.copy() if st == RH_OK else None
        return x, int(it.value), float(res.value), st

    def adjoint(self):
        F = C.c_double(0.0)
        lam = np.empty(self.n_x)
        grad = np.empty(self.n_p)
        _check(_lib.rh_adjoint(self._h, C.byref(F), _ptr(lam), _ptr(grad)))
        return lam, grad, float(F.value)

    def refactor(self):
        A = np.empty(self.dims.nnz_l + self.dims.nnz_u)
        _check(_lib.rh_refactor(self._h, _ptr(A)))
        return A

    # ---- Algorithm 2 -------------------------------------------------------------
    def hessvec(self, W, HW=None, stream=None):
        """HW = (Hess F) W.  W: (n_p, N) numpy (column-major) or a CUDA torch tensor.

        Torch tensors are taken as column-major (n_p, N): pass ``W.t().contiguous().t()``
        or a tensor of shape (N, n_p) transposed.
        """
        if _is_device(W):
            N = W.shape[1]
            assert N <= 1 or W.stride(0) == 1, "device W must be column-major (stride(0) == 1)"
            if HW is None:
                import torch
                HW = torch.empty((N, self.n_p), dtype=torch.float64, device=W.device).t()
            st = stream if stream is not None else _stream_of(W)
            ldw = W.stride(1) if N > 1 else self.n_p
            ldh = HW.stride(1) if N > 1 else self.n_p
            _check(_lib.rh_hessvec(self._h, _ptr(W), ldw, N, _ptr(HW), ldh, st, RH_DEVICE_PTRS))
            return HW
        W = np.asfortranarray(W, dtype=np.float64)
        if W.ndim == 1:
            W = W.reshape(-1, 1, order="F")
        N = W.shape[1]
        HW = np.empty((self.n_p, N), order="F")
        _check(_lib.rh_hessvec(self._h, _ptr(W), self.n_p, N, _ptr(HW), self.n_p, C.c_void_p(0), RH_HOST_PTRS))
        return HW

    def hessian(self, block_n=256, concurrent=True, out=None, stream=None):
        flags = RH_HESSIAN_CONCURRENT if concurrent else 0
        if out is not None and _is_device(out):
            st = stream if stream is not None else _stream_of(out)
            _check(_lib.rh_hessian(self._h, int(block_n), _ptr(out), out.stride(1), st, flags | RH_DEVICE_PTRS))
            return out
        H = np.empty((self.n_p, self.n_p), order="F")
        _check(_lib.rh_hessian(self._h, int(block_n), _ptr(H), self.n_p, C.c_void_p(0), flags))
        return H

    def hessian_columns(self, col0, ncols, out=None, stream=None):
        """Columns col0 .. col0 + ncols - 1 of H in one launch (rh_hessian_columns): a numpy
        (n_p, ncols) column-major array, or ``out`` (a column-major CUDA tensor) when given."""
        if out is not None and _is_device(out):
            st = stream if stream is not None else _stream_of(out)
            ld = out.stride(1) if ncols > 1 else self.n_p
            _check(_lib.rh_hessian_columns(self._h, int(col0), int(ncols), _ptr(out), ld, st, RH_DEVICE_PTRS))
            return out
        H = np.empty((self.n_p, ncols), order="F")
        _check(_lib.rh_hessian_columns(self._h, int(col0), int(ncols), _ptr(H), self.n_p, C.c_void_p(0),
                                       RH_HOST_PTRS))
        return H

    def reduced_hessian(self, out=None, stream=None):
        """Jacobians, refactorisation, adjoint and the full reduced Hessian in one call
        (the adjoint solve overlapped with the first direction sweeps).  Returns
        (H, grad, F); H is ``out`` when given (a CUDA torch tensor, column-major),
        else a new column-major numpy array."""
        F = C.c_double(0.0)
        grad = np.empty(self.n_p)
        if out is not None and _is_device(out):
            st = stream if stream is not None else _stream_of(out)
            _check(_lib.rh_reduced_hessian(self._h, _ptr(out), out.stride(1), C.byref(F), _ptr(grad), st,
                                           RH_DEVICE_PTRS))
            return out, grad, float(F.value)
        H = np.empty((self.n_p, self.n_p), order="F")
        _check(_lib.rh_reduced_hessian(self._h, _ptr(H), self.n_p, C.byref(F), _ptr(grad), C.c_void_p(0),
                                       RH_HOST_PTRS))
        return H, grad, float(F.value)

    def reduced_hessian_times(self):
        """Device times (ms) of the last reduced_hessian call, from the fork after the
        factorisation: (both direction launches, the first one, the adjoint branch)."""
        ms = (C.c_float * 3)()
        _check(_lib.rh_reduced_hessian_times(self._h, ms))
        return tuple(float(v) for v in ms)

    def reduced_hessian_flops(self, n_sm=0):
        """(algorithmic, executed) FP64 flops of the direction launches of one reduced_hessian
        call (rh_reduced_hessian_flops); n_sm = 0 takes the grid's device."""
        a, e = C.c_double(0.0), C.c_double(0.0)
        _check(_lib.rh_reduced_hessian_flops(self._h, int(n_sm), C.byref(a), C.byref(e)))
        return float(a.value), float(e.value)

    def solve(self, R, trans=False):
        R = np.array(R, dtype=np.float64, order="F", copy=True)
        if R.ndim == 1:
            R = R.reshape(-1, 1, order="F")
        _check(_lib.rh_solve(self._h, _ptr(R), self.n_x, R.shape[1], int(bool(trans)), C.c_void_p(0), RH_HOST_PTRS))
        return R

    def lagrangian_hessvec(self, V):
        V = np.asfortranarray(V, dtype=np.float64)
        if V.ndim == 1:
            V = V.reshape(-1, 1, order="F")
        nu = self.n_x + self.n_p
        Y = np.empty((nu, V.shape[1]), order="F")
        _check(_lib.rh_lagrangian_hessvec(self._h, _ptr(V), nu, V.shape[1], _ptr(Y), nu, C.c_void_p(0),
                                          RH_HOST_PTRS))
        return Y

    # ---- coloured forward-mode Jacobian (section 4.2.2) ----------------------------
    def set_jacobian_method(self, method: str):
        """'analytic' (default) or 'ad' (coloured forward-mode AD) for every later assembly."""
        _check(_lib.rh_set_jacobian_method(self._h, {"analytic": RH_JAC_ANALYTIC, "ad": RH_JAC_COLORED_AD}[method]))

    def coloring(self):
        cx = np.empty(self.n_x, np.int32)
        cp = np.empty(self.n_p, np.int32)
        ncx, ncp = C.c_int32(0), C.c_int32(0)
        _check(_lib.rh_grid_coloring(self._h, _ptr(cx), _ptr(cp), C.byref(ncx), C.byref(ncp)))
        return cx, cp, int(ncx.value), int(ncp.value)

    def jacobian(self, method: str = "ad"):
        """J_x, J_p at the current state as (row, col, value) triplets in x / p indices."""
        m = {"analytic": RH_JAC_ANALYTIC, "ad": RH_JAC_COLORED_AD}[method]
        d = self.dims
        jx = (np.empty(d.nnz_jx, np.int32), np.empty(d.nnz_jx, np.int32), np.empty(d.nnz_jx))
        jp = (np.empty(d.nnz_jp, np.int32), np.empty(d.nnz_jp, np.int32), np.empty(d.nnz_jp))
        _check(_lib.rh_jacobian(self._h, m, *[_ptr(a) for a in jx], *[_ptr(a) for a in jp]))
        return jx, jp

    # ---- real-time tracking step (section 6.3) -------------------------------------
    def rto_step(self, H=None, apply=False, stream=None):
        """rh_rto_step at the current state (after adjoint()).  Returns CUDA
        tensors d, p_next, H (n_p x n_p column-major, lower triangle = L) and the
        pivot status info (0, or the 1-based column of the first bad pivot),
        read after the stream finished."""
        import torch
        dev = torch.device("cuda", self.device)
        n = self.n_p
        if H is None:
            H = torch.empty((n, n), dtype=torch.float64, device=dev).t()
        d = torch.empty(n, dtype=torch.float64, device=dev)
        p_next = torch.empty(n, dtype=torch.float64, device=dev)
        info = torch.empty(1, dtype=torch.int32, device=dev)
        st = stream if stream is not None else C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
        _check(_lib.rh_rto_step(self._h, _ptr(H), H.stride(1), _ptr(d), _ptr(p_next), _ptr(info), st,
                                RH_RTO_APPLY if apply else 0))
        if apply:
            self._state, self._x = None, None      # parameters now set on the device
        torch.cuda.synchronize(dev)
        return d, p_next, H, int(info.item())

    # ---- planted operating point -------------------------------------------------
    def index_maps(self):
        """(ix_th, ix_v, ip_v, ip_pg) per bus, from the documented index conventions."""
        t = np.asarray(self.src.bus_type)
        n = len(t)
        ix_th = np.full(n, -1, np.int32)
        ix_v = np.full(n, -1, np.int32)
        ip_v = np.full(n, -1, np.int32)
        ip_pg = np.full(n, -1, np.int32)
        pv, pq, gen = np.flatnonzero(t == 1), np.flatnonzero(t == 2), np.flatnonzero(t != 2)
        ix_th[pv] = np.arange(len(pv))
        ix_th[pq] = len(pv) + np.arange(len(pq))
        ix_v[pq] = len(pv) + len(pq) + np.arange(len(pq))
        ip_v[gen] = np.arange(len(gen))
        ip_pg[pv] = len(gen) + np.arange(len(pv))
        return ix_th, ix_v, ip_v, ip_pg

    def plant(self, vm=None, va=None) -> Planted:
        """Loads and parameters that make the planted voltages an exact solution
        (loads at PQ buses, Pg = P_inj at PV buses), from the library's injections."""
        g = self.src
        vm = _f64(g.v_star if vm is None else vm)
        va = _f64(g.theta_star if va is None else va)
        P, Q = self.injections(vm, va)
        ix_th, ix_v, ip_v, ip_pg = self.index_maps()
        pq = ix_v >= 0
        pd = np.where(pq, -P, 0.0)
        qd = np.where(pq, -Q, 0.0)
        x = np.empty(self.n_x)
        p = np.empty(self.n_p)
        th = ix_th >= 0
        x[ix_th[th]] = va[th]
        x[ix_v[pq]] = vm[pq]
        gen = ip_v >= 0
        p[ip_v[gen]] = vm[gen]
        pv = ip_pg >= 0
        p[ip_pg[pv]] = P[pv]
        return Planted(x, p, pd, qd)


def batch_hessvec(items, width: int = 0, stream=None, threads: int = 0, split_lanes: int = 0):
    """rh_batch_hessvec_cfg: items are (Grid, W, HW, work) with CUDA torch tensors W, HW
    (column-major n_p x N views) and work (1-D float64 tensor of
    rh_hv_work_doubles(grid, N) elements) or None.  width, threads, split_lanes:
    the launch configuration (HvConfig; 0 = default).  Asynchronous on `stream`
    (default: torch's current stream)."""
    lib = load()
    arr = (HvItem * len(items))()
    for k, (grid, W, HW, work) in enumerate(items):
        n = W.shape[1]
        assert HW.shape[1] == n and W.shape[0] == HW.shape[0] == grid.n_p
        assert n <= 1 or (W.stride(0) == 1 and HW.stride(0) == 1), "W and HW must be column-major"
        # a single column's leading dimension is free (torch may report any stride there)
        ldw = W.stride(1) if n > 1 else grid.n_p
        ldh = HW.stride(1) if n > 1 else grid.n_p
        arr[k] = HvItem(grid._h.value, W.data_ptr(), ldw, n, HW.data_ptr(), ldh,
                        0 if work is None else work.data_ptr())
    if stream is None:
        import torch
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    cfg = HvConfig(int(width), int(threads), int(split_lanes))
    _check(lib.rh_batch_hessvec_cfg(len(items), arr, C.byref(cfg), stream))


def batch_hessvec_raw(items, n_items: int, cfg, stream):
    """rh_batch_hessvec_cfg on an item array already laid out as rh_hv_item records: a
    ctypes array of HvItem, or anything exposing .ctypes.data with HvItem's layout (a numpy
    record array).  cfg: an HvConfig, or a dict {"width", "threads", "split_lanes"};
    stream a c_void_p."""
    c = cfg if isinstance(cfg, HvConfig) else HvConfig(int(cfg.get("width", 0)), int(cfg.get("threads", 0)),
                                                      int(cfg.get("split_lanes", 0)))
    ptr = C.addressof(items) if isinstance(items, C.Array) else items.ctypes.data
    _check((_lib or load()).rh_batch_hessvec_cfg(int(n_items), C.c_void_p(ptr), C.byref(c), stream))


def batch_powerflow(grids, x0=None, tol=1e-12, max_iter=20):
    """Newton power flow for several grids of one topology at once (rh_batch_powerflow).

    x0: None, or one starting point per grid (numpy n_x, or None to continue from the
    grid's state).  Returns (xs, iters, resid, status) per grid; raises nothing for
    items that did not converge: their status says so."""
    lib = load()
    n = len(grids)
    hs = (C.c_void_p * n)(*[g._h.value if isinstance(g._h, C.c_void_p) else g._h for g in grids])
    keep = []
    x0p = None
    if x0 is not None:
        x0p = (C.c_void_p * n)()
        for i, x in enumerate(x0):
            if x is not None:
                a = _f64(x)
                keep.append(a)
                x0p[i] = a.ctypes.data
    xs = [np.empty(g.n_x) for g in grids]
    xop = (C.c_void_p * n)(*[x.ctypes.data for x in xs])
    iters = np.zeros(n, np.int32)
    resid = np.zeros(n)
    status = np.zeros(n, np.int32)
    st = lib.rh_batch_powerflow(n, hs, x0p, float(tol), int(max_iter), xop, _ptr(iters), _ptr(resid), _ptr(status))
    if st not in (RH_OK, RH_ENOCONV, RH_ESINGULAR):
        _check(st)
    for g, x, s_ in zip(grids, xs, status):
        if isinstance(g, Grid):
            g._x = x.copy() if s_ == RH_OK else None
    return xs, iters, resid, status


def work_doubles(grid, N: int) -> int:
    return int(load().rh_hv_work_doubles(grid._h, int(N)))


def _stream_arg(a, stream):
    if stream is not None:
        return stream
    import torch
    return C.c_void_p(torch.cuda.current_stream(a.device).cuda_stream)


def potrf(A, info=None, stream=None):
    """rh_potrf in place on a column-major CUDA float64 tensor A (n x n view with
    stride(0) == 1).  Returns the device int32 tensor info (asynchronous)."""
    import torch
    n = A.shape[0]
    assert A.shape == (n, n) and (n <= 1 or A.stride(0) == 1), "A must be a column-major n x n view"
    if info is None:
        info = torch.empty(1, dtype=torch.int32, device=A.device)
    lda = A.stride(1) if n > 1 else max(n, 1)
    _check(load().rh_potrf(n, _ptr(A), lda, _ptr(info), _stream_arg(A, stream)))
    return info


def potrs(L, B, work=None, stream=None):
    """rh_potrs: B <- (L L^T)^{-1} B in place; B a column-major CUDA (n, nrhs) view or a vector."""
    import torch
    n = L.shape[0]
    Bv = B.reshape(-1, 1) if B.dim() == 1 else B
    nrhs = Bv.shape[1]
    assert nrhs <= 1 or Bv.stride(0) == 1, "B must be column-major"
    if work is None:
        work = torch.empty(max(n * nrhs, 1), dtype=torch.float64, device=B.device)
    ldl = L.stride(1) if n > 1 else max(n, 1)
    ldb = Bv.stride(1) if nrhs > 1 else max(n, 1)
    _check(load().rh_potrs(n, _ptr(L), ldl, _ptr(Bv), ldb, nrhs, _ptr(work), _stream_arg(B, stream)))
    return B


def fp64_fma_rate(device=0, ctas_per_sm=2, threads_per_cta=384, iters=1 << 16):
    """(GFLOP/s, ms) of the device's FP64 FMA throughput (rh_fp64_fma_rate)."""
    lib = load()
    gf, ms = C.c_double(0.0), C.c_float(0.0)
    st = lib.rh_fp64_fma_rate(int(device), int(ctas_per_sm), int(threads_per_cta), int(iters), C.byref(gf),
                              C.byref(ms))
    if st != RH_OK:
        raise RHError(st, "rh_fp64_fma_rate failed")
    return float(gf.value), float(ms.value)
