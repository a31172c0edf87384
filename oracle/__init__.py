"""CPU oracle for the batched reduced-Hessian-vector product (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU baseline leg of
``bench.py`` may import this package.  It wraps ``rh_oracle.c`` (plain C, fp64)
through ctypes and shares no code with the CUDA library.

Index conventions (the reading of the paper's section 3.1 that reproduces the
n_x / n_p counts of Table 1):

* x = [theta at PV buses (ascending id), theta at PQ buses, v at PQ buses];
* p = [v at generator buses incl. the slack (ascending id), Pg at PV buses];
* the rows of g (and lambda) are ordered like x: P_i pairs with theta_i and
  Q_i with v_i.

Grids are duck-typed: any object with the attributes of
``paper_2201_00241_gb300.gridgen.Grid`` (fr, to, r, x, b, bus_type, c2, c1,
base_mva, order_level_cost, v_star, theta_star).  order_level_cost is the
weight of one forward level when the two fill-reducing orders are compared,
a parameter of the static pivot order the paper leaves unstated.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(_build.build())
    P = C.c_void_p
    I = C.c_int
    D = C.c_double
    lib.orc_grid_new.restype = P
    lib.orc_grid_new.argtypes = [I, I, P, P, P, P, P, P, P, P, D, C.c_longlong]
    lib.orc_grid_free.argtypes = [P]
    lib.orc_n_x.argtypes = [P]
    lib.orc_n_p.argtypes = [P]
    lib.orc_ref.argtypes = [P]
    lib.orc_index_maps.argtypes = [P, P, P, P, P]
    lib.orc_injections.argtypes = [P, P, P, P, P]
    lib.orc_residual.argtypes = [P, P, P, P, P, P]
    lib.orc_objective.restype = D
    lib.orc_objective.argtypes = [P, P, P, P]
    lib.orc_jacobians_dense.argtypes = [P, P, P, P, P]
    lib.orc_solve.argtypes = [P, P, P, P, I, I]
    lib.orc_newton.argtypes = [P, P, P, P, P, D, I, P, P]
    lib.orc_adjoint.argtypes = [P, P, P, P, P, P, P, P]
    lib.orc_lagrangian_hessian_dense.argtypes = [P, P, P, P, P, P]
    lib.orc_hessvec.argtypes = [P, P, P, P, P, P, I, I, P, I]
    lib.orc_hessvec_threads.argtypes = [P, P, P, P, P, P, I, I, P, I, I]
    lib.orc_symbolic.argtypes = [P] + [P] * 7 + [P, P, P]
    lib.orc_order.argtypes = [P, C.c_int, P]
    lib.orc_order.restype = C.c_int
    lib.orc_lu_dense.argtypes = [P, P, P, P, P, P]
    lib.orc_cholesky.argtypes = [I, P, I, P, I]
    lib.orc_jacobians_csc.argtypes = [P, P, P] + [P] * 8
    lib.orc_coloring.argtypes = [P, P, P, P, P]
    lib.orc_cholesky_solve.argtypes = [I, P, I, P, I, I]
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class State:
    """A power-flow operating point: state x, parameters p and bus loads."""
    x: np.ndarray
    p: np.ndarray
    pd: np.ndarray
    qd: np.ndarray


class OracleGrid:
    def __init__(self, grid):
        lib = _load()
        self.grid = grid
        self._keep = [
            np.ascontiguousarray(grid.fr, dtype=np.int32),
            np.ascontiguousarray(grid.to, dtype=np.int32),
            _f64(grid.r), _f64(grid.x), _f64(grid.b),
            np.ascontiguousarray(grid.bus_type, dtype=np.int8),
            _f64(grid.c2), _f64(grid.c1),
        ]
        k = self._keep
        self.n_bus = int(grid.n_bus)
        self._h = lib.orc_grid_new(self.n_bus, int(grid.n_branch), _p(k[0]), _p(k[1]), _p(k[2]),
                                   _p(k[3]), _p(k[4]), _p(k[5]), _p(k[6]), _p(k[7]),
                                   float(grid.base_mva), int(grid.order_level_cost))
        self.n_x = lib.orc_n_x(self._h)
        self.n_p = lib.orc_n_p(self._h)
        self.ref = lib.orc_ref(self._h)

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_grid_free(self._h)
            self._h = None

    # ---- index maps ------------------------------------------------------
    def index_maps(self):
        n = self.n_bus
        a = [np.empty(n, dtype=np.int32) for _ in range(4)]
        _lib.orc_index_maps(self._h, *[_p(v) for v in a])
        return tuple(a)  # ix_th, ix_v, ip_v, ip_pg

    # ---- model -------------------------------------------------------------
    def injections(self, vm, va):
        vm, va = _f64(vm), _f64(va)
        P = np.empty(self.n_bus)
        Q = np.empty(self.n_bus)
        _lib.orc_injections(self._h, _p(vm), _p(va), _p(P), _p(Q))
        return P, Q

    def residual(self, x, p, pd, qd):
        x, p, pd, qd = map(_f64, (x, p, pd, qd))
        out = np.empty(self.n_x)
        _lib.orc_residual(self._h, _p(x), _p(p), _p(pd), _p(qd), _p(out))
        return out

    def objective(self, x, p, pd):
        x, p, pd = map(_f64, (x, p, pd))
        return float(_lib.orc_objective(self._h, _p(x), _p(p), _p(pd)))

    def jacobians_dense(self, x, p):
        x, p = _f64(x), _f64(p)
        jx = np.empty((self.n_x, self.n_x), order="F")
        jp = np.empty((self.n_x, self.n_p), order="F")
        _lib.orc_jacobians_dense(self._h, _p(x), _p(p), _p(jx), _p(jp))
        return jx, jp

    def solve(self, x, p, R, trans=False):
        x, p = _f64(x), _f64(p)
        R = np.array(R, dtype=np.float64, order="F", copy=True)
        if R.ndim == 1:
            R = R.reshape(-1, 1, order="F")
        st = _lib.orc_solve(self._h, _p(x), _p(p), _p(R), R.shape[1], int(bool(trans)))
        if st != 0:
            raise RuntimeError("oracle LU: singular pivot")
        return R

    def newton(self, p, pd, qd, x0, tol=1e-12, max_iter=20):
        p, pd, qd = map(_f64, (p, pd, qd))
        x = np.array(x0, dtype=np.float64, copy=True)
        it = C.c_int(0)
        res = C.c_double(0.0)
        st = _lib.orc_newton(self._h, _p(p), _p(pd), _p(qd), _p(x), float(tol), int(max_iter),
                             C.byref(it), C.byref(res))
        return x, int(st), int(it.value), float(res.value)

    def adjoint(self, x, p, pd, qd):
        x, p, pd, qd = map(_f64, (x, p, pd, qd))
        lam = np.empty(self.n_x)
        grad = np.empty(self.n_p)
        F = C.c_double(0.0)
        st = _lib.orc_adjoint(self._h, _p(x), _p(p), _p(pd), _p(qd), _p(lam), _p(grad), C.byref(F))
        if st != 0:
            raise RuntimeError("oracle LU: singular pivot")
        return lam, grad, float(F.value)

    def lagrangian_hessian_dense(self, x, p, pd, lam):
        x, p, pd, lam = map(_f64, (x, p, pd, lam))
        nu = self.n_x + self.n_p
        out = np.empty((nu, nu), order="F")
        _lib.orc_lagrangian_hessian_dense(self._h, _p(x), _p(p), _p(pd), _p(lam), _p(out))
        return out

    def hessvec(self, x, p, pd, qd, W, threads=1):
        """HW, one column of W at a time (Algorithm 1); threads > 1 shares the columns out
        among that many threads (the same arithmetic per column)."""
        x, p, pd, qd = map(_f64, (x, p, pd, qd))
        W = np.asfortranarray(W, dtype=np.float64)
        if W.ndim == 1:
            W = W.reshape(-1, 1, order="F")
        assert W.shape[0] == self.n_p
        N = W.shape[1]
        HW = np.empty((self.n_p, N), order="F")
        st = _lib.orc_hessvec_threads(self._h, _p(x), _p(p), _p(pd), _p(qd), _p(W), self.n_p, N, _p(HW), self.n_p,
                                      int(threads))
        if st != 0:
            raise RuntimeError("oracle LU: singular pivot")
        return HW

    def jacobians_csc(self, x, p):
        """J_x, J_p as scipy CSC matrices with their structural pattern (explicit zeros kept)."""
        import scipy.sparse as sp
        x, p = _f64(x), _f64(p)
        nx_, np_ = C.c_int64(0), C.c_int64(0)
        null = C.c_void_p(0)
        _lib.orc_jacobians_csc(self._h, _p(x), _p(p), null, null, null, null, null, null,
                               C.byref(nx_), C.byref(np_))
        a = dict(xp=np.empty(self.n_x + 1, np.int32), xi=np.empty(nx_.value, np.int32), xx=np.empty(nx_.value),
                 pp=np.empty(self.n_p + 1, np.int32), pi=np.empty(np_.value, np.int32), px=np.empty(np_.value))
        _lib.orc_jacobians_csc(self._h, _p(x), _p(p), _p(a["xp"]), _p(a["xi"]), _p(a["xx"]), _p(a["pp"]),
                               _p(a["pi"]), _p(a["px"]), C.byref(nx_), C.byref(np_))
        Jx = sp.csc_matrix((a["xx"], a["xi"], a["xp"]), shape=(self.n_x, self.n_x))
        Jp = sp.csc_matrix((a["px"], a["pi"], a["pp"]), shape=(self.n_x, self.n_p))
        return Jx, Jp

    def coloring(self):
        """Greedy column colourings of J_x and J_p (section 4.2.2): (colors_x, colors_p, n_colors_x, n_colors_p)."""
        cx = np.empty(self.n_x, np.int32)
        cp = np.empty(self.n_p, np.int32)
        ncx, ncp = C.c_int32(0), C.c_int32(0)
        _lib.orc_coloring(self._h, _p(cx), _p(cp), C.byref(ncx), C.byref(ncp))
        return cx, cp, int(ncx.value), int(ncp.value)

    def order(self, which):
        """One candidate elimination order of the buses: "degree" (exact minimum degree),
        "fill" (minimum weighted fill) or "static" (the one the factorisation uses)."""
        out = np.empty(self.n_bus, np.int32)
        n = _lib.orc_order(self._h, {"degree": 0, "fill": 1, "static": 2}[which], _p(out))
        return out[:n]

    def symbolic(self):
        nnzL = C.c_int64(0)
        nnzU = C.c_int64(0)
        nel = C.c_int32(0)
        null = C.c_void_p(0)
        _lib.orc_symbolic(self._h, null, null, null, null, null, null, null,
                          C.byref(nnzL), C.byref(nnzU), C.byref(nel))
        nx = self.n_x
        out = dict(perm=np.empty(nx, np.int32), bus_order=np.empty(nel.value, np.int32),
                   level=np.empty(nel.value, np.int32), Lp=np.empty(nx + 1, np.int32),
                   Lj=np.empty(nnzL.value, np.int32), Up=np.empty(nx + 1, np.int32),
                   Uj=np.empty(nnzU.value, np.int32))
        _lib.orc_symbolic(self._h, _p(out["perm"]), _p(out["bus_order"]), _p(out["level"]),
                          _p(out["Lp"]), _p(out["Lj"]), _p(out["Up"]), _p(out["Uj"]),
                          C.byref(nnzL), C.byref(nnzU), C.byref(nel))
        return out

    def lu_dense(self, x, p):
        x, p = _f64(x), _f64(p)
        n = self.n_x
        perm = np.empty(n, np.int32)
        L = np.empty((n, n), order="F")
        U = np.empty((n, n), order="F")
        st = _lib.orc_lu_dense(self._h, _p(x), _p(p), _p(perm), _p(L), _p(U))
        if st != 0:
            raise RuntimeError("oracle LU: singular pivot")
        return perm, L, U

    # ---- real-time tracking step (section 6.3) ------------------------------
    def rto_step(self, x, p, pd, qd):
        """One tracking update at loads (pd, qd), eq. (18)-(19).

        Step 1: reduced gradient g (eq. 7) and reduced Hessian H (Algorithm 1
        applied to the columns of the identity) at the power-flow solution x.
        Step 2: H = L L^T, d = -H^{-1} g, p_next = p + d.
        """
        lam, g, F = self.adjoint(x, p, pd, qd)
        H = self.hessvec(x, p, pd, qd, np.eye(self.n_p))
        L, info = cholesky(H)
        if info:
            raise RuntimeError(f"oracle Cholesky: pivot {info} is not positive")
        d = -cholesky_solve(L, g)[:, 0]
        return dict(g=g, F=F, H=H, L=L, d=d, p_next=_f64(p) + d)

    # ---- planted operating point ---------------------------------------------
    def plant(self, vm=None, va=None) -> State:
        """Loads and parameters that make the grid's planted voltages an exact solution.

        Loads sit at PQ buses only: Pd = -P_inj, Qd = -Q_inj; PV generators
        produce Pg = P_inj; the slack takes the balance.
        """
        g = self.grid
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
        return State(x, p, pd, qd)


def cholesky(H):
    """Lower Cholesky factor of the symmetric positive definite H (lower triangle read).

    Returns (L, info): info = 0, or j + 1 for the first pivot that is not positive."""
    lib = _load()
    H = np.asfortranarray(H, dtype=np.float64)
    n = H.shape[0]
    L = np.zeros((n, n), order="F")
    info = lib.orc_cholesky(n, _p(H), max(n, 1), _p(L), max(n, 1))
    return L, int(info)


def cholesky_solve(L, B):
    """X with L L^T X = B (B a vector or n x nrhs)."""
    lib = _load()
    L = np.asfortranarray(L, dtype=np.float64)
    X = np.array(B, dtype=np.float64, order="F", copy=True)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    n = L.shape[0]
    lib.orc_cholesky_solve(n, _p(L), max(n, 1), _p(X), X.shape[1], max(n, 1))
    return X
