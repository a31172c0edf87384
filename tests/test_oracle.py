"""Pins of the CPU oracle against facts it does not compute itself.

Each test checks the oracle against the paper's printed numbers, a closed form,
an independent physical formulation, finite differences or brute force, so that
a dropped term, a wrong sign, a swapped index or a transposed operand in the
oracle fails at least one of them.
"""
import os

import numpy as np
import pytest

from oracle import OracleGrid
from paper_2201_00241_gb300 import gridgen as gg

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(n_bus, n_branch, n_gen, seed, lossless=False):
    return gg.make_grid(n_bus, n_branch, n_gen, seed, lossless=lossless)


def flat_start(o):
    ix_th, ix_v, _, _ = o.index_maps()
    x0 = np.zeros(o.n_x)
    x0[ix_v[ix_v >= 0]] = 1.0
    return x0


# ---------------------------------------------------------------------------
# Table 1: dimension counts (pins the index reading of x and p)
# ---------------------------------------------------------------------------

def test_table1_dimension_counts():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "table1_dims.txt"))
            if ln.strip() and not ln.startswith("#")]
    shapes = {118: "case118", 1354: "case1354", 2869: "case2869", 9241: "case9241"}
    for name, n_v, n_e, n_x, n_p in rows:
        c = gg.CASES[shapes[int(n_v)]]
        assert c["n_bus"] == int(n_v) and c["n_branch"] == int(n_e)
        assert 2 * c["n_gen"] - 1 == int(n_p), name
        # the oracle's own counts, from its own index maps, on the grid itself
        if int(n_v) <= 2869:
            o = OracleGrid(gg.make_case(shapes[int(n_v)]))
            assert (o.n_x, o.n_p) == (int(n_x), int(n_p)), name


def test_index_maps_order():
    g = tiny(12, 16, 4, 3)
    o = OracleGrid(g)
    ix_th, ix_v, ip_v, ip_pg = o.index_maps()
    t = g.bus_type
    pv, pq, gen = np.flatnonzero(t == 1), np.flatnonzero(t == 2), np.flatnonzero(t != 2)
    assert list(ix_th[pv]) == list(range(len(pv)))
    assert list(ix_th[pq]) == list(range(len(pv), len(pv) + len(pq)))
    assert list(ix_v[pq]) == list(range(len(pv) + len(pq), len(pv) + 2 * len(pq)))
    assert list(ip_v[gen]) == list(range(len(gen)))
    assert list(ip_pg[pv]) == list(range(len(gen), len(gen) + len(pv)))
    assert ix_th[t == 0] == -1 and ip_pg[t == 0] == -1


# ---------------------------------------------------------------------------
# eq. (2): injections against Kirchhoff's laws on the branch currents
# ---------------------------------------------------------------------------

def branch_power(g, vm, va, fr, to, r, x, b):
    """Complex power injected at each bus, summed over pi-model branch ends."""
    V = vm * np.exp(1j * va)
    S = np.zeros(g.n_bus, dtype=complex)
    for f, t, rr, xx, bb in zip(fr, to, r, x, b):
        ys = 1.0 / complex(rr, xx)
        I_f = ys * (V[f] - V[t]) + 0.5j * bb * V[f]
        I_t = ys * (V[t] - V[f]) + 0.5j * bb * V[t]
        S[f] += V[f] * np.conj(I_f)
        S[t] += V[t] * np.conj(I_t)
    return S


def test_injections_match_branch_currents():
    g = tiny(30, 41, 6, 11)
    # add a parallel branch to check that the admittances of parallel lines add
    g.fr = np.append(g.fr, g.fr[3]).astype(np.int32)
    g.to = np.append(g.to, g.to[3]).astype(np.int32)
    g.r, g.x, g.b = np.append(g.r, 0.02), np.append(g.x, 0.1), np.append(g.b, 0.01)
    g.n_branch += 1
    o = OracleGrid(g)
    rng = np.random.default_rng(5)
    vm = rng.uniform(0.9, 1.1, g.n_bus)
    va = rng.normal(0, 0.2, g.n_bus)
    P, Q = o.injections(vm, va)
    S = branch_power(g, vm, va, g.fr, g.to, g.r, g.x, g.b)
    np.testing.assert_allclose(P, S.real, rtol=0, atol=1e-10 * abs(S).max())
    np.testing.assert_allclose(Q, S.imag, rtol=0, atol=1e-10 * abs(S).max())


def test_lossless_injections_sum_to_zero():
    g = tiny(40, 55, 8, 12, lossless=True)
    o = OracleGrid(g)
    P, Q = o.injections(g.v_star, g.theta_star)
    assert abs(P.sum()) <= 1e-12 * abs(P).sum()


# ---------------------------------------------------------------------------
# eq. (3) and the Jacobians
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(5, 6, 2, 1), (9, 12, 3, 2), (14, 20, 5, 3), (30, 41, 6, 4)])
def test_jacobians_match_central_differences(shape):
    o = OracleGrid(tiny(*shape))
    st = o.plant()
    rng = np.random.default_rng(7)
    x = st.x + rng.normal(0, 0.05, o.n_x)      # off the solution: g != 0
    jx, jp = o.jacobians_dense(x, st.p)
    h = 1e-6
    fx = np.column_stack([(o.residual(x + h * e, st.p, st.pd, st.qd) - o.residual(x - h * e, st.p, st.pd, st.qd)) / (2 * h)
                          for e in np.eye(o.n_x)])
    fp = np.column_stack([(o.residual(x, st.p + h * e, st.pd, st.qd) - o.residual(x, st.p - h * e, st.pd, st.qd)) / (2 * h)
                          for e in np.eye(o.n_p)])
    assert abs(jx - fx).max() <= 1e-6 * abs(jx).max()
    assert abs(jp - fp).max() <= 1e-6 * abs(jp).max()
    # J_x is structurally symmetric (P_i pairs with theta_i, Q_i with v_i)
    assert ((jx != 0) == (jx.T != 0)).all()


def test_planted_point_and_newton_from_flat_start():
    g = gg.make_case("case118")
    o = OracleGrid(g)
    st = o.plant()
    assert abs(o.residual(st.x, st.p, st.pd, st.qd)).max() <= 1e-12
    x, status, iters, res = o.newton(st.p, st.pd, st.qd, flat_start(o))
    assert status == 0 and res <= 1e-12 and iters >= 3
    assert abs(x - st.x).max() <= 1e-8


# ---------------------------------------------------------------------------
# the oracle's LU (static fill-reducing order, no pivoting)
# ---------------------------------------------------------------------------

def test_lu_against_dense_factorisation():
    o = OracleGrid(tiny(30, 41, 6, 4))
    st = o.plant()
    jx, _ = o.jacobians_dense(st.x, st.p)
    perm, L, U = o.lu_dense(st.x, st.p)
    B = jx[np.ix_(perm, perm)]
    assert np.allclose(np.tril(L, -1) + np.eye(o.n_x), L) and np.allclose(np.triu(U), U)
    assert abs(L @ U - B).max() <= 1e-13 * abs(B).max()
    R = np.random.default_rng(3).normal(size=(o.n_x, 3))
    for trans in (False, True):
        X = o.solve(st.x, st.p, R, trans=trans)
        A = jx.T if trans else jx
        np.testing.assert_allclose(X, np.linalg.solve(A, R), rtol=1e-11, atol=1e-12 * abs(X).max())


# ---------------------------------------------------------------------------
# first order: lambda and the reduced gradient, eq. (6)-(7)
# ---------------------------------------------------------------------------

def reduced(o, st, p, tol=1e-13):
    x, status, _, _ = o.newton(p, st.pd, st.qd, st.x, tol=tol)
    assert status == 0
    return x


def test_adjoint_solves_first_order_condition():
    o = OracleGrid(tiny(30, 41, 6, 4))
    st = o.plant()
    lam, grad, F = o.adjoint(st.x, st.p, st.pd, st.qd)
    jx, _ = o.jacobians_dense(st.x, st.p)
    h = 1e-5
    dfdx = np.array([(o.objective(st.x + h * e, st.p, st.pd) - o.objective(st.x - h * e, st.p, st.pd)) / (2 * h)
                     for e in np.eye(o.n_x)])
    # grad_x f + lambda^T J_x = 0
    assert abs(dfdx + jx.T @ lam).max() <= 1e-7 * abs(dfdx).max()
    assert F == pytest.approx(o.objective(st.x, st.p, st.pd), rel=1e-15)


@pytest.mark.parametrize("shape", [(9, 12, 3, 2), (30, 41, 6, 4)])
def test_reduced_gradient_matches_central_differences(shape):
    o = OracleGrid(tiny(*shape))
    st = o.plant()
    _, grad, _ = o.adjoint(st.x, st.p, st.pd, st.qd)
    h = 1e-6
    fd = np.empty(o.n_p)
    for k in range(o.n_p):
        e = np.zeros(o.n_p)
        e[k] = h
        fd[k] = (o.objective(reduced(o, st, st.p + e), st.p + e, st.pd)
                 - o.objective(reduced(o, st, st.p - e), st.p - e, st.pd)) / (2 * h)
    assert abs(grad - fd).max() <= 1e-6 * abs(grad).max()


# ---------------------------------------------------------------------------
# second order: Hessian of the Lagrangian and the reduced Hessian
# ---------------------------------------------------------------------------

def test_lagrangian_hessian_matches_second_differences():
    o = OracleGrid(tiny(9, 12, 3, 2))
    st = o.plant()
    rng = np.random.default_rng(9)
    x = st.x + rng.normal(0, 0.05, o.n_x)
    lam = rng.normal(0, 100.0, o.n_x)
    K = o.lagrangian_hessian_dense(x, st.p, st.pd, lam)
    nx = o.n_x

    def ell(u):
        return o.objective(u[:nx], u[nx:], st.pd) + lam @ o.residual(u[:nx], u[nx:], st.pd, st.qd)

    u0 = np.concatenate([x, st.p])
    n = len(u0)
    h = 1e-4
    fd = np.empty((n, n))
    E = np.eye(n) * h
    for a in range(n):
        for b in range(n):
            fd[a, b] = (ell(u0 + E[a] + E[b]) - ell(u0 + E[a] - E[b]) - ell(u0 - E[a] + E[b])
                        + ell(u0 - E[a] - E[b])) / (4 * h * h)
    assert abs(K - K.T).max() <= 1e-14 * abs(K).max()
    assert abs(K - fd).max() <= 2e-6 * abs(K).max()


def full_hessian(o, st):
    return o.hessvec(st.x, st.p, st.pd, st.qd, np.eye(o.n_p))


@pytest.mark.parametrize("shape", [(5, 6, 2, 1), (9, 12, 3, 2), (14, 20, 5, 3), (30, 41, 6, 4)])
def test_reduced_hessian_matches_differences_of_gradient(shape):
    o = OracleGrid(tiny(*shape))
    st = o.plant()
    H = full_hessian(o, st)
    h = 1e-6
    fd = np.empty_like(H)
    for k in range(o.n_p):
        e = np.zeros(o.n_p)
        e[k] = h
        gp = o.adjoint(reduced(o, st, st.p + e), st.p + e, st.pd, st.qd)[1]
        gm = o.adjoint(reduced(o, st, st.p - e), st.p - e, st.pd, st.qd)[1]
        fd[:, k] = (gp - gm) / (2 * h)
    assert abs(H - fd).max() <= 1e-6 * abs(H).max()


def test_reduced_hessian_quadratic_form_matches_second_difference():
    o = OracleGrid(gg.make_case("case118"))
    st = o.plant()
    w = gg.random_directions(o.n_p, 1, 118)[:, 0]
    hw = o.hessvec(st.x, st.p, st.pd, st.qd, w[:, None])[:, 0]
    h = 1e-4

    def F(p):
        return o.objective(reduced(o, st, p), p, st.pd)

    d2 = (F(st.p + h * w) - 2 * F(st.p) + F(st.p - h * w)) / (h * h)
    assert w @ hw == pytest.approx(d2, rel=1e-5)


def test_reduced_hessian_is_symmetric():
    o = OracleGrid(gg.make_case("case118"))
    st = o.plant()
    H = full_hessian(o, st)
    assert abs(H - H.T).max() <= 1e-11 * abs(H).max()


def test_lossless_closed_form():
    """With r = 0 the losses vanish, so F(p) = sum_PV c_k(Pg_k) + c_ref(sum Pd - sum_PV Pg_k):
    H[Pg_k, Pg_l] = c''_k delta_kl + c''_ref and every v row and column is zero."""
    g = gg.make_grid(118, 186, 54, 20220100, lossless=True)
    o = OracleGrid(g)
    st = o.plant()
    H = full_hessian(o, st)
    _, _, ip_v, ip_pg = o.index_maps()
    S = g.base_mva
    ref = int(np.flatnonzero(g.bus_type == 0)[0])
    pv = np.flatnonzero(ip_pg >= 0)
    ng = int((ip_v >= 0).sum())
    expect = np.zeros((o.n_p, o.n_p))
    expect[ng:, ng:] = 2 * g.c2[ref] * S * S
    expect[ip_pg[pv], ip_pg[pv]] += 2 * g.c2[pv] * S * S
    assert abs(H - expect).max() <= 1e-9 * abs(expect).max()


def test_lossless_closed_form_case9241():
    """The same closed form at the size of the benchmark grid (all 2889 columns): the
    pipeline's cancellation holds through the large factorisation and every sweep."""
    g = gg.make_case("case9241", lossless=True)
    o = OracleGrid(g)
    st = o.plant()
    H = full_hessian(o, st)
    _, _, ip_v, ip_pg = o.index_maps()
    S = g.base_mva
    ref = int(np.flatnonzero(g.bus_type == 0)[0])
    pv = np.flatnonzero(ip_pg >= 0)
    ng = int((ip_v >= 0).sum())
    expect = np.zeros((o.n_p, o.n_p))
    expect[ng:, ng:] = 2 * g.c2[ref] * S * S
    expect[ip_pg[pv], ip_pg[pv]] += 2 * g.c2[pv] * S * S
    assert abs(H - expect).max() <= 1e-9 * abs(expect).max()


def test_bus_relabelling_permutes_the_hessian():
    g = gg.make_case("case118")
    o = OracleGrid(g)
    st = o.plant()
    H = full_hessian(o, st)
    rng = np.random.default_rng(4)
    pi = rng.permutation(g.n_bus)            # old bus id -> new bus id
    g2 = gg.make_case("case118")
    inv = np.argsort(pi)
    g2.fr, g2.to = pi[g.fr].astype(np.int32), pi[g.to].astype(np.int32)
    for name in ("bus_type", "v_star", "theta_star", "c2", "c1"):
        setattr(g2, name, getattr(g, name)[inv])
    o2 = OracleGrid(g2)
    st2 = o2.plant()
    H2 = full_hessian(o2, st2)
    # map p indices: variable of bus b in grid 1 is variable of bus pi[b] in grid 2
    _, _, ipv1, ipg1 = o.index_maps()
    _, _, ipv2, ipg2 = o2.index_maps()
    m = np.empty(o.n_p, dtype=int)
    for b in range(g.n_bus):
        if ipv1[b] >= 0:
            m[ipv1[b]] = ipv2[pi[b]]
        if ipg1[b] >= 0:
            m[ipg1[b]] = ipg2[pi[b]]
    assert abs(H2[np.ix_(m, m)] - H).max() <= 1e-10 * abs(H).max()


# ---------------------------------------------------------------------------
# symbolic data: ordering, patterns, levels (brute force on small graphs)
# ---------------------------------------------------------------------------

def brute_min_weighted_fill(g):
    """The ordering by its definition: at every step, score every remaining bus from
    scratch (the weight w_a * w_b of each pair of its neighbours that is not yet
    adjacent, w = 1 for a PV bus and 2 for a PQ bus; ties: the sum of w over its
    neighbours, then the bus id) and eliminate the smallest."""
    alive = {i for i in range(g.n_bus) if g.bus_type[i] != 0}
    w = {i: 2 if g.bus_type[i] == 2 else 1 for i in alive}
    adj = {i: set() for i in alive}
    for f, t in zip(g.fr, g.to):
        if f in alive and t in alive and f != t:
            adj[f].add(t)
            adj[t].add(f)

    def score(i):
        nb = sorted(adj[i])
        fill = sum(w[a] * w[b] for x, a in enumerate(nb) for b in nb[x + 1:] if b not in adj[a])
        return fill, sum(w[a] for a in nb), i

    order = []
    while alive:
        best = min(alive, key=score)
        nb = adj.pop(best)
        alive.remove(best)
        for a in nb:
            adj[a].discard(best)
            adj[a] |= nb - {a}
        order.append(best)
    return order


def _bus_graph(g):
    alive = {i for i in range(g.n_bus) if g.bus_type[i] != 0}
    adj = {i: set() for i in alive}
    for f, t in zip(g.fr, g.to):
        if f in alive and t in alive and f != t:
            adj[f].add(t)
            adj[t].add(f)
    return alive, adj


def brute_min_degree(g):
    alive, adj = _bus_graph(g)
    order = []
    while alive:
        best = min(alive, key=lambda i: (len(adj[i]), i))
        nb = adj.pop(best)
        alive.remove(best)
        for a in nb:
            adj[a].discard(best)
            adj[a] |= nb - {a}
        order.append(best)
    return order


def order_cost(g, order, n_dirs, level_cost=None):
    """Factor entries outside the bus blocks (w_k times the weight of the neighbours bus
    k has when eliminated) times n_dirs, plus level_cost (default: the grid record's
    order_level_cost) per forward level."""
    if level_cost is None:
        level_cost = g.order_level_cost
    alive, adj = _bus_graph(g)
    w = {i: 2 if g.bus_type[i] == 2 else 1 for i in alive}
    lev = {i: 0 for i in alive}
    entries = 0
    for b in order:
        nb = adj.pop(b)
        entries += w[b] * sum(w[c] for c in nb)
        for a in nb:
            lev[a] = max(lev[a], lev[b] + 1)
            adj[a].discard(b)
            adj[a] |= nb - {a}
    return entries * n_dirs + level_cost * (max(lev.values()) + 1)


def brute_static_order(g, n_p):
    md, mf = brute_min_degree(g), brute_min_weighted_fill(g)
    return mf if order_cost(g, mf, n_p) < order_cost(g, md, n_p) else md


@pytest.mark.parametrize("shape", [(9, 12, 3, 2), (30, 41, 6, 4), (118, 186, 54, 20220100)])
def test_both_candidate_orders_against_brute_force(shape):
    """Each of the oracle's two candidate orders equals its from-scratch definition, and
    the order it uses is the cheaper one by the stated cost (ties: minimum degree)."""
    g = tiny(*shape)
    o = OracleGrid(g)
    assert list(o.order("degree")) == brute_min_degree(g)
    assert list(o.order("fill")) == brute_min_weighted_fill(g)
    assert list(o.order("static")) == brute_static_order(g, o.n_p)


@pytest.mark.parametrize("level_cost", [0, 10**12])
def test_static_order_follows_the_level_cost_parameter(level_cost):
    """The level weight is a parameter of the grid record: 0 keeps the order with fewer
    entries, a huge weight the one with fewer levels, each as the brute force says."""
    import dataclasses
    g = dataclasses.replace(tiny(118, 186, 54, 20220100), order_level_cost=level_cost)
    o = OracleGrid(g)
    assert list(o.order("static")) == brute_static_order(g, o.n_p)


def test_weighted_fill_order_beats_minimum_degree_on_fill():
    """A property the heuristic is chosen for: on the 118-bus grid the factor it gives
    holds no more entries than the one of exact minimum degree."""
    g = tiny(118, 186, 54, 20220100)
    assert order_cost(g, brute_min_weighted_fill(g), 1, 0) <= order_cost(g, brute_min_degree(g), 1, 0)


@pytest.mark.parametrize("shape", [(9, 12, 3, 2), (30, 41, 6, 4), (118, 186, 54, 20220100)])
def test_symbolic_ordering_patterns_levels(shape):
    g = tiny(*shape)
    o = OracleGrid(g)
    sym = o.symbolic()
    assert list(sym["bus_order"]) == brute_static_order(g, o.n_p)
    ix_th, ix_v, _, _ = o.index_maps()
    perm = []
    for b in sym["bus_order"]:
        perm.append(ix_th[b])
        if ix_v[b] >= 0:
            perm.append(ix_v[b])
    assert list(sym["perm"]) == perm
    # patterns equal the nonzero pattern of a dense LU of random values placed on the
    # structural pattern of J_x (power-flow values can cancel exactly: P_i and Q_i
    # depend on angle differences only)
    st = o.plant()
    jx, _ = o.jacobians_dense(st.x + np.random.default_rng(1).normal(0, 0.01, o.n_x), st.p)
    n = o.n_x
    rng = np.random.default_rng(2)
    A = np.where(jx != 0, rng.uniform(-1, 1, (n, n)), 0.0) + n * np.eye(n)
    B = A[np.ix_(sym["perm"], sym["perm"])]
    L, U = np.eye(n), B.copy()
    for k in range(n):
        L[k + 1:, k] = U[k + 1:, k] / U[k, k]
        U[k + 1:, :] -= np.outer(L[k + 1:, k], U[k, :])
        U[k + 1:, k] = 0.0
    Lpat = np.zeros((n, n), bool)
    Upat = np.zeros((n, n), bool)
    for r in range(n):
        Lpat[r, sym["Lj"][sym["Lp"][r]:sym["Lp"][r + 1]]] = True
        Upat[r, sym["Uj"][sym["Up"][r]:sym["Up"][r + 1]]] = True
    assert ((np.tril(L, -1) != 0) == Lpat).all()
    assert ((U != 0) == Upat).all()
    assert (Lpat == Upat.T & ~np.eye(n, dtype=bool)).all()        # structural symmetry
    # levels: longest dependency chain between buses through L rows
    bus_of = np.repeat(np.arange(len(sym["bus_order"])),
                       [2 if ix_v[b] >= 0 else 1 for b in sym["bus_order"]])
    lev = np.zeros(len(sym["bus_order"]), int)
    for r in range(n):
        for c in np.flatnonzero(Lpat[r]):
            if bus_of[c] != bus_of[r]:
                lev[bus_of[r]] = max(lev[bus_of[r]], lev[bus_of[c]] + 1)
    assert (lev == sym["level"]).all()


# ---------------------------------------------------------------------------
# Real-time tracking step (section 6.3, eq. 18-19): dense Cholesky and solve
# ---------------------------------------------------------------------------

def _binom(n, k):
    from math import comb
    return comb(n, k)


def test_cholesky_of_pascal_matrix_is_the_binomial_matrix():
    """The symmetric Pascal matrix P_ij = C(i+j, i) factors as L L^T with
    L_ij = C(i, j) (Vandermonde's identity): an exact integer closed form."""
    from oracle import cholesky
    n = 15
    P = np.array([[_binom(i + j, i) for j in range(n)] for i in range(n)], dtype=float)
    L, info = cholesky(P)
    assert info == 0
    expect = np.array([[_binom(i, j) if j <= i else 0 for j in range(n)] for i in range(n)], dtype=float)
    assert np.array_equal(L, expect)


def test_cholesky_of_second_difference_matrix_closed_form():
    """tridiag(-1, 2, -1): L_kk = sqrt((k+2)/(k+1)), L_{k+1,k} = -sqrt((k+1)/(k+2)), zero elsewhere."""
    from oracle import cholesky
    n = 40
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    L, info = cholesky(T)
    assert info == 0
    k = np.arange(n)
    assert np.allclose(np.diag(L), np.sqrt((k + 2) / (k + 1)), rtol=1e-15, atol=0)
    assert np.allclose(np.diag(L, -1), -np.sqrt((k[:-1] + 1) / (k[:-1] + 2)), rtol=1e-15, atol=0)
    assert np.count_nonzero(L) == 2 * n - 1


def test_cholesky_reads_the_lower_triangle_and_matches_a_library_factor():
    from oracle import cholesky
    rng = np.random.default_rng(11)
    n = 57
    A = rng.standard_normal((n, n))
    H = A @ A.T / n + np.eye(n)
    garbage = H + np.triu(rng.standard_normal((n, n)) * 1e3, 1)   # upper triangle must not be read
    L, info = cholesky(garbage)
    assert info == 0
    assert np.array_equal(L, np.tril(L))
    assert np.abs(L - np.linalg.cholesky(H)).max() <= 1e-13 * np.abs(L).max()
    assert np.abs(L @ L.T - H).max() <= 1e-13 * np.abs(H).max()


def test_cholesky_reports_the_first_non_positive_pivot():
    from oracle import cholesky
    assert cholesky(np.diag([4.0, 9.0, -1.0, 16.0]))[1] == 3
    assert cholesky(np.array([[1.0, 2.0], [2.0, 1.0]]))[1] == 2       # 1 - 2^2 < 0
    assert cholesky(np.array([[1.0, 1.0], [1.0, 1.0]]))[1] == 2       # singular: pivot exactly 0
    assert cholesky(np.zeros((0, 0)))[1] == 0


def test_cholesky_solve_is_exact_on_an_integer_system():
    """Unit-diagonal integer L (Pascal): forward and back substitution are exact."""
    from oracle import cholesky, cholesky_solve
    n = 10
    P = np.array([[_binom(i + j, i) for j in range(n)] for i in range(n)], dtype=float)
    L, _ = cholesky(P)
    X = np.random.default_rng(3).integers(-5, 6, size=(n, 3)).astype(float)
    assert np.array_equal(cholesky_solve(L, P @ X), X)


def test_tracking_step_is_the_newton_direction_of_the_reduced_objective():
    """d = -H^{-1} grad F makes grad F(p + a d) = (1 - a) grad F(p) + O(a^2):
    the residual must shrink by 4 when a halves (independent power-flow solves
    and adjoint gradients at the moved parameters), F must decrease along d
    (the paper's descent direction), and H d = -g must hold."""
    g = gg.make_case("case118")
    o = OracleGrid(g)
    st = o.plant()
    pd, qd = 1.05 * st.pd, 1.05 * st.qd
    x, s, _, _ = o.newton(st.p, pd, qd, st.x)
    assert s == 0
    r = o.rto_step(x, st.p, pd, qd)
    g0, d = r["g"], r["d"]
    assert g0 @ d < 0
    assert np.abs(r["H"] @ d + g0).max() <= 1e-11 * np.abs(g0).max()
    res = []
    for a in (1e-4, 2e-4):
        xa, s, _, _ = o.newton(st.p + a * d, pd, qd, x)
        assert s == 0
        _, ga, Fa = o.adjoint(xa, st.p + a * d, pd, qd)
        assert Fa < r["F"]
        res.append(np.abs(ga - (1 - a) * g0).max())
    assert res[0] <= 1e-3 * 1e-4 * np.abs(g0).max()
    assert 3.9 < res[1] / res[0] < 4.1


def test_tracking_step_refuses_an_indefinite_reduced_hessian():
    """The 30-bus seed-4 grid has an indefinite reduced Hessian at its planted
    point (H_00 < 0): the Cholesky step stops at the first pivot."""
    from oracle import cholesky
    o = OracleGrid(tiny(30, 41, 6, 4))
    st = o.plant()
    H = o.hessvec(st.x, st.p, st.pd, st.qd, np.eye(o.n_p))
    assert H[0, 0] < 0 and np.linalg.eigvalsh(0.5 * (H + H.T))[0] < 0
    assert cholesky(H)[1] == 1
    with pytest.raises(RuntimeError, match="pivot 1"):
        o.rto_step(st.x, st.p, st.pd, st.qd)


# ---------------------------------------------------------------------------
# Column colouring of the Jacobians (section 4.2.2, Fig. 2)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case", ["tiny30", "case118", "case1354"])
def test_coloring_equals_library_greedy_on_the_column_intersection_graph(case):
    """The oracle's colouring is the greedy colouring (columns in index order,
    smallest colour unused by earlier conflicting columns) of the graph whose
    edges join columns sharing a row: rebuilt here with scipy (pattern of
    |J|^T |J|) and coloured by networkx's greedy routine in the same order."""
    nx = pytest.importorskip("networkx")
    g = tiny(30, 41, 6, 4) if case == "tiny30" else gg.make_case(case)
    o = OracleGrid(g)
    st = o.plant()
    Jx, Jp = o.jacobians_csc(st.x, st.p)
    cx, cp, ncx, ncp = o.coloring()
    for J, col, nc in ((Jx, cx, ncx), (Jp, cp, ncp)):
        S = J.copy()
        S.data[:] = 1.0
        C = (S.T @ S).tocoo()
        G = nx.Graph()
        G.add_nodes_from(range(J.shape[1]))
        G.add_edges_from((int(a), int(b)) for a, b in zip(C.row, C.col) if a != b)
        ref = nx.coloring.greedy_color(G, strategy=lambda G, colors: sorted(G.nodes()))
        assert [ref[q] for q in range(J.shape[1])] == list(col)
        assert nc == max(ref.values()) + 1


@pytest.mark.parametrize("case", ["case118", "case9241"])
def test_coloring_compresses_the_jacobian_exactly(case):
    """Fig. 2: J times the 0/1 seed of a colour holds, in every row, the one
    entry of that colour's columns; so every structural entry is recovered
    bit for bit, and no colouring can use fewer colours than the widest row."""
    o = OracleGrid(gg.make_case(case))
    st = o.plant()
    Jx, Jp = o.jacobians_csc(st.x, st.p)
    cx, cp, ncx, ncp = o.coloring()
    for J, col, nc in ((Jx, cx, ncx), (Jp, cp, ncp)):
        seeds = np.zeros((J.shape[1], nc))
        seeds[np.arange(J.shape[1]), col] = 1.0
        comp = J @ seeds                                  # n_rows x n_colours
        coo = J.tocoo()
        assert np.array_equal(comp[coo.row, col[coo.col]], coo.data)
        assert nc >= np.diff(J.tocsr().indptr).max()
        # columns of one colour never share a row
        for c in range(nc):
            sub = J[:, np.flatnonzero(col == c)]
            sub.data[:] = 1.0
            assert (sub.sum(axis=1) <= 1).all()


def test_sparse_jacobians_equal_the_dense_ones():
    o = OracleGrid(tiny(30, 41, 6, 4))
    st = o.plant()
    Jx, Jp = o.jacobians_csc(st.x, st.p)
    jx, jp = o.jacobians_dense(st.x, st.p)
    assert np.array_equal(Jx.toarray(), jx) and np.array_equal(Jp.toarray(), jp)


def test_threaded_oracle_equals_one_thread_bit_for_bit():
    """Sharing the columns of W out among threads changes no arithmetic: every column
    runs the same steps on its own work vectors."""
    o = OracleGrid(gg.make_case("case118"))
    st = o.plant()
    W = gg.random_directions(o.n_p, 37, 3)
    a = o.hessvec(st.x, st.p, st.pd, st.qd, W)
    for threads in (2, 5, 64):
        assert np.array_equal(o.hessvec(st.x, st.p, st.pd, st.qd, W, threads=threads), a)
