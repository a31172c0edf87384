"""The launch schedules of the dense factorisations, emulated on the host.

`csrc/dense.cu` (the tracking step's Cholesky) and the dense-tail LU of
`csrc/kernels.cu` run one launch per tile column, in which panel CTAs refactor
the diagonal tile redundantly, a diagonal CTA stores the previous column's
diagonal tile one launch later, and trailing CTAs apply the column's update.
These tests replay that schedule tile by tile in numpy, CTA by CTA, with the
kernels' arithmetic for the diagonal tile (power-of-two equilibration for the
Cholesky, cross-multiplied elimination steps with an exact power-of-two
rescale, the multipliers and scales formed from the running product s):

* within a launch no CTA writes a tile that another CTA of the launch reads or
  writes (the launches need no grid-wide synchronisation);
* the factors (and the fused forward solve) agree with plain textbook
  factorisations (numpy's Cholesky and triangular solve; an unpivoted LU
  written out here) to rounding, over one tile, ragged tails and several tile
  columns, and for matrices scaled by powers of two far beyond the square root
  of the FP64 range, where the cross-multiplied products would overflow
  without the equilibration.

Runs without a GPU; the kernels' own parity is tested on the GPU against the
oracle (tests/test_gpu_rto.py, the refactorisation parity tests).
"""
import math

import numpy as np
import pytest

TINY = np.finfo(float).tiny


def pivot_shift(d):
    """e with 2^-e d in [1, 2) for a positive normal d (e <= 1022), else 0."""
    if not (d >= TINY) or not math.isfinite(d):
        return 0
    return min(math.frexp(d)[1] - 1, 1022)


def half_exponent(a):
    """floor((exponent of a) / 2) for a positive normal a, else 0."""
    if not (a >= TINY) or not math.isfinite(a):
        return 0
    return (math.frexp(a)[1] - 1) >> 1


def eliminate(D, kb, symmetric):
    """Cross-multiplied elimination of the tile D (unit-padded beyond kb), the
    lower triangle only when symmetric: returns the tile and s_0 .. s_{TB-1}."""
    TB = D.shape[0]
    D = D.copy()
    s, S = 1.0, [1.0]
    for j in range(kb - 1):
        d = D[j, j]
        sh = pivot_shift(d)
        for c in range(j + 1, TB):
            for r in range(c if symmetric else j + 1, TB):
                other = D[c, j] if symmetric else D[j, c]
                D[r, c] = math.ldexp(d * D[r, c] - D[r, j] * other, -sh)
        s *= math.ldexp(d, -sh)
        S.append(s)
    return D, np.array(S + [0.0] * (TB - len(S)))


def check_launch(reads, writes, k):
    for a, wa in enumerate(writes):
        for b, (rb, wb) in enumerate(zip(reads, writes)):
            if a != b:
                assert not (wa & (rb | wb)), (k, sorted(wa), sorted(rb | wb))


# ---- Cholesky (csrc/dense.cu) ------------------------------------------------------

def chol_factor_tile(Ds, kb):
    """The kernel's factorisation of an equilibrated diagonal tile (lower triangle):
    elimination, W = 1/sqrt(s d), Inv = s W, Rd = s W^2."""
    TB = Ds.shape[0]
    Ds, S = eliminate(Ds, kb, True)
    W, Inv, Rd = np.zeros(TB), np.zeros(TB), np.zeros(TB)
    for t in range(kb):
        w = 1.0 / math.sqrt(S[t] * Ds[t, t])
        W[t], Inv[t], Rd[t] = w, S[t] * w, S[t] * w * w
    return Ds, W, Inv, Rd


def chol_schedule(H, b, TB):
    n = H.shape[0]
    A = np.tril(H).copy()
    y = b.copy()
    nt = (n + TB - 1) // TB

    def sl(i):
        return slice(i * TB, min(n, (i + 1) * TB))

    def diag(c, k):
        # equilibrated at load by 2^-(E_r + E_c), E the half exponents of the stored
        # diagonal; the last update is scaled the same way
        kb = min(TB, n - c * TB)
        E = np.array([half_exponent(A[c * TB + t, c * TB + t]) if t < kb else 0 for t in range(TB)])
        sc = np.array([[math.ldexp(1.0, -int(E[r] + E[q])) for q in range(TB)] for r in range(TB)])
        D = np.eye(TB)
        D[:kb, :kb] = np.tril(A[sl(c), sl(c)]) * sc[:kb, :kb]
        rd = {(c, c)}
        if k >= 0:
            Lc = np.zeros((TB, TB))
            Lc[:kb, :] = A[sl(c), sl(k)]
            D -= np.tril(Lc @ Lc.T) * sc
            rd.add((c, k))
        return chol_factor_tile(D, kb) + (E, kb, rd)

    for k in range(-1, nt):
        c = k + 1
        U = nt - c - 1 if c < nt else 0
        reads, writes, out, ynew = [], [], [], {}
        for bb in range(U):                                   # panel CTAs
            i = c + 1 + bb
            Ds, W, Inv, Rd, E, kb, rd = diag(c, k)
            ib = min(TB, n - i * TB)
            X = np.zeros((TB, TB))
            X[:ib, :kb] = A[sl(i), sl(c)]
            rd = rd | {(i, c)}
            if k >= 0:
                Li = np.zeros((TB, TB))
                Li[:ib, :] = A[sl(i), sl(k)]
                Lc = np.zeros((TB, TB))
                Lc[:kb, :] = A[sl(c), sl(k)]
                X -= Li @ Lc.T
                rd.add((i, k))
            M = Ds.copy()
            for cc in range(TB):
                M[cc + 1:, cc] *= Rd[cc]
            X = X * np.array([math.ldexp(1.0, -int(e)) for e in E])[None, :]
            for r in range(TB):
                x = X[r].copy()
                for j in range(kb - 1):
                    x[j + 1:] -= x[j] * M[j + 1:, j]
                X[r] = x * Inv
            reads.append(rd)
            writes.append({(i, c)})
            out.append(((i, c), X[:ib, :kb]))
        if k >= 0:                                            # diagonal CTA
            Ds, W, Inv, Rd, E, kb, rd = diag(k, k - 1)
            L = np.tril(Ds * W[None, :]) * np.array([math.ldexp(1.0, int(e)) for e in E])[:, None]
            reads.append(rd)
            writes.append({(k, k)})
            out.append(((k, k), L[:kb, :kb]))
        if c < nt:                                            # y_c solve
            Ds, W, Inv, Rd, E, kb, rd = diag(c, k)
            z = np.zeros(TB)
            z[:kb] = y[sl(c)] - (A[sl(c), sl(k)] @ y[sl(k)] if k >= 0 else 0.0)
            z *= np.array([math.ldexp(1.0, -int(e)) for e in E])
            for j in range(kb - 1):
                z[j + 1:] -= Ds[j + 1:, j] * Rd[j] * z[j]
            ynew[c] = (z * Inv)[:kb]
            reads.append(rd | {("y", c), ("y", k)})
            writes.append({("y", c)})
        if k >= 0:
            for ii in range(U):                               # trailing and y-update CTAs
                i = c + 1 + ii
                for jj in range(ii + 1):
                    j = c + 1 + jj
                    reads.append({(i, k), (j, k), (i, j)})
                    writes.append({(i, j)})
                    upd = A[sl(i), sl(j)] - A[sl(i), sl(k)] @ A[sl(j), sl(k)].T
                    out.append(((i, j), np.tril(upd) if i == j else upd))
                reads.append({(i, k), ("y", k), ("y", i)})
                writes.append({("y", i)})
                ynew[i] = y[sl(i)] - A[sl(i), sl(k)] @ y[sl(k)]
        check_launch(reads, writes, k)
        for (i, j), v in out:
            A[sl(i), sl(j)] = v
        for i, v in ynew.items():
            y[sl(i)] = v
    return A, y


def spd(n, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    return M @ M.T / n + np.eye(n), rng.standard_normal(n)


@pytest.mark.parametrize("n,TB", [(1, 16), (5, 16), (16, 16), (17, 16), (40, 16), (70, 32), (33, 32)])
def test_cholesky_schedule_matches_textbook_factor(n, TB):
    H, b = spd(n, n)
    L, y = chol_schedule(H, b, TB)
    Lr = np.linalg.cholesky(H)
    yr = np.linalg.solve(Lr, b)
    assert np.abs(L - Lr).max() <= 64 * n * np.finfo(float).eps * np.abs(Lr).max()
    assert np.abs(y - yr).max() <= 64 * n * np.finfo(float).eps * np.abs(yr).max() * np.linalg.cond(Lr)


@pytest.mark.parametrize("spread", [0, 600, 1000])
def test_cholesky_schedule_under_extreme_power_of_two_scaling(spread):
    # H_s = P H P with P = diag(2^k_i): L(H_s) = P L(H) exactly in exact arithmetic.
    # Uniform 2^450 makes the entries about 2^900, whose products leave the FP64
    # range; the spreads put the diagonal between 2^-spread and 2^spread.
    n, TB = 40, 16
    H, b = spd(n, 3)
    rng = np.random.default_rng(9)
    k = rng.integers(-spread // 2, spread // 2 + 1, n) if spread else np.full(n, 450)
    P = np.array([math.ldexp(1.0, int(e)) for e in k])
    Hs = H * P[:, None] * P[None, :]
    L, _ = chol_schedule(Hs, b, TB)
    Lr = np.linalg.cholesky(H)
    assert np.all(np.isfinite(L))
    assert np.abs(L / P[:, None] - Lr).max() <= 64 * n * np.finfo(float).eps * np.abs(Lr).max()


# ---- dense-tail LU (csrc/kernels.cu, k_tail_step) ------------------------------------

def lu_schedule(A0, TB=16):
    """Row-major T x T tail, one launch per tile column; L unit lower below the
    diagonal, U on and above it, as the kernels store them."""
    T = A0.shape[0]
    A = A0.copy()
    nt = (T + TB - 1) // TB

    def sl(i):
        return slice(i * TB, min(T, (i + 1) * TB))

    def diag(c, k):
        kb = min(TB, T - c * TB)
        D = np.eye(TB)
        D[:kb, :kb] = A[sl(c), sl(c)]
        rd = {(c, c)}
        if k >= 0:
            Lk = np.zeros((TB, TB))
            Lk[:kb, :] = A[sl(c), sl(k)]
            Uk = np.zeros((TB, TB))
            Uk[:, :kb] = A[sl(k), sl(c)]
            D -= Lk @ Uk
            rd |= {(c, k), (k, c)}
        Dk, S = eliminate(D, kb, False)
        Rd = np.array([1.0 / Dk[t, t] if t < kb else 0.0 for t in range(TB)])
        return Dk, S, Rd, kb, rd

    for k in range(-1, nt):
        c = k + 1
        U = nt - c - 1 if c < nt else 0
        reads, writes, out = [], [], []
        for bb in range(2 * U):                                # panel CTAs
            ltile = bb < U
            o = c + 1 + (bb if ltile else bb - U)
            Dk, S, Rd, kb, rd = diag(c, k)
            M = Dk.copy()
            for r in range(TB):
                for cc in range(TB):
                    if r != cc:
                        M[r, cc] *= Rd[min(r, cc)]
            ob = min(TB, T - o * TB)
            X = np.zeros((TB, TB))
            if ltile:                                          # X U_cc = A_oc
                X[:ob, :kb] = A[sl(o), sl(c)]
                rd |= {(o, c)}
                if k >= 0:
                    Xk = np.zeros((TB, TB))
                    Xk[:ob, :] = A[sl(o), sl(k)]
                    Uk = np.zeros((TB, TB))
                    Uk[:, :kb] = A[sl(k), sl(c)]
                    X -= Xk @ Uk
                    rd.add((o, k))
                for r in range(TB):
                    x = X[r].copy()
                    for j in range(kb - 1):
                        x[j + 1:] -= x[j] * M[j, j + 1:]
                    X[r] = x * S * Rd
                out.append(((o, c), X[:ob, :kb]))
                writes.append({(o, c)})
            else:                                              # L_cc Y = A_co, unit L
                X[:kb, :ob] = A[sl(c), sl(o)]
                rd |= {(c, o)}
                if k >= 0:
                    Xk = np.zeros((TB, TB))
                    Xk[:, :ob] = A[sl(k), sl(o)]
                    Lk = np.zeros((TB, TB))
                    Lk[:kb, :] = A[sl(c), sl(k)]
                    X -= Lk @ Xk
                    rd.add((k, o))
                for col in range(TB):
                    yv = X[:, col].copy()
                    for j in range(kb - 1):
                        yv[j + 1:] -= M[j + 1:, j] * yv[j]
                    X[:, col] = yv
                out.append(((c, o), X[:kb, :ob]))
                writes.append({(c, o)})
            reads.append(rd)
        if k >= 0:                                             # diagonal CTA
            Dk, S, Rd, kb, rd = diag(k, k - 1)
            Z = np.empty((kb, kb))
            for r in range(kb):
                for cc in range(kb):
                    Z[r, cc] = Dk[r, cc] * Rd[cc] if r > cc else Dk[r, cc] * (1.0 / S[r])
            out.append(((k, k), Z))
            reads.append(rd)
            writes.append({(k, k)})
            for bi in range(U):                                # trailing CTAs
                for bj in range(U):
                    i, j = c + 1 + bi, c + 1 + bj
                    reads.append({(i, k), (k, j), (i, j)})
                    writes.append({(i, j)})
                    out.append(((i, j), A[sl(i), sl(j)] - A[sl(i), sl(k)] @ A[sl(k), sl(j)]))
        check_launch(reads, writes, k)
        for (i, j), v in out:
            A[sl(i), sl(j)] = v
    return A


def textbook_lu(A0):
    """Unpivoted right-looking LU: multipliers below the diagonal, U on and above."""
    R = A0.copy()
    for j in range(R.shape[0]):
        R[j + 1:, j] /= R[j, j]
        R[j + 1:, j + 1:] -= np.outer(R[j + 1:, j], R[j, j + 1:])
    return R


@pytest.mark.parametrize("T", [1, 5, 16, 17, 40, 48, 100, 128])
def test_tail_lu_schedule_matches_textbook_lu(T):
    rng = np.random.default_rng(T)
    A0 = rng.standard_normal((T, T)) + 3.0 * math.sqrt(T) * np.eye(T)   # no pivoting needed
    got = lu_schedule(A0)
    ref = textbook_lu(A0)
    assert np.abs(got - ref).max() <= 64 * T * np.finfo(float).eps * np.abs(ref).max()
