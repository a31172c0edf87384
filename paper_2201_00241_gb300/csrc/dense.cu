// dense.cu -- dense FP64 Cholesky factorisation and solves of the real-time
// tracking step (section 6.3, eq. 18-19): H_t d_t = -g_t with H_t = L L^T.
//
// Right-looking tiled algorithm over TB x TB tiles of a column-major matrix,
// one launch per tile column.  Launch k (k = -1 .. T - 1 for T tile columns;
// c = k + 1 is the column it factors) holds:
//   panel CTAs     one per tile i > c of column c: the tile and the diagonal
//                  tile take their last update (column k), the diagonal tile
//                  is factored, and L_ic = A_ic L_cc^{-T} is stored
//   a diagonal CTA that factors tile (k, k) once more and stores L_kk and the
//                  pivot status: the panel CTAs of launch k - 1 read that tile,
//                  so it is only overwritten one launch later
//   trailing CTAs  A_ij -= L_ik L_jk^T for every tile c < j <= i (lower half
//                  only on the diagonal)
//   with a right-hand side y (the fused forward solve L y = b): one CTA that
//   takes y_c -= L_ck y_k and solves y_c = L_cc^{-1} y_c, and one CTA per tile
//   row i > c that takes y_i -= L_ik y_k.
// Every CTA that needs L_cc factors the diagonal tile itself, from the same
// inputs with the same code, so all copies agree bit for bit.  The panel CTAs
// come first in the grid: they carry the launch's critical path (update,
// factorisation, triangular solve).  No launch reads a tile that another of
// its CTAs writes.
//
// The solves run one launch per tile: the forward sweep L y = b writes y into a
// workspace while the other CTAs of the launch subtract L_ik y_k from the
// right-hand side below it, and the backward sweep L^T x = y writes x back into
// B while its other CTAs update the workspace above.
//
// The diagonal tile is eliminated without divisions: step j replaces every
// trailing entry by 2^-e_j (d_j a_rc - a_rj a_cj), with d_j the current pivot and
// 2^-e_j the power of two that brings it into [1, 2) (cross-multiplied
// elimination, as in Bareiss's fraction-free Gaussian elimination, with an exact
// power-of-two rescaling in place of Bareiss's exact division).  The trailing
// block after step j is then s_{j+1} times the ordinary Schur complement, with
// s_{j+1} = s_j 2^-e_j d_j in [s_j, 2 s_j): bounded by 2^TB inside a tile.  At the
// end l_rc = a_rc / sqrt(s_c d_c) for r >= c (d_c = a_cc), one reciprocal
// square root per column, and 1 / l_cc = s_c / sqrt(s_c d_c) and
// 1 / d_c = s_c / (s_c d_c) follow by multiplications.  A step is one FMA and an
// exponent update on the critical path instead of a division.  GB300 runs FP64
// on the CUDA cores (the tensor cores have no fast FP64 mode) at one warp
// instruction per 64 cycles per SM sub-partition, and a dependent FP64
// instruction waits those 64 cycles, so every step also keeps its FP64 work on
// as few warps per sub-partition as it can.  The products square the entries'
// magnitudes, so every diagonal tile is first equilibrated by powers of two
// (load_diag).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "rh_kernels.h"

namespace rh {
namespace {

constexpr int kDenseThreads = 256;

// Entry p of the packed lower triangle of a TB x TB tile taken in reverse
// column-major order (p = 0 is the last column's last row): the entries of the
// columns > j are exactly p < (TB - 1 - j)(TB - j) / 2, so the entries that a
// step updates are the first threads of the CTA, one warp per sub-partition
// while they fit in four warps.
template <int TB>
__device__ __forceinline__ void packed_entry(int p, int& r, int& c) {
    const int e = TB * (TB + 1) / 2 - 1 - p;
    int cc = 0;
    while (cc + 1 < TB && (cc + 1) * TB - (cc + 1) * cc / 2 <= e) cc++;
    c = cc;
    r = cc + (e - (cc * TB - cc * (cc - 1) / 2));
}

// Loads the TB x TB tile of A at (i0, j0) with rb x cb live entries into T,
// zero elsewhere; lanes run along rows (coalesced).
template <int TB>
__device__ __forceinline__ void load_tile(double (*T)[TB + 1], const double* __restrict__ A, int64_t lda, int i0,
                                          int j0, int rb, int cb) {
    constexpr int R = TB * TB / kDenseThreads;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = threadIdx.x + q * kDenseThreads, r = e % TB, c = e / TB;
        T[r][c] = (r < rb && c < cb) ? A[(i0 + r) + (int64_t)(j0 + c) * lda] : 0.0;
    }
}

// 2^k for |k| <= 1022.
__device__ __forceinline__ double pow2i(int k) { return __longlong_as_double((long long)(1023 + k) << 52); }

// floor(exponent / 2) of a positive normal a (|result| <= 511); 0 otherwise.
__device__ __forceinline__ int half_exponent(double a) {
    const int f = (int)((__double_as_longlong(a) >> 52) & 0x7ff);
    return (a > 0.0 && f != 0 && f != 0x7ff) ? (f - 1023) >> 1 : 0;
}

// Loads the diagonal tile at (c0, c0) with kb live rows: its lower triangle,
// unit padding beyond kb, zero above the diagonal; the owners of the diagonal
// entries write Es[r], the half exponent of the stored a_rr (read after the
// caller's next barrier).
//
// The tile is then equilibrated (by syrk_diag with its last update, or by
// equilibrate_diag): row and column r scaled by 2^-Es[r].  The updates only
// lower the diagonal of a positive definite matrix, so every entry of the
// scaled tile and of its Schur complements is below 4 in magnitude and the
// cross-multiplied products of the elimination stay far inside the FP64 range
// whatever the scaling of the input.  The scaling is exact; the caller undoes
// it: l_rc of the input is 2^Es[r] times the scaled tile's, and right-hand sides
// are scaled by 2^-Es before the solves with the scaled tile's multipliers.
template <int TB>
__device__ __forceinline__ void load_diag(double (*D)[TB + 1], int* Es, const double* __restrict__ A, int64_t lda,
                                          int c0, int kb) {
    constexpr int R = TB * TB / kDenseThreads;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = threadIdx.x + q * kDenseThreads, r = e % TB, c = e / TB;
        const double a = (r < kb && c <= r) ? A[(c0 + r) + (int64_t)(c0 + c) * lda] : (r == c ? 1.0 : 0.0);
        D[r][c] = a;
        if (r == c) Es[r] = r < kb ? half_exponent(a) : 0;
    }
}

// Equilibrated last update of the diagonal tile: D = (D - Lc Lc^T) 2^-(Es[r] + Es[c])
// on the lower triangle (the scaled entry is formed beside the dot product, so
// the scaling adds nothing to the chain).
template <int TB>
__device__ __forceinline__ void syrk_diag(double (*D)[TB + 1], const double (*Lc)[TB + 1], const int* Es) {
    constexpr int NP = TB * (TB + 1) / 2;
    for (int p = threadIdx.x; p < NP; p += kDenseThreads) {
        int r, c;
        packed_entry<TB>(p, r, c);
        const double sc = pow2i(-(Es[r] + Es[c]));
        const double ds = D[r][c] * sc;
        double acc = 0.0;
#pragma unroll
        for (int m = 0; m < TB; m++) acc = fma(Lc[r][m], Lc[c][m], acc);
        D[r][c] = fma(-acc, sc, ds);
    }
}

// Equilibration of a diagonal tile without an update (the first tile column).
template <int TB>
__device__ __forceinline__ void equilibrate_diag(double (*D)[TB + 1], const int* Es) {
    constexpr int NP = TB * (TB + 1) / 2;
    for (int p = threadIdx.x; p < NP; p += kDenseThreads) {
        int r, c;
        packed_entry<TB>(p, r, c);
        D[r][c] *= pow2i(-(Es[r] + Es[c]));
    }
}

// Barrier among the first NB threads of the CTA: __syncthreads for the whole
// CTA, otherwise named barrier 1, so that the other warps can work meanwhile.
template <int NB>
__device__ __forceinline__ void tile_sync() {
    if constexpr (NB == kDenseThreads)
        __syncthreads();
    else
        asm volatile("bar.sync 1, %0;" ::"n"(NB) : "memory");
}

// Eliminates the diagonal tile held in D (lower triangle, unit-padded beyond
// kb) without divisions: afterwards D[r][c] = s_c a_rc for r >= c, with a_rc the
// entries of the ordinary elimination (a_cc the pivot d_c), and
//   W[c] = 1 / sqrt(s_c D[c][c]),  so l_rc = D[r][c] W[c] (the diagonal too),
//   Inv[c] = s_c W[c] = 1 / l_cc,  Rd[c] = s_c W[c]^2 = 1 / D[c][c].
// Run by the first NB threads of the CTA (and only by them); the last of them
// keeps the running product s in S.  Column 0 is never updated, so the
// TB (TB - 1) / 2 entries of the other columns are the ones that threads own.
template <int TB, int NB>
__device__ __forceinline__ void chol_tile(double (*D)[TB + 1], int kb, double* S, double* W, double* Inv,
                                          double* Rd) {
    constexpr int NU = TB * (TB - 1) / 2;
    constexpr int QP = (NU + NB - 1) / NB;
    const int t = threadIdx.x;
    int er[QP], ec[QP];
#pragma unroll
    for (int q = 0; q < QP; q++) packed_entry<TB>(min(t + q * NB, NU - 1), er[q], ec[q]);
    double s = 1.0;
    for (int j = 0; j < kb - 1; j++) {
        const int na = (TB - 1 - j) * (TB - j) / 2;
        const double d = D[j][j];
        const int sh = pivot_shift(d);
#pragma unroll
        for (int q = 0; q < QP; q++) {
            if (t + q * NB < na) {
                const int r = er[q], c = ec[q];
                const double prod = D[r][j] * D[c][j];
                D[r][c] = scale_pow2(fma(d, D[r][c], -prod), sh);
            }
        }
        if (t == NB - 1) {
            s *= scale_pow2(d, sh);
            S[j + 1] = s;
        }
        tile_sync<NB>();
    }
    if (t < kb) {
        const double st = t ? S[t] : 1.0;        // S[0] is never written (kb = 1 has no step)
        const double w = rsqrt(st * D[t][t]);
        W[t] = w;
        Inv[t] = st * w;
        Rd[t] = (st * w) * w;
    } else if (t < TB) {
        W[t] = 0.0;
        Inv[t] = 0.0;
        Rd[t] = 0.0;
    }
    tile_sync<NB>();
}

// Stores L_cc from an eliminated tile and records its first pivot that is not
// positive (or NaN from an earlier failure): the launches run in column order,
// so the first value written to info is the first failure overall.  s_c > 0
// while every earlier pivot is positive, so the sign of D[c][c] is the pivot's.
template <int TB>
__device__ __forceinline__ void chol_store_tile(double* __restrict__ A, int64_t lda, int k0, int kb,
                                                const double (*D)[TB + 1], const double* W, const int* Es,
                                                int* __restrict__ info) {
    constexpr int R = TB * TB / kDenseThreads;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = threadIdx.x + q * kDenseThreads, r = e % TB, c = e / TB;
        if (r < kb && c <= r) A[(k0 + r) + (int64_t)(k0 + c) * lda] = (D[r][c] * W[c]) * pow2i(Es[r]);
    }
    if (threadIdx.x == 0) {
        for (int j = 0; j < kb; j++)
            if (!(D[j][j] > 0.0)) {
                atomicCAS(info, 0, k0 + j + 1);
                break;
            }
    }
}

// After chol_tile: D[c][j] = l_cj / l_jj below the diagonal (the multipliers of
// the unscaled triangular solves).
template <int TB>
__device__ __forceinline__ void diag_multipliers(double (*D)[TB + 1], const double* Rd) {
    constexpr int NP = TB * (TB + 1) / 2;
    for (int p = threadIdx.x; p < NP; p += kDenseThreads) {
        int r, c;
        packed_entry<TB>(p, r, c);
        if (r > c) D[r][c] *= Rd[c];
    }
    __syncthreads();
}

// Launch k of the factorisation (see the top of this file); c = k + 1.
template <int TB>
__global__ void __launch_bounds__(kDenseThreads)
    k_chol_step(int n, double* __restrict__ A, int64_t lda, int k, double* __restrict__ y, int* __restrict__ info) {
    constexpr int R = TB * TB / kDenseThreads;
    constexpr int CS = kDenseThreads / TB;      // column (or row) stride between a thread's entries
    __shared__ double D[TB][TB + 1];
    __shared__ double X[TB][TB + 1];
    __shared__ double Li[TB][TB + 1];
    __shared__ double Lc[TB][TB + 1];
    __shared__ double S[TB], W[TB], Inv[TB], Rd[TB], Z[TB];
    __shared__ int Es[TB];
    const int t = threadIdx.x;
    const int nt = (n + TB - 1) / TB;
    const int c = k + 1;
    const int c0 = c * TB, k0 = k * TB;
    const int64_t U = c < nt ? nt - c - 1 : 0;  // tiles below the diagonal in column c
    const int64_t nd = k >= 0 ? 1 : 0, ny = (y && c < nt) ? 1 : 0;
    int64_t b = blockIdx.x;
    // programmatic dependent launch: everything below reads what the previous
    // launch wrote, so wait for it first.  The next launch is scheduled as this
    // one's CTAs exit (the implicit trigger; triggering at the start, which
    // keeps the next launch's CTAs resident and waiting, measured slower).
    pdl_wait();
    if (b < U) {
        // panel CTA: tile i of column c
        const int kb = min(TB, n - c0);
        const int i0 = c0 + (int)(b + 1) * TB, ib = min(TB, n - i0);
        load_diag<TB>(D, Es, A, lda, c0, kb);
        load_tile<TB>(X, A, lda, i0, c0, ib, kb);
        if (k >= 0) {
            load_tile<TB>(Lc, A, lda, c0, k0, kb, TB);
            load_tile<TB>(Li, A, lda, i0, k0, ib, TB);
        }
        __syncthreads();
        if (k >= 0)
            syrk_diag<TB>(D, Lc, Es);
        else
            equilibrate_diag<TB>(D, Es);
        __syncthreads();
        // the tile's update X = (A_ic - L_ik L_ck^T) 2^-E (columns scaled like the
        // equilibrated diagonal tile, so the scaled tile's solve applies)
        auto update_x = [&](int e) {
            const int r = e % TB, cc = e / TB;
            double acc = 0.0;
            if (k >= 0) {
#pragma unroll
                for (int m = 0; m < TB; m++) acc = fma(Li[r][m], Lc[cc][m], acc);
            }
            X[r][cc] = (X[r][cc] - acc) * pow2i(-Es[cc]);
        };
        if constexpr (TB * (TB - 1) / 2 <= kDenseThreads / 2) {
            // the factorisation needs half the CTA: the other half updates X meanwhile
            constexpr int H = kDenseThreads / 2;
            if (t < H) {
                chol_tile<TB, H>(D, kb, S, W, Inv, Rd);
            } else {
                for (int e = t - H; e < TB * TB; e += H) update_x(e);
            }
            __syncthreads();
        } else {
#pragma unroll
            for (int q = 0; q < R; q++) update_x(t + q * kDenseThreads);
            __syncthreads();
            chol_tile<TB, kDenseThreads>(D, kb, S, W, Inv, Rd);
        }
        diag_multipliers<TB>(D, Rd);
        // X L_cc^T = A_ic, unscaled (x_rj l_jj): the rows are independent, each
        // in TB lanes of one warp (one per column); a step broadcasts X[r][j]
        const int cl = t % TB, rt = t / TB;
        double x[R];
#pragma unroll
        for (int q = 0; q < R; q++) x[q] = X[rt + q * CS][cl];
#pragma unroll
        for (int j = 0; j < TB - 1; j++) {
            if (j < kb - 1) {
                const double mcj = D[cl][j];
#pragma unroll
                for (int q = 0; q < R; q++) {
                    const double xj = __shfl_sync(0xffffffffu, x[q], j, TB);
                    if (cl > j) x[q] = fma(-xj, mcj, x[q]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int r = rt + q * CS;
            if (r < ib && cl < kb) A[(i0 + r) + (int64_t)(c0 + cl) * lda] = x[q] * Inv[cl];
        }
        return;
    }
    b -= U;
    if (b < nd) {
        // diagonal CTA: L_kk, from tile (k, k) and its last update (column k - 1)
        const int kb = min(TB, n - k0);
        load_diag<TB>(D, Es, A, lda, k0, kb);
        if (k >= 1) load_tile<TB>(Lc, A, lda, k0, k0 - TB, kb, TB);
        __syncthreads();
        if (k >= 1)
            syrk_diag<TB>(D, Lc, Es);
        else
            equilibrate_diag<TB>(D, Es);
        __syncthreads();
        chol_tile<TB, kDenseThreads>(D, kb, S, W, Inv, Rd);
        chol_store_tile<TB>(A, lda, k0, kb, D, W, Es, info);
        return;
    }
    b -= nd;
    if (b < ny) {
        // y_c -= L_ck y_k, then y_c = L_cc^{-1} y_c, unscaled (z_j l_jj) like the panel
        const int kb = min(TB, n - c0);
        load_diag<TB>(D, Es, A, lda, c0, kb);
        if (k >= 0) {
            load_tile<TB>(Lc, A, lda, c0, k0, kb, TB);
            if (t < TB) X[0][t] = y[k0 + t];
        }
        // y_c 2^-E (E[t] as load_diag forms it): the scaled tile's solve applies
        if (t < TB)
            Z[t] = t < kb ? y[c0 + t] * pow2i(-half_exponent(A[(c0 + t) + (int64_t)(c0 + t) * lda])) : 0.0;
        __syncthreads();
        if (k >= 0) {
            syrk_diag<TB>(D, Lc, Es);
            if (t >= kDenseThreads - TB) {
                const int r = t - (kDenseThreads - TB);
                double acc = 0.0;
#pragma unroll
                for (int m = 0; m < TB; m++) acc = fma(Lc[r][m], X[0][m], acc);
                Z[r] = fma(-acc, pow2i(-Es[r]), Z[r]);
            }
        } else {
            equilibrate_diag<TB>(D, Es);
        }
        __syncthreads();
        chol_tile<TB, kDenseThreads>(D, kb, S, W, Inv, Rd);
        diag_multipliers<TB>(D, Rd);
        if (t < 32) {
            const int r = t % TB;
            double z = Z[r];
#pragma unroll
            for (int j = 0; j < TB - 1; j++) {
                if (j < kb - 1) {
                    const double zj = __shfl_sync(0xffffffffu, z, j, TB);
                    if (r > j) z = fma(-D[r][j], zj, z);
                }
            }
            if (t < TB && r < kb) y[c0 + r] = z * Inv[r];
        }
        return;
    }
    b -= ny;
    const int64_t ntr = U * (U + 1) / 2;
    if (b >= ntr) {
        // y_i -= L_ik y_k for tile row i > c
        const int i0 = c0 + (int)(b - ntr + 1) * TB, ib = min(TB, n - i0);
        load_tile<TB>(Li, A, lda, i0, k0, ib, TB);
        if (t < TB) X[0][t] = y[k0 + t];
        __syncthreads();
        if (t < ib) {
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < TB; m++) s = fma(Li[t][m], X[0][m], s);
            y[i0 + t] -= s;
        }
        return;
    }
    // trailing tile (i, j), c < j <= i, from the linear block index
    int ii = (int)((sqrt(8.0 * (double)b + 1.0) - 1.0) * 0.5);
    while ((int64_t)ii * (ii + 1) / 2 > b) ii--;
    while ((int64_t)(ii + 1) * (ii + 2) / 2 <= b) ii++;
    const int jj = (int)(b - (int64_t)ii * (ii + 1) / 2);
    const int i0 = c0 + (ii + 1) * TB, j0 = c0 + (jj + 1) * TB;
    const int ib = min(TB, n - i0), jb = min(TB, n - j0);
    const bool diag = (i0 == j0);
    const int r = t % TB, cb = t / TB;
    // the target entries are read before the barrier, next to the L tiles: no
    // other CTA of the launch reads or writes this tile
    double a0[R];
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int cc = cb + q * CS;
        a0[q] = (r < ib && cc < jb && (!diag || r >= cc)) ? A[(i0 + r) + (int64_t)(j0 + cc) * lda] : 0.0;
    }
    load_tile<TB>(Li, A, lda, i0, k0, ib, TB);
    load_tile<TB>(Lc, A, lda, j0, k0, jb, TB);
    __syncthreads();
    double acc[R];
#pragma unroll
    for (int q = 0; q < R; q++) acc[q] = 0.0;
#pragma unroll
    for (int m = 0; m < TB; m++) {
        const double a = Li[r][m];
#pragma unroll
        for (int q = 0; q < R; q++) acc[q] = fma(a, Lc[cb + q * CS][m], acc[q]);
    }
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int cc = cb + q * CS;
        if (r < ib && cc < jb && (!diag || r >= cc)) A[(i0 + r) + (int64_t)(j0 + cc) * lda] = a0[q] - acc[q];
    }
}

// Triangular solves, one launch per tile.  Every CTA loads the diagonal tile
// L_kk, forms the multipliers m_rj = l_rj / l_jj and solves its right-hand
// sides' slice of tile k redundantly: the TB values of one right-hand side live
// in TB lanes of a warp, a step broadcasts z_j with a shuffle and takes
// z_r -= m z_j (unscaled, z_j = x_j l_jj), no barrier; x_r = z_r / l_rr.
// Right-hand-side columns beyond nrhs do no FP64 work.
//
// Forward sweep, tile k: y_k = L_kk^{-1} b_k; CTA 0 stores y_k in Y, CTA b > 0
// takes b_i -= L_ik y_k for tile i = k + b.
template <int TB>
__global__ void __launch_bounds__(kDenseThreads)
    k_chol_fwd(int n, const double* __restrict__ L, int64_t ldl, double* __restrict__ B, int64_t ldb,
               double* __restrict__ Y, int nrhs, int k) {
    constexpr int R = TB * TB / kDenseThreads;
    constexpr int RC = kDenseThreads / TB;      // right-hand sides per CTA
    __shared__ double D[TB][TB + 1];
    __shared__ double M[TB][TB + 1];
    __shared__ double Yk[TB][RC + 1];
    __shared__ double Inv[TB];
    pdl_wait();
    const int t = threadIdx.x, r = t % TB, c = t / TB;
    const int col = blockIdx.y * RC + c;
    const bool live = col < nrhs;
    const int k0 = k * TB, kb = min(TB, n - k0);
    const int b = blockIdx.x, i0 = k0 + b * TB, ib = b ? min(TB, n - i0) : 0;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, rr = e % TB, cc = e / TB;
        D[rr][cc] = (rr < kb && cc <= rr) ? L[(k0 + rr) + (int64_t)(k0 + cc) * ldl] : (rr == cc ? 1.0 : 0.0);
        if (b) M[rr][cc] = (rr < ib && cc < kb) ? L[(i0 + rr) + (int64_t)(k0 + cc) * ldl] : 0.0;
    }
    double z = (r < kb && live) ? B[(k0 + r) + (int64_t)col * ldb] : 0.0;
    __syncthreads();
    if (t < TB) Inv[t] = 1.0 / D[t][t];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, rr = e % TB, cc = e / TB;
        if (rr > cc) D[rr][cc] *= Inv[cc];
    }
    __syncthreads();
    if (__any_sync(0xffffffffu, live)) {
#pragma unroll
        for (int j = 0; j < TB - 1; j++) {
            if (j < kb - 1) {
                const double zj = __shfl_sync(0xffffffffu, z, j, TB);
                if (live && r > j) z = fma(-D[r][j], zj, z);
            }
        }
    }
    const double y = live ? z * Inv[r] : 0.0;
    if (b == 0) {
        if (r < kb && live) Y[(k0 + r) + (int64_t)col * n] = y;
        return;
    }
    Yk[r][c] = y;
    __syncthreads();
    if (r < ib && live) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < TB; m++) s = fma(M[r][m], Yk[m][c], s);
        B[(i0 + r) + (int64_t)col * ldb] -= s;
    }
}

// Backward sweep, tile k (descending): x_k = L_kk^{-T} y_k; CTA 0 stores x_k in
// B, CTA b > 0 takes y_i -= L_ki^T x_k for tile i = k - b.
template <int TB>
__global__ void __launch_bounds__(kDenseThreads)
    k_chol_bwd(int n, const double* __restrict__ L, int64_t ldl, double* __restrict__ B, int64_t ldb,
               double* __restrict__ Y, int nrhs, int k) {
    constexpr int R = TB * TB / kDenseThreads;
    constexpr int RC = kDenseThreads / TB;
    __shared__ double D[TB][TB + 1];
    __shared__ double M[TB][TB + 1];     // M[m][r] = L(k0 + m, i0 + r)
    __shared__ double Yk[TB][RC + 1];
    __shared__ double Inv[TB];
    pdl_wait();
    const int t = threadIdx.x, r = t % TB, c = t / TB;
    const int col = blockIdx.y * RC + c;
    const bool live = col < nrhs;
    const int k0 = k * TB, kb = min(TB, n - k0);
    const int b = blockIdx.x, i0 = k0 - b * TB;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, rr = e % TB, cc = e / TB;
        D[rr][cc] = (rr < kb && cc <= rr) ? L[(k0 + rr) + (int64_t)(k0 + cc) * ldl] : (rr == cc ? 1.0 : 0.0);
        // rr indexes the row inside tile k (coalesced), cc the column inside tile i
        if (b) M[rr][cc] = (rr < kb) ? L[(k0 + rr) + (int64_t)(i0 + cc) * ldl] : 0.0;
    }
    double z = (r < kb && live) ? Y[(k0 + r) + (int64_t)col * n] : 0.0;
    __syncthreads();
    if (t < TB) Inv[t] = 1.0 / D[t][t];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, rr = e % TB, cc = e / TB;
        if (rr > cc) D[rr][cc] *= Inv[rr];       // l_jr / l_jj with j = rr > r = cc
    }
    __syncthreads();
    if (__any_sync(0xffffffffu, live)) {
#pragma unroll
        for (int j = TB - 1; j > 0; j--) {
            if (j < kb) {
                const double zj = __shfl_sync(0xffffffffu, z, j, TB);
                if (live && r < j) z = fma(-D[j][r], zj, z);
            }
        }
    }
    const double x = live ? z * Inv[r] : 0.0;
    if (b == 0) {
        if (r < kb && live) B[(k0 + r) + (int64_t)col * ldb] = x;
        return;
    }
    Yk[r][c] = x;
    __syncthreads();
    if (live) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < TB; m++) s = fma(M[m][r], Yk[m][c], s);
        Y[(i0 + r) + (int64_t)col * n] -= s;
    }
}

// Launches of at most 4.5 x (SM count) CTAs request enough dynamic shared
// memory (unused) that every CTA has an SM to itself: the panel CTAs, first in
// the grid, then run their latency-bound chain without trailing CTAs beside them
// on the FP64 pipes, and the trailing CTAs take the other SMs in waves.  Larger
// launches keep the default residency, where the waves would cost more.  The
// attribute is set once per device, outside stream capture.
constexpr int kMaxDenseDevices = 64;
struct DenseDevice {
    bool ready = false;
    int n_sm = 0;
    int solo16 = 0, solo32 = 0;   // dynamic bytes for one CTA per SM (0: not set)
};
std::mutex g_dense_mu;
DenseDevice g_dense[kMaxDenseDevices];

template <int TB>
int solo_smem_for(int per_sm, int optin) {
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_chol_step<TB>) != cudaSuccess) return 0;
    const int want = per_sm / 2 + 1024 - (int)fa.sharedSizeBytes;
    if (want <= 0 || want + (int)fa.sharedSizeBytes > optin) return 0;
    if (cudaFuncSetAttribute(k_chol_step<TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, want) != cudaSuccess)
        return 0;
    return want;
}

// The device's entry, prepared on first use outside a stream capture; nullptr
// when it cannot be (the launches then keep the default residency).
const DenseDevice* dense_device(cudaStream_t s) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDenseDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_dense_mu);
    DenseDevice& d = g_dense[dev];
    if (d.ready) return &d;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    int per_sm = 0, optin = 0;
    if (cudaDeviceGetAttribute(&d.n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return nullptr;
    d.solo16 = solo_smem_for<16>(per_sm, optin);
    d.solo32 = solo_smem_for<32>(per_sm, optin);
    d.ready = true;
    return &d;
}

template <int TB>
cudaError_t potrf_tiles(int n, double* A, int64_t lda, int* info, double* y, cudaStream_t s) {
    const DenseDevice* dd = dense_device(s);
    const int solo = dd ? (TB == 16 ? dd->solo16 : dd->solo32) : 0;
    const int nt = (n + TB - 1) / TB;
    bool pdl = false;   // the first launch follows the memset of info
    for (int k = -1; k < nt; k++) {
        const int c = k + 1;
        const int64_t U = c < nt ? nt - c - 1 : 0;
        const int64_t grid = U + (k >= 0 ? 1 : 0) + ((y && c < nt) ? 1 : 0) + (k >= 0 ? U * (U + 1) / 2 : 0) +
                             ((y && k >= 0) ? U : 0);
        if (grid == 0) continue;
        const size_t dyn = (solo > 0 && 2 * grid <= 9 * (int64_t)dd->n_sm) ? (size_t)solo : 0;
        const cudaError_t e = launch_pdl(pdl, k_chol_step<TB>, dim3((unsigned)grid), dim3(kDenseThreads), dyn, s, n,
                                         A, lda, k, y, info);
        if (e != cudaSuccess) return e;
        pdl = true;
    }
    return cudaGetLastError();
}

template <int TB>
cudaError_t potrs_tiles(int n, const double* L, int64_t ldl, double* B, int64_t ldb, int nrhs, double* Y,
                        bool forward, cudaStream_t s) {
    constexpr int RC = kDenseThreads / TB;
    const int nt = (n + TB - 1) / TB;
    const unsigned gy = (unsigned)((nrhs + RC - 1) / RC);
    bool pdl = false;   // the first launch follows whatever the caller enqueued
    if (forward)
        for (int k = 0; k < nt; k++) {
            const cudaError_t e = launch_pdl(pdl, k_chol_fwd<TB>, dim3(nt - k, gy), dim3(kDenseThreads), 0, s, n, L,
                                             ldl, B, ldb, Y, nrhs, k);
            if (e != cudaSuccess) return e;
            pdl = true;
        }
    for (int k = nt - 1; k >= 0; k--) {
        const cudaError_t e = launch_pdl(pdl, k_chol_bwd<TB>, dim3(k + 1, gy), dim3(kDenseThreads), 0, s, n, L, ldl,
                                         B, ldb, Y, nrhs, k);
        if (e != cudaSuccess) return e;
        pdl = true;
    }
    return cudaGetLastError();
}

}  // namespace

int dense_tile(int n) { return n <= 2048 ? 16 : 32; }

cudaError_t launch_potrf(int n, double* A, int64_t lda, int* info, double* y, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(info, 0, sizeof(int), s);
    if (e != cudaSuccess || n == 0) return e;
    return dense_tile(n) == 16 ? potrf_tiles<16>(n, A, lda, info, y, s) : potrf_tiles<32>(n, A, lda, info, y, s);
}

cudaError_t launch_potrs(int n, const double* L, int64_t ldl, double* B, int64_t ldb, int nrhs, double* work,
                         bool forward, cudaStream_t s) {
    if (n == 0 || nrhs == 0) return cudaSuccess;
    return dense_tile(n) == 16 ? potrs_tiles<16>(n, L, ldl, B, ldb, nrhs, work, forward, s)
                               : potrs_tiles<32>(n, L, ldl, B, ldb, nrhs, work, forward, s);
}

}  // namespace rh
