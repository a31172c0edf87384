// dense.cu -- dense FP64 Cholesky factorisation and solves of the real-time
// tracking step (section 6.3, eq. 18-19): H_t d_t = -g_t with H_t = L L^T.
//
// Right-looking tiled algorithm over TB x TB tiles of a column-major matrix:
// for every tile column k
//   k_chol_panel   CTA 0 factors the diagonal tile A_kk; CTA b > 0 solves the
//                  tile b rows below it, L_ik = A_ik L_kk^{-T}.  Each CTA
//                  eliminates the stacked [A_kk; A_ik] in shared memory
//                  (the diagonal part redundantly), so one launch finishes the
//                  whole tile column;
//   k_chol_update  every trailing tile (i, j), k < j <= i, takes
//                  A_ij -= L_ik L_jk^T (lower half only on the diagonal).
// The solves run one launch per tile: the forward sweep L y = b writes y into a
// workspace while the other CTAs of the launch subtract L_ik y_k from the
// right-hand side below it, and the backward sweep L^T x = y writes x back into
// B while its other CTAs update the workspace above.  Reads and writes of one
// launch never touch the same tile, so no launch needs a grid-wide barrier.
//
// Eliminations inside a tile keep the columns unscaled until the end
// (a_rc -= a_rj a_cj / a_jj), so a step reads only a column that nothing in
// that step writes: one barrier per step.  FP64 throughout; GB300 runs FP64 on
// the CUDA cores (the tensor cores have no fast FP64 mode), so the factorisation
// is bound by the DFMA rate and by the dependency chain of the tile columns.
#include <cuda_runtime.h>

#include <cstdint>

#include "rh_kernels.h"

namespace rh {
namespace {

constexpr int kDenseThreads = 256;

template <int TB>
__global__ void __launch_bounds__(kDenseThreads)
    k_chol_panel(int n, double* __restrict__ A, int64_t lda, int k, int* __restrict__ info, double* __restrict__ y) {
    constexpr int R = TB * TB / kDenseThreads;
    __shared__ double D[TB][TB + 1];
    __shared__ double X[TB][TB + 1];
    __shared__ double Inv[TB], Sq[TB], Sinv[TB];
    const int t = threadIdx.x;
    const int k0 = k * TB, kb = min(TB, n - k0);
    const int b = blockIdx.x;
    const int r0 = k0 + b * TB, rb = b ? min(TB, n - r0) : 0;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, r = e % TB, c = e / TB;
        // lower triangle of A_kk; padding rows/columns get a unit pivot and no coupling
        D[r][c] = (r < kb && c <= r) ? A[(k0 + r) + (int64_t)(k0 + c) * lda] : (r == c ? 1.0 : 0.0);
        if (b) X[r][c] = (r < rb && c < kb) ? A[(r0 + r) + (int64_t)(k0 + c) * lda] : 0.0;
    }
    __syncthreads();
    if (t == 0) Inv[0] = 1.0 / D[0][0];
    __syncthreads();
    // Unscaled elimination: after step j, D[r][j] = l_rj * l_jj and D[j][j] = l_jj^2.
    // The thread that completes the next pivot also forms its reciprocal, so a
    // step costs one multiply and one or two FMAs per element and no division.
    for (int j = 0; j < kb - 1; j++) {
        const double inv = Inv[j];
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int e = t + q * kDenseThreads, r = e % TB, c = e / TB;
            if (c > j) {
                const double lc = D[c][j] * inv;
                if (r >= c) {
                    D[r][c] -= D[r][j] * lc;
                    if (r == j + 1 && c == j + 1) Inv[j + 1] = 1.0 / D[r][c];
                }
                if (b) X[r][c] -= X[r][j] * lc;
            }
        }
        __syncthreads();
    }
    if (t < TB) {
        const double sq = sqrt(D[t][t]);
        Sq[t] = sq;
        Sinv[t] = 1.0 / sq;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, r = e % TB, c = e / TB;
        if (b == 0) {
            if (r < kb && c <= r) A[(k0 + r) + (int64_t)(k0 + c) * lda] = (r == c) ? Sq[c] : D[r][c] * Sinv[c];
        } else if (r < rb && c < kb) {
            A[(r0 + r) + (int64_t)(k0 + c) * lda] = X[r][c] * Sinv[c];
        }
    }
    if (b != 0) return;
    if (t == 0) {
        for (int j = 0; j < kb; j++)
            if (!(D[j][j] > 0.0)) {      // not positive, or NaN from an earlier failed pivot
                atomicCAS(info, 0, k0 + j + 1);
                break;
            }
    }
    // Fused forward solve of one right-hand side: y_k = L_kk^{-1} b_k in place
    // (b_k already holds b_k - sum_{m<k} L_km y_m from the earlier updates).
    // One warp, unscaled like the elimination: z_r -= D[r][j] z_j / D[j][j],
    // then y_r = z_r / l_rr.
    if (y && t < 32) {
        const int r = t;
        double z = (r < kb) ? y[k0 + r] : 0.0;
        for (int j = 0; j < kb - 1; j++) {
            const double zj = __shfl_sync(0xffffffffu, z, j) * Inv[j];
            if (r > j && r < kb) z -= D[r][j] * zj;
        }
        if (r < kb) y[k0 + r] = z * Sinv[r];
    }
}

template <int TB>
__global__ void __launch_bounds__(kDenseThreads)
    k_chol_update(int n, double* __restrict__ A, int64_t lda, int k, double* __restrict__ y) {
    constexpr int R = TB * TB / kDenseThreads;
    constexpr int CS = kDenseThreads / TB;      // column stride between a thread's outputs
    __shared__ double Li[TB][TB + 1];
    __shared__ double Lj[TB][TB + 1];
    const int t = threadIdx.x;
    const int k0 = k * TB, kb = min(TB, n - k0);
    const int nt = (n + TB - 1) / TB;
    const int64_t T = nt - k - 1;
    const int64_t lin = blockIdx.x;
    if (lin >= T * (T + 1) / 2) {
        // fused forward solve: b_i -= L_ik y_k for tile row i (one CTA per row)
        const int i0 = (k + 1 + (int)(lin - T * (T + 1) / 2)) * TB, ib = min(TB, n - i0);
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int e = t + q * kDenseThreads, r = e % TB, m = e / TB;
            Li[r][m] = (r < ib && m < kb) ? A[(i0 + r) + (int64_t)(k0 + m) * lda] : 0.0;
        }
        if (t < TB) Lj[0][t] = (t < kb) ? y[k0 + t] : 0.0;
        __syncthreads();
        if (t < ib) {
            double s = 0.0;
#pragma unroll
            for (int m = 0; m < TB; m++) s = fma(Li[t][m], Lj[0][m], s);
            y[i0 + t] -= s;
        }
        return;
    }
    // trailing tile (i, j) with k < j <= i from the linear block index
    int ii = (int)((sqrt(8.0 * (double)lin + 1.0) - 1.0) * 0.5);
    while ((int64_t)ii * (ii + 1) / 2 > lin) ii--;
    while ((int64_t)(ii + 1) * (ii + 2) / 2 <= lin) ii++;
    const int jj = (int)(lin - (int64_t)ii * (ii + 1) / 2);
    const int i0 = (k + 1 + ii) * TB, j0 = (k + 1 + jj) * TB;
    const int ib = min(TB, n - i0), jb = min(TB, n - j0);
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, r = e % TB, m = e / TB;
        Li[r][m] = (r < ib && m < kb) ? A[(i0 + r) + (int64_t)(k0 + m) * lda] : 0.0;
        Lj[r][m] = (r < jb && m < kb) ? A[(j0 + r) + (int64_t)(k0 + m) * lda] : 0.0;
    }
    __syncthreads();
    const int r = t % TB, c0 = t / TB;
    double acc[R];
#pragma unroll
    for (int q = 0; q < R; q++) acc[q] = 0.0;
#pragma unroll
    for (int m = 0; m < TB; m++) {
        const double a = Li[r][m];
#pragma unroll
        for (int q = 0; q < R; q++) acc[q] = fma(a, Lj[c0 + q * CS][m], acc[q]);
    }
    const bool diag = (i0 == j0);
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int c = c0 + q * CS;
        if (r < ib && c < jb && (!diag || r >= c)) A[(i0 + r) + (int64_t)(j0 + c) * lda] -= acc[q];
    }
}

// Forward sweep, tile k: y_k = L_kk^{-1} b_k (every CTA, redundantly); CTA 0
// stores y_k in Y, CTA b > 0 takes b_i -= L_ik y_k for tile i = k + b.
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
    const int t = threadIdx.x, r = t % TB, c = t / TB;
    const int col = blockIdx.y * RC + c;
    const bool live = col < nrhs;               // warp-uniform for TB >= 16: padding columns do no FP64 work
    const int k0 = k * TB, kb = min(TB, n - k0);
    const int b = blockIdx.x, i0 = k0 + b * TB, ib = b ? min(TB, n - i0) : 0;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, rr = e % TB, cc = e / TB;
        D[rr][cc] = (rr < kb && cc <= rr) ? L[(k0 + rr) + (int64_t)(k0 + cc) * ldl] : (rr == cc ? 1.0 : 0.0);
        if (b) M[rr][cc] = (rr < ib && cc < kb) ? L[(i0 + rr) + (int64_t)(k0 + cc) * ldl] : 0.0;
    }
    Yk[r][c] = (r < kb && live) ? B[(k0 + r) + (int64_t)col * ldb] : 0.0;
    __syncthreads();
    if (t < TB) Inv[t] = 1.0 / D[t][t];
    __syncthreads();
    for (int j = 0; j < kb - 1; j++) {
        if (live && r > j) Yk[r][c] -= D[r][j] * (Yk[j][c] * Inv[j]);
        __syncthreads();
    }
    const double y = live ? Yk[r][c] * Inv[r] : 0.0;
    __syncthreads();
    Yk[r][c] = y;
    if (b == 0) {
        if (r < kb && live) Y[(k0 + r) + (int64_t)col * n] = y;
        return;
    }
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
    Yk[r][c] = (r < kb && live) ? Y[(k0 + r) + (int64_t)col * n] : 0.0;
    __syncthreads();
    if (t < TB) Inv[t] = 1.0 / D[t][t];
    __syncthreads();
    for (int j = kb - 1; j > 0; j--) {
        if (live && r < j) Yk[r][c] -= D[j][r] * (Yk[j][c] * Inv[j]);
        __syncthreads();
    }
    const double x = live ? Yk[r][c] * Inv[r] : 0.0;
    __syncthreads();
    Yk[r][c] = x;
    if (b == 0) {
        if (r < kb && live) B[(k0 + r) + (int64_t)col * ldb] = x;
        return;
    }
    __syncthreads();
    if (live) {
        double s = 0.0;
#pragma unroll
        for (int m = 0; m < TB; m++) s = fma(M[m][r], Yk[m][c], s);
        Y[(i0 + r) + (int64_t)col * n] -= s;
    }
}

template <int TB>
cudaError_t potrf_tiles(int n, double* A, int64_t lda, int* info, double* y, cudaStream_t s) {
    const int nt = (n + TB - 1) / TB;
    for (int k = 0; k < nt; k++) {
        k_chol_panel<TB><<<nt - k, kDenseThreads, 0, s>>>(n, A, lda, k, info, y);
        const int64_t T = nt - k - 1;
        if (T > 0)
            k_chol_update<TB><<<(unsigned)(T * (T + 1) / 2 + (y ? T : 0)), kDenseThreads, 0, s>>>(n, A, lda, k, y);
    }
    return cudaGetLastError();
}

template <int TB>
cudaError_t potrs_tiles(int n, const double* L, int64_t ldl, double* B, int64_t ldb, int nrhs, double* Y,
                        bool forward, cudaStream_t s) {
    constexpr int RC = kDenseThreads / TB;
    const int nt = (n + TB - 1) / TB;
    const unsigned gy = (unsigned)((nrhs + RC - 1) / RC);
    if (forward)
        for (int k = 0; k < nt; k++)
            k_chol_fwd<TB><<<dim3(nt - k, gy), kDenseThreads, 0, s>>>(n, L, ldl, B, ldb, Y, nrhs, k);
    for (int k = nt - 1; k >= 0; k--)
        k_chol_bwd<TB><<<dim3(k + 1, gy), kDenseThreads, 0, s>>>(n, L, ldl, B, ldb, Y, nrhs, k);
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
