// dense.cu -- dense FP64 Cholesky factorisation and solves of the real-time
// tracking step (section 6.3, eq. 18-19): H_t d_t = -g_t with H_t = L L^T.
//
// Right-looking tiled algorithm over TB x TB tiles of a column-major matrix.
// The diagonal tile of tile column k is factored by the CTA that gives it its
// last trailing update (in the update launch of column k - 1; k_chol_diag0 for
// the first one), so no launch reads a tile that another of its CTAs writes:
//   k_chol_panel   L_ik = A_ik L_kk^{-T} for every tile i below the diagonal,
//                  one CTA each; fused: the forward solve y_k = L_kk^{-1} b_k
//   k_chol_update  A_ij -= L_ik L_jk^T for every trailing tile, k < j <= i
//                  (lower half only on the diagonal); the CTA of tile
//                  (k + 1, k + 1) then factors it; fused: b_i -= L_ik y_k
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

// Eliminates the symmetric tile held (lower triangle, unit-padded beyond kb) in
// D: afterwards D[r][c] = l_rc l_cc for r >= c, Sq[c] = l_cc, Sinv[c] = 1 / l_cc.
// The thread that completes the next pivot forms its reciprocal, so a step is
// one multiply and one FMA per element and no division.
template <int TB>
__device__ __forceinline__ void chol_tile(double (*D)[TB + 1], int kb, double* Inv, double* Sq, double* Sinv) {
    constexpr int R = TB * TB / kDenseThreads;
    const int t = threadIdx.x;
    if (t == 0) Inv[0] = 1.0 / D[0][0];
    __syncthreads();
    for (int j = 0; j < kb - 1; j++) {
        const double inv = Inv[j];
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int e = t + q * kDenseThreads, r = e % TB, c = e / TB;
            if (c > j && r >= c) {
                const double lc = D[c][j] * inv;
                D[r][c] = fma(-D[r][j], lc, D[r][c]);
                if (r == j + 1 && c == j + 1) Inv[j + 1] = 1.0 / D[r][c];
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
}

// Stores L_kk from an eliminated tile and records its first pivot that is not
// positive (or NaN from an earlier failure): the steps run in order, so the
// first value written to info is the first failure overall.
template <int TB>
__device__ __forceinline__ void chol_store_tile(double* __restrict__ A, int64_t lda, int k0, int kb,
                                                const double (*D)[TB + 1], const double* Sq, const double* Sinv,
                                                int* __restrict__ info) {
    constexpr int R = TB * TB / kDenseThreads;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = threadIdx.x + q * kDenseThreads, r = e % TB, c = e / TB;
        if (r < kb && c <= r) A[(k0 + r) + (int64_t)(k0 + c) * lda] = (r == c) ? Sq[c] : D[r][c] * Sinv[c];
    }
    if (threadIdx.x == 0) {
        for (int j = 0; j < kb; j++)
            if (!(D[j][j] > 0.0)) {
                atomicCAS(info, 0, k0 + j + 1);
                break;
            }
    }
}

template <int TB>
__global__ void __launch_bounds__(kDenseThreads) k_chol_diag0(int n, double* __restrict__ A, int64_t lda,
                                                              int* __restrict__ info) {
    constexpr int R = TB * TB / kDenseThreads;
    __shared__ double D[TB][TB + 1];
    __shared__ double Inv[TB], Sq[TB], Sinv[TB];
    const int kb = min(TB, n);
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = threadIdx.x + q * kDenseThreads, r = e % TB, c = e / TB;
        D[r][c] = (r < kb && c <= r) ? A[r + (int64_t)c * lda] : (r == c ? 1.0 : 0.0);
    }
    __syncthreads();
    chol_tile<TB>(D, kb, Inv, Sq, Sinv);
    chol_store_tile<TB>(A, lda, 0, kb, D, Sq, Sinv, info);
}

// Tile column k, with L_kk already stored: CTA b < m solves tile k + 1 + b,
// X L_kk^T = A_ik; CTA m (only with y) solves y_k = L_kk^{-1} y_k in place.
// With M[c][j] = l_cj / l_jj and X kept unscaled (x_rj l_jj), a step is
// X[r][c] -= X[r][j] M[c][j]; the result is x_rc = X[r][c] / l_cc.
template <int TB>
__global__ void __launch_bounds__(kDenseThreads)
    k_chol_panel(int n, double* __restrict__ A, int64_t lda, int k, double* __restrict__ y) {
    constexpr int R = TB * TB / kDenseThreads;
    __shared__ double M[TB][TB + 1];
    __shared__ double X[TB][TB + 1];
    __shared__ double Inv[TB];
    const int t = threadIdx.x;
    const int k0 = k * TB, kb = min(TB, n - k0);
    const int nt = (n + TB - 1) / TB, m = nt - k - 1;
    const int b = blockIdx.x;
    const int r0 = k0 + (b + 1) * TB, rb = b < m ? min(TB, n - r0) : 0;
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, r = e % TB, c = e / TB;
        M[r][c] = (r < kb && c <= r) ? A[(k0 + r) + (int64_t)(k0 + c) * lda] : (r == c ? 1.0 : 0.0);
        if (b < m) X[r][c] = (r < rb && c < kb) ? A[(r0 + r) + (int64_t)(k0 + c) * lda] : 0.0;
    }
    __syncthreads();
    if (t < TB) Inv[t] = 1.0 / M[t][t];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int e = t + q * kDenseThreads, r = e % TB, c = e / TB;
        if (r > c) M[r][c] *= Inv[c];
    }
    __syncthreads();
    if (b < m) {
        for (int j = 0; j < kb - 1; j++) {
#pragma unroll
            for (int q = 0; q < R; q++) {
                const int e = t + q * kDenseThreads, r = e % TB, c = e / TB;
                if (c > j) X[r][c] = fma(-X[r][j], M[c][j], X[r][c]);
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int e = t + q * kDenseThreads, r = e % TB, c = e / TB;
            if (r < rb && c < kb) A[(r0 + r) + (int64_t)(k0 + c) * lda] = X[r][c] * Inv[c];
        }
        return;
    }
    // fused forward solve, one warp: z_r -= M[r][j] z_j with z unscaled (y_j l_jj), then y_r = z_r / l_rr
    if (t < 32) {
        const int r = t;
        double z = (r < kb) ? y[k0 + r] : 0.0;
        for (int j = 0; j < kb - 1; j++) {
            const double zj = __shfl_sync(0xffffffffu, z, j);
            if (r > j && r < kb) z = fma(-M[r][j], zj, z);
        }
        if (r < kb) y[k0 + r] = z * Inv[r];
    }
}

template <int TB>
__global__ void __launch_bounds__(kDenseThreads)
    k_chol_update(int n, double* __restrict__ A, int64_t lda, int k, double* __restrict__ y, int* __restrict__ info) {
    constexpr int R = TB * TB / kDenseThreads;
    constexpr int CS = kDenseThreads / TB;      // column stride between a thread's outputs
    __shared__ double Li[TB][TB + 1];
    __shared__ double Lj[TB][TB + 1];
    __shared__ double Inv[TB], Sq[TB], Sinv[TB];
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
    if (!(ii == 0 && jj == 0)) {
#pragma unroll
        for (int q = 0; q < R; q++) {
            const int c = c0 + q * CS;
            if (r < ib && c < jb && (!diag || r >= c)) A[(i0 + r) + (int64_t)(j0 + c) * lda] -= acc[q];
        }
        return;
    }
    // tile (k + 1, k + 1) has its last update: factor it here
    __syncthreads();                           // every thread is done reading Li
#pragma unroll
    for (int q = 0; q < R; q++) {
        const int c = c0 + q * CS;
        Li[r][c] = (r < ib && c <= r) ? A[(i0 + r) + (int64_t)(i0 + c) * lda] - acc[q] : (r == c ? 1.0 : 0.0);
    }
    __syncthreads();
    chol_tile<TB>(Li, ib, Inv, Sq, Sinv);
    chol_store_tile<TB>(A, lda, i0, ib, Li, Sq, Sinv, info);
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
    k_chol_diag0<TB><<<1, kDenseThreads, 0, s>>>(n, A, lda, info);
    for (int k = 0; k < nt; k++) {
        const int64_t T = nt - k - 1;
        const unsigned panel = (unsigned)(T + (y ? 1 : 0));
        if (panel) k_chol_panel<TB><<<panel, kDenseThreads, 0, s>>>(n, A, lda, k, y);
        if (T > 0)
            k_chol_update<TB><<<(unsigned)(T * (T + 1) / 2 + (y ? T : 0)), kDenseThreads, 0, s>>>(n, A, lda, k, y,
                                                                                              info);
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
