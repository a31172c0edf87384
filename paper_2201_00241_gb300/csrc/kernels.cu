// kernels.cu -- FP64 device kernels of librh (sm_103a).
//
// The hot path (Algorithm 2 of arXiv 2201.00241) is FP64-ALU-bound on GB300:
// one FP64 pipe per SM sub-partition retires one warp-wide DFMA per 64 cycles
// (about 1.2 TFLOP/s for the chip) and masked-off lanes cost the same issue
// slot.  The kernels are therefore organised to keep every lane of every
// DFMA useful:
//
//  * Directions are independent, so the direction kernel gives each CTA its
//    own slice of the N directions and runs every step of Algorithm 2 on it
//    (SpMul, both triangular sweeps, the projection, both transposed sweeps,
//    SpMulAdd) with only CTA-local barriers: no grid-wide synchronisation.
//  * Inside a CTA the work of a level is flattened over (bus, direction)
//    pairs; in narrow levels near the top of the elimination tree each row's
//    dot product is further split over adjacent lanes of a warp and summed with
//    shuffles, so that more warps issue FP64 work and a level needs one barrier.
//  * A bus is a block of one (PV) or two (PQ) variables whose rows share the
//    same columns outside the bus; one load of x_c feeds two FMAs.
//  * Right-hand sides are interleaved, row-major [row][ld]: the D directions
//    of a CTA are contiguous in each row.
#include <cstdio>
#include <mutex>

#include "../../include/rh.h"
#include "rh_kernels.h"

namespace rh {

namespace {

// Direction CTAs: 384 threads, 2 resident per SM (80 registers).  With 24 warps per
// SM either way, 2 CTAs of 384 run the full 9241-bus Hessian in 6.47 ms against
// 7.39 ms for 3 of 256: more directions per CTA put fewer buses (with different
// row lengths) in a warp and more items in every level.
constexpr int kDirThreads = 384;
constexpr int kDirCtasPerSm = 2;
constexpr int kPartCap = 4096;   // doubles of the CTA's dense-tail rows (T x directions)
constexpr int kDMax = 256;       // max directions per CTA

// Index checks of the bounds-checking build (-DRH_BOUNDS): a failed check sets a
// bit of g_bounds_err and the access is skipped (never a trap, never an early
// return that a barrier would wait for); rh_bounds_check reads the word.  In the
// normal build every check is the constant true and compiles away.
#ifdef RH_BOUNDS
__device__ unsigned int g_bounds_err;
__device__ __forceinline__ bool inb(long long i, long long n) {
    const bool ok = i >= 0 && i < n;
    if (!ok) atomicOr(&g_bounds_err, 1u);
    return ok;
}
#else
__device__ __forceinline__ constexpr bool inb(long long, long long) { return true; }
#endif

__device__ __forceinline__ unsigned long long ordered_bits(double v) {
    // |v| as a bit pattern whose unsigned order is the numeric order (NaN above inf)
    return (unsigned long long)__double_as_longlong(fabs(v));
}

// ---------------------------------------------------------------------------
// power flow: injections (eq. 2), residual (eq. 3), Jacobians
// ---------------------------------------------------------------------------

__global__ void k_injections(PfGrid g, PfState s) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_bus) return;
    double vi = s.vm[i], ai = s.va[i], p = 0.0, q = 0.0;
    for (int t = g.yp[i]; t < g.yp[i + 1]; t++) {
        int j = g.yj[t];
        double sn, cs;
        sincos(ai - s.va[j], &sn, &cs);
        p += s.vm[j] * (g.G[t] * cs + g.B[t] * sn);
        q += s.vm[j] * (g.G[t] * sn - g.B[t] * cs);
    }
    s.P[i] = vi * p;
    s.Q[i] = vi * q;
}

// One thread per bus: injections, the two residual rows of the bus and the
// Jacobian entries of those rows, scattered into the fixed LU / J_p slots.
// the four derivatives of admittance entry t into their slots of A (J_x) or J_p
__device__ __forceinline__ void jac_store(const PfGrid& g, int t, const double (&d)[4], double* A, double* jpv,
                                          unsigned long long& jm) {
    for (int u = 0; u < 4; u++) {
        const int dst = g.jac_dst[4 * t + u];
        if (dst >= 0) {
            if (!inb(dst, g.nnz_a)) continue;
            A[dst] = d[u];
            const unsigned long long b = ordered_bits(d[u]);
            jm = b > jm ? b : jm;
        } else if (dst <= -2) {
            if (!inb(-(dst + 2), g.nnz_jp)) continue;
            jpv[-(dst + 2)] = d[u];
        }
    }
}

__device__ __forceinline__ void k_pf_eval_body(PfGrid g, PfState s, double* gres, double* A, double* jpv,
                          unsigned long long* gmax, unsigned long long* jmax, int want_jac) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_bus) return;
    const double vi = s.vm[i], ai = s.va[i];
    const int rP = g.qth[i];
    const bool jac = want_jac && rP >= 0;
    double P = 0.0, Q = 0.0;
    unsigned long long jm = 0;
    int tdiag = -1;
    // one pass over the admittance row: the injection sums and, for j != i, the
    // off-diagonal Jacobian entries from the same sin/cos of theta_i - theta_j
    for (int t = g.yp[i]; t < g.yp[i + 1]; t++) {
        const int j = g.yj[t];
        double sn = 0.0, cs = 1.0;
        if (j != i) sincos(ai - s.va[j], &sn, &cs);
        else tdiag = t;
        const double vj = s.vm[j], Gij = g.G[t], Bij = g.B[t];
        P += vj * (Gij * cs + Bij * sn);
        Q += vj * (Gij * sn - Bij * cs);
        if (jac && j != i) {
            double d[4];  // dP/dtheta_j, dP/dv_j, dQ/dtheta_j, dQ/dv_j
            d[0] = vi * vj * (Gij * sn - Bij * cs);
            d[1] = vi * (Gij * cs + Bij * sn);
            d[2] = -vi * vj * (Gij * cs + Bij * sn);
            d[3] = vi * (Gij * sn - Bij * cs);
            jac_store(g, t, d, A, jpv, jm);
        }
    }
    P *= vi;
    Q *= vi;
    s.P[i] = P;
    s.Q[i] = Q;
    const int rQ = g.qv[i];
    if (rP < 0) return;  // slack: no rows
    if (gres) {
        double gp = P - s.pg[i] + s.pd[i];
        gres[rP] = gp;
        unsigned long long m = ordered_bits(gp);
        if (rQ >= 0) {
            double gq = Q + s.qd[i];
            gres[rQ] = gq;
            unsigned long long mq = ordered_bits(gq);
            m = mq > m ? mq : m;
        }
        atomicMax(gmax, m);
    }
    if (!want_jac) return;
    if (tdiag >= 0) {
        const double Gii = g.G[tdiag], Bii = g.B[tdiag];
        double d[4];
        d[0] = -Q - Bii * vi * vi;
        d[1] = P / vi + Gii * vi;
        d[2] = P - Gii * vi * vi;
        d[3] = Q / vi - Bii * vi;
        jac_store(g, tdiag, d, A, jpv, jm);
    }
    if (g.ip_pg[i] >= 0) jpv[g.pg_slot[i]] = -1.0;
    atomicMax(jmax, jm);
}
__global__ void k_pf_eval(PfGrid g, PfState s, double* gres, double* A, double* jpv,
                          unsigned long long* gmax, unsigned long long* jmax, int want_jac) { k_pf_eval_body(g, s, gres, A, jpv, gmax, jmax, want_jac); }

// Per-state preparation of the assembly: sin and cos of every bus angle (the
// assembly then forms sin and cos of each angle difference with two products), and,
// with zero, A (the slots the assembly and the refactorisation fill), the maxima and
// the pivot flag cleared.
__device__ __forceinline__ void pf_prep_body(const PfGrid& g, const PfState& s, double* A, unsigned long long* umax,
                                             int* err, int zero) {
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
    if (zero) {
        for (int64_t k = i0; k < g.nnz_a; k += stride) A[k] = 0.0;
        if (i0 == 0) {
            umax[0] = 0ull;
            umax[1] = 0ull;
            if (err) *err = 0;
        }
    }
    if (s.sc)
        for (int64_t b = i0; b < g.n_bus; b += stride) {
            double sn, cs;
            sincos(s.va[b], &sn, &cs);
            s.sc[2 * b] = sn;
            s.sc[2 * b + 1] = cs;
        }
}
__global__ void k_pf_prep(PfGrid g, PfState s, double* A, unsigned long long* umax, int* err, int zero) {
    pf_prep_body(g, s, A, umax, err, zero);
}

// The same evaluation with one admittance entry per lane: warp w takes the buses
// [pf_wb[w], pf_wb[w + 1]) (at most 32 entries together).  Each lane forms its
// entry's sin/cos, the two injection terms and, off the diagonal, its four Jacobian
// entries; after a warp barrier the lane of each bus sums its row's terms in row
// order and finishes the bus (residual, diagonal Jacobian block) as above.  The
// maxima go through one atomic per warp.  Blocks of kPfWarps warps.
constexpr int kPfWarps = 4;
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long u = __shfl_xor_sync(0xffffffffu, v, o);
        v = u > v ? u : v;
    }
    return v;
}
__device__ __forceinline__ void pf_eval_warp_body(const PfGrid& g, const PfState& s, double* gres, double* A,
                                                  double* jpv, unsigned long long* gmax, unsigned long long* jmax,
                                                  int want_jac) {
    __shared__ double sh[kPfWarps][96];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int w = blockIdx.x * kPfWarps + wl;
    if (w >= g.n_pfw) return;                                   // warp-uniform
    double* sw = sh[wl];
    const int b0 = g.pf_wb[w], b1 = g.pf_wb[w + 1];
    const int e0 = g.yp[b0], e1 = g.yp[b1];
    const int t = e0 + lane;
    unsigned long long jm = 0, gm = 0;
    double vj = 0.0, xp = 0.0, xq = 0.0;
    if (t < e1) {
        const int i = g.yrow[t], j = g.yj[t];
        double sn = 0.0, cs = 1.0;
        if (j != i) {
            if (s.sc) {            // sin / cos of theta_i - theta_j from the buses' own
                const double si = s.sc[2 * i], ci = s.sc[2 * i + 1], sj = s.sc[2 * j], cj = s.sc[2 * j + 1];
                sn = fma(si, cj, -(ci * sj));
                cs = fma(ci, cj, si * sj);
            } else {
                sincos(s.va[i] - s.va[j], &sn, &cs);
            }
        }
        vj = s.vm[j];
        const double Gij = g.G[t], Bij = g.B[t];
        xp = Gij * cs + Bij * sn;
        xq = Gij * sn - Bij * cs;
        if (want_jac && j != i && g.qth[i] >= 0) {
            const double vi = s.vm[i];
            double d[4];  // dP/dtheta_j, dP/dv_j, dQ/dtheta_j, dQ/dv_j
            d[0] = vi * vj * xq;
            d[1] = vi * xp;
            d[2] = -vi * vj * xp;
            d[3] = vi * xq;
            jac_store(g, t, d, A, jpv, jm);
        }
    }
    sw[lane] = vj;
    sw[32 + lane] = xp;
    sw[64 + lane] = xq;
    __syncwarp();
    const int i = b0 + lane;
    if (i < b1) {
        const double vi = s.vm[i];
        double P = 0.0, Q = 0.0;
        int tdiag = -1;
        for (int tt = g.yp[i]; tt < g.yp[i + 1]; tt++) {
            const int k = tt - e0;
            P += sw[k] * sw[32 + k];
            Q += sw[k] * sw[64 + k];
            if (g.yj[tt] == i) tdiag = tt;
        }
        P *= vi;
        Q *= vi;
        s.P[i] = P;
        s.Q[i] = Q;
        const int rP = g.qth[i], rQ = g.qv[i];
        if (rP >= 0) {                                          // the slack has no rows
            if (gres) {
                const double gp = P - s.pg[i] + s.pd[i];
                gres[rP] = gp;
                gm = ordered_bits(gp);
                if (rQ >= 0) {
                    const double gq = Q + s.qd[i];
                    gres[rQ] = gq;
                    const unsigned long long mq = ordered_bits(gq);
                    gm = mq > gm ? mq : gm;
                }
            }
            if (want_jac) {
                if (tdiag >= 0) {
                    const double Gii = g.G[tdiag], Bii = g.B[tdiag];
                    double d[4];
                    d[0] = -Q - Bii * vi * vi;
                    d[1] = P / vi + Gii * vi;
                    d[2] = P - Gii * vi * vi;
                    d[3] = Q / vi - Bii * vi;
                    jac_store(g, tdiag, d, A, jpv, jm);
                }
                if (g.ip_pg[i] >= 0) jpv[g.pg_slot[i]] = -1.0;
            }
        }
    }
    gm = warp_max_u64(gm);
    jm = warp_max_u64(jm);
    if (lane == 0) {
        if (gres) atomicMax(gmax, gm);
        if (want_jac) atomicMax(jmax, jm);
    }
}
__global__ void __launch_bounds__(32 * kPfWarps) k_pf_eval_warp(PfGrid g, PfState s, double* gres, double* A,
                                                                double* jpv, unsigned long long* gmax,
                                                                unsigned long long* jmax, int want_jac) {
    pf_eval_warp_body(g, s, gres, A, jpv, gmax, jmax, want_jac);
}

__device__ __forceinline__ void k_newton_update_body(PfGrid g, PfState s, const double* dx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_bus) return;
    if (g.qth[i] >= 0) s.va[i] -= dx[g.qth[i]];
    if (g.qv[i] >= 0) s.vm[i] -= dx[g.qv[i]];
}
__global__ void k_newton_update(PfGrid g, PfState s, const double* dx) { k_newton_update_body(g, s, dx); }

// ---------------------------------------------------------------------------
// coloured forward-mode Jacobian (section 4.2.2, Fig. 2)
// ---------------------------------------------------------------------------
// A dual number carries a value and CH tangent components.  Every variable of
// x and p is seeded with the unit tangent of its column colour, so the
// tangent c of a residual row is the sum of that row's derivatives over the
// columns of colour c, which the colouring makes a single entry.  Colours are
// processed CH at a time (one grid row per chunk; the values are recomputed in
// every chunk, as in chunked forward mode).

template <int CH>
struct Dual {
    double v;
    double d[CH];
};

template <int CH>
__device__ __forceinline__ Dual<CH> dual_seed(double v, int k) {
    Dual<CH> r;
    r.v = v;
#pragma unroll
    for (int m = 0; m < CH; m++) r.d[m] = (m == k) ? 1.0 : 0.0;
    return r;
}

template <int CH>
__global__ void __launch_bounds__(128) k_jac_ad(PfGrid g, PfState s, const int* __restrict__ col_th,
                                                const int* __restrict__ col_v, const int* __restrict__ col_pg,
                                                double* A, double* jpv, unsigned long long* jmax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_bus || g.qth[i] < 0) return;      // the slack has no rows
    const int c0 = blockIdx.y * CH;
    const Dual<CH> th_i = dual_seed<CH>(s.va[i], col_th[i] - c0);
    const Dual<CH> v_i = dual_seed<CH>(s.vm[i], col_v[i] - c0);
    // P_i / v_i and Q_i / v_i accumulated over the admittance row (eq. 2)
    Dual<CH> p = dual_seed<CH>(0.0, -1), q = dual_seed<CH>(0.0, -1);
    for (int t = g.yp[i]; t < g.yp[i + 1]; t++) {
        const int j = g.yj[t];
        const double G = g.G[t], B = g.B[t];
        const int kth = col_th[j] - c0, kv = col_v[j] - c0;
        double sn, cs;
        sincos(th_i.v - s.va[j], &sn, &cs);
        const double vj = s.vm[j];
        const double gc = G * cs + B * sn, gs = G * sn - B * cs;   // value parts of the two brackets
        p.v = fma(vj, gc, p.v);
        q.v = fma(vj, gs, q.v);
#pragma unroll
        for (int m = 0; m < CH; m++) {
            // d(theta_i - theta_j); d cos = -sin d(.), d sin = cos d(.)
            const double da = th_i.d[m] - (m == kth ? 1.0 : 0.0);
            const double dvj = (m == kv) ? 1.0 : 0.0;
            const double dgc = (B * cs - G * sn) * da;              // d(G cos + B sin)
            const double dgs = (G * cs + B * sn) * da;              // d(G sin - B cos)
            p.d[m] = fma(vj, dgc, fma(dvj, gc, p.d[m]));
            q.d[m] = fma(vj, dgs, fma(dvj, gs, q.d[m]));
        }
    }
    // g_P = v_i p - Pg_i + Pd_i,  g_Q = v_i q + Qd_i
    Dual<CH> gP, gQ;
    const int kpg = col_pg[i] - c0;
    gP.v = v_i.v * p.v;
    gQ.v = v_i.v * q.v;
#pragma unroll
    for (int m = 0; m < CH; m++) {
        gP.d[m] = fma(v_i.v, p.d[m], v_i.d[m] * p.v) - (m == kpg ? 1.0 : 0.0);
        gQ.d[m] = fma(v_i.v, q.d[m], v_i.d[m] * q.v);
    }
    // uncompress: each structural entry reads the tangent of its column's colour
    unsigned long long jm = 0;
    for (int t = g.yp[i]; t < g.yp[i + 1]; t++) {
        const int j = g.yj[t];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int dst = g.jac_dst[4 * t + u];
            if (dst == -1) continue;
            const int k = ((u & 1) ? col_v[j] : col_th[j]) - c0;
            if (k < 0 || k >= CH) continue;
            double val = 0.0;
#pragma unroll
            for (int m = 0; m < CH; m++)
                if (m == k) val = (u < 2) ? gP.d[m] : gQ.d[m];
            if (dst >= 0) {
                A[dst] = val;
                const unsigned long long b = ordered_bits(val);
                jm = b > jm ? b : jm;
            } else {
                jpv[-(dst + 2)] = val;
            }
        }
    }
    if (kpg >= 0 && kpg < CH) {
        double val = 0.0;
#pragma unroll
        for (int m = 0; m < CH; m++)
            if (m == kpg) val = gP.d[m];
        jpv[g.pg_slot[i]] = val;
    }
    if (jm) atomicMax(jmax, jm);
}

// ---------------------------------------------------------------------------
// fixed-pattern LU refactorisation (row-wise elimination, static pivots)
// ---------------------------------------------------------------------------

// Right-looking refactorisation, pivot steps of every sparse bus k, once all
// levels are done.  Bus block (theta, v) of a PQ bus:
//   u_tt = a_tt, l_vt = a_vt / u_tt, u_vv = a_vv - l_vt u_tv,
//   U row of v:    u_vj = a_vj - l_vt u_tj,
//   L columns:     l_jt = a_jt / u_tt,  l_jv = (a_jv - l_jt u_tv) / u_vv
// for every later variable j of the bus's pattern (a PV bus has theta only), with
// 1/u_tt, l_vt, 1/u_vv, u_tv from the bus's pivot job.  Thread x < n_piv does bus
// x's block, the others one entry j each (positions a_tj, a_vj, a_jt, a_jv).
__device__ __forceinline__ void k_rf_pivot_body(const RfGrid& g) {
    const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (x < g.n_piv) {
        const int k = (int)x;
        const int qt = g.q0[k];
        const int dt = g.diagpos[qt];
        const double tau = 1e-14 * __longlong_as_double((long long)*g.jmax);
        const double4_32a pq = g.piv[k];
        if (!(fabs(g.A[dt]) > tau)) atomicOr(g.err, 1);
        g.invdiag[qt] = pq.x;
        if (g.nv[k] == 2) {
            const int dv = g.diagpos[qt + 1];
            if (!(inb(dv, g.nnz) && inb(qt + 1, g.n_x))) return;
            const double uvv = fma(-pq.y, pq.w, g.A[dv]);
            g.A[dv - 1] = pq.y;
            g.A[dv] = uvv;
            g.invdiag[qt + 1] = pq.z;
            if (!(fabs(uvv) > tau)) atomicOr(g.err, 1);
        }
        return;
    }
    const int64_t e = x - g.n_piv;
    if (e >= g.n_pe) return;
    const int k = g.pe_bus[e];
    const int4 p = g.pe_pos[e];                     // a_tj, a_vj, a_jt, a_jv
    if (!(inb(k, g.n_piv) && inb(p.x, g.nnz) && inb(p.z, g.nnz) && (p.y < 0 || (inb(p.y, g.nnz) && inb(p.w, g.nnz)))))
        return;
    const double4_32a pq = g.piv[k];
    const double lt = g.A[p.z] * pq.x;
    g.A[p.z] = lt;
    if (p.y >= 0) {
        g.A[p.y] = fma(-pq.y, g.A[p.x], g.A[p.y]);
        g.A[p.w] = fma(-lt, pq.w, g.A[p.w]) * pq.z;
    }
}
__global__ void k_rf_pivot(RfGrid g) {
    pdl_wait();
    k_rf_pivot_body(g);
}

// Pivot quantities of a bus from its block [a_tt a_tv; a_vt a_vv]: 1/u_tt,
// l_vt = a_vt / u_tt, and 1/u_vv = a_tt / det (u_vv = det / a_tt, det = a_tt a_vv -
// a_vt a_tv), so that the two reciprocals 1/a_tt and 1/det are independent (it
// and idet given).  Stored as {1/u_tt, l_vt, 1/u_vv, u_tv}.
__device__ __forceinline__ double rf_det(double att, double atv, double avt, double avv) {
    return fma(att, avv, -(avt * atv));
}
__device__ __forceinline__ void rf_piv_store(const RfGrid& g, int j, double att, double atv, double avt, double it,
                                             double idet, bool two) {
    double lvt = 0.0, iv = 0.0, utv = 0.0;
    if (two) {
        utv = atv;
        lvt = avt * it;
        iv = att * idet;
    }
    if (inb(j, g.n_piv)) {
        double4_32a r;
        r.x = it; r.y = lvt; r.z = iv; r.w = utv;
        g.piv[j] = r;
    }
}
// Pivot jobs of the leaves (buses whose block no level updates), before the
// first level: one thread per job, the block read from A.
__device__ __forceinline__ void k_rf_leaf_piv_body(const RfGrid& g, int njob) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= njob) return;
    double v[4];
    for (int e = 0; e < 4; e++) {
        const int pp = g.piv_pos[4 * q + e];
        v[e] = (pp >= 0 && inb(pp, g.nnz)) ? g.A[pp] : 0.0;
    }
    const bool two = g.piv_pos[4 * q + 3] >= 0;
    const double it = 1.0 / v[0];
    const double idet = two ? 1.0 / rf_det(v[0], v[1], v[2], v[3]) : 0.0;
    rf_piv_store(g, g.piv_bus[q], v[0], v[1], v[2], it, idet, two);
}
__global__ void k_rf_leaf_piv(RfGrid g, int njob) {
    pdl_wait();
    k_rf_leaf_piv_body(g, njob);
}

// Update step of one level: every target entry a_ij of the level subtracts
// sum_k l_ik u_kj over the buses k of the level whose pattern holds i and j
// (fixed order: bus, then theta before v).  Bus k's pivot step has not run:
// l_it, l_iv and u_vj are formed from k's raw entries and its pivot quantities
// with the operations of the pivot step, so the factors equal those of a pivot
// step before every level, while the pivot steps of all sparse buses run once,
// in one launch, at the end.  The pivot quantities (1/u_tt, l_vt, 1/u_vv, u_tv)
// are formed once per bus by its pivot job, in the launch of the last level
// that updates k's block (the leaves' in a launch before the first level).  No
// entry a group reads is a target of the same level (its bus would depend on
// the level's own buses).
__device__ __forceinline__ double rf_group(const RfGrid& g, int2 d, int2 tu, int2 vu, double acc) {
    if (tu.x < 0) return acc;
    if (!(inb(d.x, g.n_piv) && inb(tu.x, g.nnz) && inb(tu.y, g.nnz) &&
          (d.y < 0 || (inb(vu.x, g.nnz) && inb(vu.y, g.nnz)))))
        return acc;
    const double4_32a pq = g.piv[d.x];
    const double lt = g.A[tu.x] * pq.x;
    const double ut = g.A[tu.y];
    if (d.y >= 0) {
        const double lv = fma(-lt, pq.w, g.A[vu.x]) * pq.z;
        const double uv = fma(-pq.y, ut, g.A[vu.y]);
        acc = fma(lt, ut, acc);
        return fma(lv, uv, acc);
    }
    return fma(lt, ut, acc);
}

// Targets [t0, t0 + nt) of one level; the first 4 * njob of them are the quads of
// the level's pivot jobs j0 .. j0 + njob - 1 (lane e of job q: entry e of the bus's
// block a_tt, a_tv, a_vt, a_vv, a target of this level or an empty lane).
__device__ __forceinline__ void k_rf_update_body(const RfGrid& g, int64_t t0, int64_t nt, int j0, int njob) {
    const int64_t tl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t t = t0 + (tl < nt ? tl : 0);
    double nv = 0.0;
    int p = -1;
    if (tl < nt) {
        p = g.tgt_pos[t];
        const int2 d = g.grp[3 * t], tu = g.grp[3 * t + 1], vu = g.grp[3 * t + 2];
        const int64_t x0 = g.xptr[t], x1 = g.xptr[t + 1];
        if (p >= 0 && inb(p, g.nnz)) {
            double acc = rf_group(g, d, tu, vu, 0.0);
            int64_t c = x0;
            for (; c + 1 < x1; c += 2) {
                const int2 da = g.xgrp[3 * c], tua = g.xgrp[3 * c + 1], vua = g.xgrp[3 * c + 2];
                const int2 db = g.xgrp[3 * c + 3], tub = g.xgrp[3 * c + 4], vub = g.xgrp[3 * c + 5];
                acc = rf_group(g, da, tua, vua, acc);
                acc = rf_group(g, db, tub, vub, acc);
            }
            if (c < x1) acc = rf_group(g, g.xgrp[3 * c], g.xgrp[3 * c + 1], g.xgrp[3 * c + 2], acc);
            nv = g.A[p] - acc;
            g.A[p] = nv;
        }
    }
    // pivot jobs: the quads are whole within a warp, and a warp that holds any of
    // them runs the shuffles with all its lanes
    const int64_t wbase = tl - (int64_t)(threadIdx.x & 31);
    if (wbase < 4 * (int64_t)njob) {
        const int e = (int)(tl & 3);
        const int64_t q = tl >> 2;
        const bool mine = tl < 4 * (int64_t)njob;
        double v = nv;
        int pos3 = -1;
        if (mine) {
            pos3 = g.piv_pos[4 * (j0 + q) + 3];
            if (p < 0) {
                const int pp = g.piv_pos[4 * (j0 + q) + e];
                v = (pp >= 0 && inb(pp, g.nnz)) ? g.A[pp] : 0.0;
            }
        }
        const int b = (int)(threadIdx.x & 28);
        const double att = __shfl_sync(0xffffffffu, v, b);
        const double atv = __shfl_sync(0xffffffffu, v, b + 1);
        const double avt = __shfl_sync(0xffffffffu, v, b + 2);
        const double avv = __shfl_sync(0xffffffffu, v, b + 3);
        // the two reciprocals in one division: 1/a_tt on lane 0 of the quad, 1/det on lane 3
        const double x = e == 0 ? att : (e == 3 && pos3 >= 0 ? rf_det(att, atv, avt, avv) : 1.0);
        const double r = 1.0 / x;
        const double idet = __shfl_sync(0xffffffffu, r, b + 3);
        if (mine && e == 0) rf_piv_store(g, g.piv_bus[j0 + q], att, atv, avt, r, idet, pos3 >= 0);
    }
}
__global__ void k_rf_update(RfGrid g, int64_t t0, int64_t nt, int j0, int njob) {
    pdl_wait();
    k_rf_update_body(g, t0, nt, j0, njob);
}

// Dense trailing block [t0, n_x) as a tiled right-looking LU over TB x TB tiles
// of a row-major scratch copy, spread over many SMs (GB300 runs FP64 on the
// CUDA cores at 2 lane-FMAs per clock per SM, so one CTA would need T^3 / 3
// FMAs on a single SM).  Static diagonal pivots, unit lower L.  One launch per
// tile column: launch k (k = -1 .. nt - 1) factors column c = k + 1 and holds
//   panel CTAs     one per tile (i, c) and (c, i), i > c: the tile and the
//                  diagonal tile take their last update (column k), the
//                  diagonal tile is factored, and L_ic = A_ic U_cc^{-1} or
//                  U_ci = L_cc^{-1} A_ci is stored
//   a diagonal CTA that factors tile (k, k) once more and stores its L and U:
//                  the panel CTAs of launch k - 1 read that tile, so it is only
//                  overwritten one launch later
//   trailing CTAs  A_ij -= L_ik U_kj for every tile i, j > c.
// Every CTA that needs the factored diagonal tile factors it itself from the
// same inputs with the same code, so all copies agree bit for bit; no launch
// reads a tile that another of its CTAs writes.  The diagonal tile is
// eliminated without divisions (cross-multiplied steps with an exact
// power-of-two rescale): the trailing block after step j is s_{j+1} times the
// ordinary one, so u_rc = a_rc / s_r (r <= c), l_rc = a_rc / a_cc (r > c) and
// 1 / u_cc = s_c / a_cc, with one division per column for 1 / a_cc.
constexpr int kTailTB = 16;

__device__ __forceinline__ void k_tail_gather_body(RfGrid g) {
    const int T = g.T;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= T * T) return;
    const int p = g.tail_pos[idx];
    g.tailD[idx] = (p >= 0 && inb(p, g.nnz)) ? g.A[p] : 0.0;
}
__global__ void k_tail_gather(RfGrid g) {
    pdl_wait();
    k_tail_gather_body(g);
}

// Entry p of a TB x TB tile in shells of decreasing min(r, c) (p = 0 is the
// last diagonal entry): the entries with r, c > j are exactly p < (TB-1-j)^2.
__device__ __forceinline__ void tail_shell_entry(int p, int& r, int& c) {
    constexpr int TB = kTailTB;
    int q = 0;
    while ((q + 1) * (q + 1) <= p) q++;
    const int m = TB - 1 - q, o = p - q * q;
    r = o <= q ? m : m + (o - q);
    c = o == 0 ? m : (o <= q ? m + o : m);
}

// Eliminates the tile in Dk (unit-padded beyond kb) without divisions:
// afterwards Dk[r][c] = s_{min(r,c)} a_rc (a the ordinary elimination's values
// when the entry is final), S[c] = s_c and Rd[c] = 1 / Dk[c][c].
__device__ __forceinline__ void tail_factor(double (*Dk)[kTailTB + 1], int kb, double* S, double* Rd) {
    constexpr int TB = kTailTB;
    const int t = threadIdx.x;
    int er = 0, ec = 0;
    tail_shell_entry(min(t, (TB - 1) * (TB - 1) - 1), er, ec);
    double s = 1.0;
    for (int j = 0; j < kb - 1; j++) {
        const int na = (TB - 1 - j) * (TB - 1 - j);
        const double d = Dk[j][j];
        const int sh = pivot_shift(d);
        if (t < na) {
            const double prod = Dk[er][j] * Dk[j][ec];
            Dk[er][ec] = scale_pow2(fma(d, Dk[er][ec], -prod), sh);
        }
        if (t == (int)blockDim.x - 1) {
            s *= scale_pow2(d, sh);
            S[j + 1] = s;
        }
        __syncthreads();
    }
    if (t < TB) {
        if (t < kb) {
            if (t == 0) S[0] = 1.0;
            Rd[t] = 1.0 / Dk[t][t];
        } else {
            S[t] = 0.0;
            Rd[t] = 0.0;
        }
    }
    __syncthreads();
}

// Loads a TB x TB tile of the row-major T x T scratch at (i0, j0), rb x cb live.
__device__ __forceinline__ void tail_load(double (*X)[kTailTB + 1], const double* D, int T, int i0, int j0, int rb,
                                          int cb) {
    const int r = threadIdx.x / kTailTB, c = threadIdx.x % kTailTB;   // lanes along a row (coalesced)
    X[r][c] = (r < rb && c < cb) ? D[(size_t)(i0 + r) * T + j0 + c] : 0.0;
}

// The diagonal tile of column c0 / TB with its last update (column kk0 / TB,
// if kk0 >= 0): Dk = A_cc - L_ck U_kc, unit-padded beyond kb.  Uses Lk and Uk.
__device__ __forceinline__ void tail_diag_tile(const RfGrid& g, int c0, int kb, int kk0, double (*Dk)[kTailTB + 1],
                                               double (*Lk)[kTailTB + 1], double (*Uk)[kTailTB + 1]) {
    constexpr int TB = kTailTB;
    const int T = g.T, t = threadIdx.x, r = t / TB, c = t % TB;
    const double* D = g.tailD;
    const double a = (r < kb && c < kb) ? D[(size_t)(c0 + r) * T + c0 + c] : (r == c ? 1.0 : 0.0);
    if (kk0 >= 0) {
        tail_load(Lk, D, T, c0, kk0, kb, TB);
        tail_load(Uk, D, T, kk0, c0, TB, kb);
    }
    __syncthreads();
    double acc = 0.0;
    if (kk0 >= 0) {
#pragma unroll
        for (int q = 0; q < TB; q++) acc = fma(Lk[r][q], Uk[q][c], acc);
    }
    Dk[r][c] = a - acc;
    __syncthreads();
}

__device__ __forceinline__ void k_tail_step_body(RfGrid g, int k) {
    constexpr int TB = kTailTB;
    __shared__ double Dk[TB][TB + 1];
    __shared__ double X[TB][TB + 1];
    __shared__ double Lk[TB][TB + 1];
    __shared__ double Uk[TB][TB + 1];
    __shared__ double Xk[TB][TB + 1];
    __shared__ double S[TB], Rd[TB];
    const int T = g.T, nt = (T + TB - 1) / TB;
    const int t = threadIdx.x;
    const int c = k + 1, c0 = c * TB, k0 = k * TB;
    const int U = c < nt ? nt - c - 1 : 0;
    double* D = g.tailD;
    int b = (int)blockIdx.x;
    if (b < 2 * U) {
        // panel CTA: tile (i, c) (L) for b < U, tile (c, i) (U) otherwise
        const bool ltile = b < U;
        const int o0 = c0 + ((ltile ? b : b - U) + 1) * TB, ob = min(TB, T - o0);
        const int kb = min(TB, T - c0);
        // own tile and its last update: A_ic - L_ik U_kc, or A_ci - L_ck U_ki
        if (ltile) {
            tail_load(X, D, T, o0, c0, ob, kb);
            if (k >= 0) tail_load(Xk, D, T, o0, k0, ob, TB);   // L_ik
        } else {
            tail_load(X, D, T, c0, o0, kb, ob);
            if (k >= 0) tail_load(Xk, D, T, k0, o0, TB, ob);   // U_ki
        }
        tail_diag_tile(g, c0, kb, k >= 0 ? k0 : -1, Dk, Lk, Uk);   // its barriers also cover X, Xk
        if (k >= 0) {
            const int r = t / TB, cc = t % TB;
            double acc = 0.0;
#pragma unroll
            for (int q = 0; q < TB; q++)
                acc = ltile ? fma(Xk[r][q], Uk[q][cc], acc) : fma(Lk[r][q], Xk[q][cc], acc);
            X[r][cc] -= acc;
        }
        tail_factor(Dk, kb, S, Rd);   // begins by reading only Dk; its barriers cover X
        // multipliers in place: u_jc / u_jj = Dk[j][c] Rd[j] above the diagonal,
        // l_rj = Dk[r][j] Rd[j] below it
        {
            const int r = t / TB, cc = t % TB;
            if (r != cc) Dk[r][cc] *= Rd[min(r, cc)];
            __syncthreads();
        }
        if (ltile) {
            // X U_cc = A_ic, unscaled (x_rj u_jj), with the multipliers u_jc / u_jj;
            // the rows are independent, each in TB lanes (one per column)
            const int r = t / TB, cl = t % TB;
            double x = X[r][cl];
#pragma unroll
            for (int j = 0; j < TB - 1; j++) {
                if (j < kb - 1) {
                    const double xj = __shfl_sync(0xffffffffu, x, j, TB);
                    if (cl > j) x = fma(-xj, Dk[j][cl], x);
                }
            }
            // 1 / u_cc = s_c / Dk[c][c]
            if (r < ob && cl < kb) D[(size_t)(o0 + r) * T + c0 + cl] = x * (S[cl] * Rd[cl]);
        } else {
            // L_cc Y = A_ci with unit L; the columns are independent, each in TB
            // lanes (one per row)
            const int col = t / TB, r = t % TB;
            double y = X[r][col];
#pragma unroll
            for (int j = 0; j < TB - 1; j++) {
                if (j < kb - 1) {
                    const double yj = __shfl_sync(0xffffffffu, y, j, TB);
                    if (r > j) y = fma(-Dk[r][j], yj, y);
                }
            }
            if (r < kb && col < ob) D[(size_t)(c0 + r) * T + o0 + col] = y;
        }
        return;
    }
    b -= 2 * U;
    if (k >= 0 && b == 0) {
        // diagonal CTA: factor tile (k, k) with its last update (column k - 1) and store
        // U (r <= c: Dk / s_r) and L (r > c: Dk / Dk[c][c])
        const int kb = min(TB, T - k0);
        tail_diag_tile(g, k0, kb, k >= 1 ? k0 - TB : -1, Dk, Lk, Uk);
        tail_factor(Dk, kb, S, Rd);
        const int r = t / TB, cl = t % TB;
        if (t < TB) Xk[0][t] = t < kb ? 1.0 / S[t] : 0.0;
        __syncthreads();
        if (r < kb && cl < kb) D[(size_t)(k0 + r) * T + k0 + cl] = r > cl ? Dk[r][cl] * Rd[cl] : Dk[r][cl] * Xk[0][r];
        return;
    }
    if (k >= 0) b -= 1;
    if (k < 0 || b >= U * U) return;
    // trailing tile (i, j), i, j > c: A_ij -= L_ik U_kj
    const int bi = b / U, bj = b % U;
    const int i0 = c0 + (bi + 1) * TB, j0 = c0 + (bj + 1) * TB;
    const int ib = min(TB, T - i0), jb = min(TB, T - j0);
    const int r = t / TB, cc = t % TB;
    const double a = (r < ib && cc < jb) ? D[(size_t)(i0 + r) * T + j0 + cc] : 0.0;
    tail_load(Lk, D, T, i0, k0, ib, TB);
    tail_load(Uk, D, T, k0, j0, TB, jb);
    __syncthreads();
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < TB; q++) acc = fma(Lk[r][q], Uk[q][cc], acc);
    if (r < ib && cc < jb) D[(size_t)(i0 + r) * T + j0 + cc] = a - acc;
}
__global__ void __launch_bounds__(256) k_tail_step(RfGrid g, int k) {
    pdl_wait();
    k_tail_step_body(g, k);
}

__device__ __forceinline__ void k_tail_scatter_body(RfGrid g) {
    const int T = g.T;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= T * T) return;
    const int p = g.tail_pos[idx];
    const double v = g.tailD[idx];
    if (p >= 0 && inb(p, g.nnz)) g.A[p] = v;
    const int i = idx / T, j = idx - i * T;
    if (i == j) {
        g.invdiag[g.t0 + i] = 1.0 / v;
        const double tau = 1e-14 * __longlong_as_double((long long)*g.jmax);
        if (!(fabs(v) > tau)) atomicOr(g.err, 1);
    }
}
__global__ void k_tail_scatter(RfGrid g) {
    pdl_wait();
    k_tail_scatter_body(g);
}

// Transposed copies of the factor values and of J_p, and the unit-diagonal
// factors of the direction kernel.  With D = diag(U), J_x = L U = D L'' U' where
// L'' = D^-1 L D and U' = D^-1 U are both unit triangular:
//   l''_qc = l_qc u_cc / u_qq (c < q),   u'_qc = u_qc / u_qq (c > q).
// J_x z = b is then L'' y = D^-1 b, U' z = y, and J_x^T psi = r is U'^T u = r,
// L''^T w = u, psi = D^-1 w: no sweep multiplies by a pivot, and D^-1 folds into
// the rows of J_p (SpMul's right-hand sides, SpMulAdd's J_p^T psi).  One thread
// per position of A (row arow[i], column col[i]) and per entry of J_p.
__device__ __forceinline__ double unit_scale(const double* A, const int* diagpos, const double* invdiag, int r,
                                             int c) {
    return c < r ? A[diagpos[c]] * invdiag[r] : (c > r ? invdiag[r] : 0.0);
}
__global__ void k_transpose_values(int nnz, const int* __restrict__ tpos, const int* __restrict__ arow,
                                   const int* __restrict__ col, const int* __restrict__ diagpos,
                                   const double* __restrict__ A, const double* __restrict__ invdiag,
                                   double* __restrict__ At, double* __restrict__ Ad, double* __restrict__ Atd,
                                   int nnz_jp, const int* __restrict__ jpt_src, const int* __restrict__ jpt_row,
                                   const double* __restrict__ jpv, double* __restrict__ jptv,
                                   double* __restrict__ jptvd) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nnz) {
        const int r = arow[i], c = col[i];
        const double at = A[tpos[i]];
        At[i] = at;
        Ad[i] = r == c ? 1.0 : A[i] * unit_scale(A, diagpos, invdiag, r, c);
        Atd[i] = r == c ? 1.0 : at * unit_scale(A, diagpos, invdiag, c, r);
    }
    if (i < nnz_jp) {
        const double v = jpv[jpt_src[i]];
        jptv[i] = v;
        jptvd[i] = v * invdiag[jpt_row[i]];
    }
}

// The four packed triangles of the dense tail for the sweeps, one thread per
// (i, j) of the T x T block; pos maps (i, j) to A (-1: structurally zero).
// x[r] *= s[r] for the first n rows of an n x N row-major block (leading dimension ld)
__global__ void k_scale_rows(int n, int N, const double* __restrict__ s, double* x, int64_t ld) {
    const int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= (int64_t)n * N) return;
    const int r = (int)(it / N), c = (int)(it - (int64_t)r * N);
    x[(int64_t)r * ld + c] *= s[r];
}

// The dense tail's triangles: for the single solves (columns of U scaled by
// 1/u_jj), and of the unit-diagonal factors L'', U' for the direction kernel.
__device__ __forceinline__ void k_build_tail_body(int T, int t0, const int* __restrict__ pos, const double* __restrict__ A,
                             const double* __restrict__ invdiag, double* triL, double* triU, double* triUt,
                             double* triLt, double* triLd, double* triUd, double* triUtd, double* triLtd) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= T * T) return;
    int i = idx / T, j = idx - i * T;
    if (i == j) return;
    int pij = pos[idx], pji = pos[j * T + i];
    double aij = pij >= 0 ? A[pij] : 0.0, aji = pji >= 0 ? A[pji] : 0.0;
    const double ii = invdiag[t0 + i], ij = invdiag[t0 + j];
    if (i > j) {
        int o = j * (T - 1) - j * (j - 1) / 2 + (i - j - 1);
        triL[o] = aij;                              // L_ij
        triUt[o] = aji * ij;                        // (U^T)_ij = U_ji, scaled by 1/u_jj
        triLd[o] = aij * A[pos[j * T + j]] * ii;    // L''_ij
        triUtd[o] = aji * ij;                       // (U'^T)_ij = U'_ji
    } else {
        int o = j * (j - 1) / 2 + i;
        triU[o] = aij * ij;                         // U_ij scaled by 1/u_jj
        triLt[o] = aji;                             // (L^T)_ij = L_ji
        triUd[o] = aij * ii;                        // U'_ij
        triLtd[o] = aji * A[pos[i * T + i]] * ij;   // (L''^T)_ij = L''_ji
    }
}
__global__ void k_build_tail(int T, int t0, const int* __restrict__ pos, const double* __restrict__ A,
                             const double* __restrict__ invdiag, double* triL, double* triU, double* triUt,
                             double* triLt, double* triLd, double* triUd, double* triUtd, double* triLtd) { k_build_tail_body(T, t0, pos, A, invdiag, triL, triU, triUt, triLt, triLd, triUd, triUtd, triLtd); }

// ---------------------------------------------------------------------------
// the direction kernel: Algorithm 2 for a slice of directions per CTA
// ---------------------------------------------------------------------------

// Narrow levels (fewer than blockDim / 2 (bus, direction) items): every row's dot
// product is split over ks adjacent lanes of a warp, ks a power of two up to the
// cap (at most 32) and at most half the row, as long as the items still fit in the
// CTA's threads.  1: no split.
__device__ __forceinline__ int split_lanes(int nb, int D, int maxext, int cap) {
    const int base = nb * D;
    if (2 * base > (int)blockDim.x) return 1;
    int ks = 1;
    while (2 * ks <= cap && 2 * base * ks <= (int)blockDim.x && 2 * ks <= maxext) ks *= 2;
    return ks;
}

// a0 -= sum_e v0[e] x[col[e]], a1 -= sum_e v1[e] x[col[e]] over e in [e0, e1) of
// one bus block (two rows sharing their columns when TWO).  Unrolled by 4 so
// that each lane has four independent loads in flight, with one FMA chain per
// row: the FP64 pipe takes one warp instruction per 64 cycles per sub-partition,
// far longer than the chain's latency, so a second accumulator would only cost
// an extra FP64 add.
//
// TWO is chosen per warp (any lane with a second row): a predicated FP64
// instruction occupies the pipe even with its lanes off, so warps of
// single-row buses must not issue the second row at all.  In a mixed warp the
// single-row lanes run the second row on a copy of their first (r1 == r0) and
// ignore the result.
// CMASK: x of a row whose bit in cmask is clear is zero and is not read.
__device__ __forceinline__ bool mask_get(const unsigned* m, int q) { return (m[q >> 5] >> (q & 31)) & 1u; }
template <bool CMASK>
__device__ __forceinline__ double ldx(const double* X, int i, int64_t ld, int64_t c, const unsigned* cmask,
                                      int nrows) {
    return (inb(i, nrows) && (!CMASK || mask_get(cmask, i))) ? X[(int64_t)i * ld + c] : 0.0;
}
// n, or 0 when a row part [r0, r0 + n) or [r1, r1 + n) would leave the nnz
// positions of the pattern (bounds build only; the item is then left as it is)
__device__ __forceinline__ int part_len(int n, int r0, int r1, int nnz) {
    return (inb(r0, nnz + 1) && inb(r0 + n, nnz + 1) && inb(r1, nnz + 1) && inb(r1 + n, nnz + 1)) ? n : 0;
}
// X[q][c] = v for a row q that must lie below nrows (checked in the bounds build)
__device__ __forceinline__ void stx(double* X, int q, int64_t ld, int64_t c, double v, int nrows) {
    if (inb(q, nrows)) X[(int64_t)q * ld + c] = v;
}
template <bool TWO, bool CMASK = false>
__device__ __forceinline__ void block_sub(const int* __restrict__ col, const double* __restrict__ vals, int r0, int r1,
                                          int e0, int e1, const double* X, int64_t ld, int64_t c, double& a0,
                                          double& a1, const unsigned* cmask = nullptr, int nrows = 0x7fffffff) {
    int e = e0;
    for (; e + 4 <= e1; e += 4) {
        const int i0 = col[r0 + e], i1 = col[r0 + e + 1], i2 = col[r0 + e + 2], i3 = col[r0 + e + 3];
        const double x0 = ldx<CMASK>(X, i0, ld, c, cmask, nrows), x1 = ldx<CMASK>(X, i1, ld, c, cmask, nrows);
        const double x2 = ldx<CMASK>(X, i2, ld, c, cmask, nrows), x3 = ldx<CMASK>(X, i3, ld, c, cmask, nrows);
        a0 = fma(-vals[r0 + e], x0, a0);
        a0 = fma(-vals[r0 + e + 1], x1, a0);
        a0 = fma(-vals[r0 + e + 2], x2, a0);
        a0 = fma(-vals[r0 + e + 3], x3, a0);
        if constexpr (TWO) {
            a1 = fma(-vals[r1 + e], x0, a1);
            a1 = fma(-vals[r1 + e + 1], x1, a1);
            a1 = fma(-vals[r1 + e + 2], x2, a1);
            a1 = fma(-vals[r1 + e + 3], x3, a1);
        }
    }
    for (; e < e1; e++) {
        const double xv = ldx<CMASK>(X, col[r0 + e], ld, c, cmask, nrows);
        a0 = fma(-vals[r0 + e], xv, a0);
        if constexpr (TWO) a1 = fma(-vals[r1 + e], xv, a1);
    }
}

// a0 -= sum v0[e] x[col[e]], a1 likewise, over e = e0, e0 + step, ... < n: the share of
// one lane of a split row (adjacent lanes read adjacent entries)
template <bool TWO, bool CMASK>
__device__ __forceinline__ void strided_sub(const int* __restrict__ col, const double* __restrict__ vals, int r0,
                                            int r1, int e, int n, int step, const double* X, int64_t ld, int64_t c,
                                            double& a0, double& a1, const unsigned* cmask, int nrows) {
    for (; e + step < n; e += 2 * step) {
        const int i0 = col[r0 + e], i1 = col[r0 + e + step];
        const double x0 = ldx<CMASK>(X, i0, ld, c, cmask, nrows), x1 = ldx<CMASK>(X, i1, ld, c, cmask, nrows);
        a0 = fma(-vals[r0 + e], x0, a0);
        a0 = fma(-vals[r0 + e + step], x1, a0);
        if constexpr (TWO) {
            a1 = fma(-vals[r1 + e], x0, a1);
            a1 = fma(-vals[r1 + e + step], x1, a1);
        }
    }
    if (e < n) {
        const double xv = ldx<CMASK>(X, col[r0 + e], ld, c, cmask, nrows);
        a0 = fma(-vals[r0 + e], xv, a0);
        if constexpr (TWO) a1 = fma(-vals[r1 + e], xv, a1);
    }
}

// sum of a lane's partial sums over the ks adjacent lanes of its item (all 32 lanes of
// the warp take part; ks divides 32)
__device__ __forceinline__ void split_sum(int ks, bool wtwo, double& s0, double& s1) {
    for (int off = ks >> 1; off > 0; off >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, off, ks);
        if (wtwo) s1 += __shfl_down_sync(0xffffffffu, s1, off, ks);
    }
}

// warp-uniform choice of the two-row path (lanes that left the item loop do not vote)
__device__ __forceinline__ bool warp_any(bool p) { return __any_sync(__activemask(), p); }

// forward sweep over the L pattern: x_q = (b_q - sum_{c<q} v_qc x_c) [* 1/u_qq]
template <bool SCALE, bool TWO>
__device__ __forceinline__ void fwd_finish(const DirGrid& g, const double* __restrict__ vals, double* X, int64_t ld,
                                           int64_t c, int q, bool two, int pos_vt, double a0, double a1) {
    double x0 = SCALE ? a0 * g.invdiag[q] : a0;
    stx(X, q, ld, c, x0, g.n_x);
    if constexpr (TWO) {
        a1 = fma(-vals[pos_vt], x0, a1);
        const double i1 = (SCALE && two) ? g.invdiag[q + 1] : 1.0;
        const double x1 = SCALE ? a1 * i1 : a1;
        if (two) stx(X, q + 1, ld, c, x1, g.n_x);
    }
}

// One level of a sweep is flattened over (bus, direction) items, or, when the
// level is too narrow to give every warp work, over (bus, direction, lane of the
// row) with the row's lanes adjacent in a warp.  Each bus block is described by one packed slot
//   forward:  {q, n, rp, rpv}  theta row q, n columns left of the bus, L parts of
//             the theta row at rp and of the v row at rpv (-1 for a PV bus)
//   backward: {q, n, ue0, ue1} U parts right of the bus at ue0 / ue1 (-1: PV)
// so an item needs a single dependent load before its row data; the next
// item's slot is prefetched while the current one is computed.
// EXT: subtract the row parts only (the dense tail's external phase), no finish.
// mask (optional, forward L sweep with identity W): bit q is set for the theta row q of
// every bus whose x can be nonzero for this CTA's directions; every processed bus
// activates its tree parent, an inactive bus only stores its zeros.  seed: the buses
// whose right-hand side was written (zeroed, then the J_p entries scattered); every
// other active bus has b = 0, so V need not be zeroed beforehand.
__device__ __forceinline__ void mask_set(unsigned* m, int q) { atomicOr(m + (q >> 5), 1u << (q & 31)); }
// activate a bus given its encoded theta row (theta row * 2 + 1 if it has a v row)
__device__ __forceinline__ void mask_bus(unsigned* m, int enc) {
    if (enc < 0) return;
    mask_set(m, enc >> 1);
    if (enc & 1) mask_set(m, (enc >> 1) + 1);
}
template <bool SCALE, bool EXT = false, bool CMASK = false>
__device__ void sweep_fwd(const DirGrid& g, const LevelSet& ls, const double* __restrict__ vals, double* X,
                          int64_t ld, int c0, int D, double* part, unsigned* mask = nullptr,
                          const unsigned* seed = nullptr, const unsigned* cmask = nullptr) {
    for (int lev = 0; lev < ls.n_lev; lev++) {
        const int b0 = ls.ptr[lev], nb = ls.ptr[lev + 1] - b0;
        const int4* __restrict__ slots = ls.slots + b0;
        const int ks = split_lanes(nb, D, ls.maxext[lev], g.ks_cap);
        if (ks == 1) {
            const int items = nb * D;
            int it = threadIdx.x;
            int bi = it / D;
            int4 nxt = it < items ? slots[bi] : make_int4(0, 0, 0, -1);
            for (; it < items; it += blockDim.x) {
                const int4 sl = nxt;
                const int d = it - bi * D;
                const int it2 = it + blockDim.x, bi2 = it2 / D;
                if (it2 < items) nxt = slots[bi2];
                const int q = sl.x, rp = sl.z;
                bi = bi2;
                const bool two = sl.w >= 0;
                const int64_t c = c0 + d;
                if (mask && !(inb(q, g.n_x) && mask_get(mask, q))) continue;   // outside the reach: x = 0, never read
                const int rpv = two ? sl.w : rp;
                const int n = part_len(sl.y, rp, rpv, g.nnz);
                const bool has_b = !seed || mask_get(seed, q);
                double a0 = (has_b && inb(q, g.n_x)) ? X[(int64_t)q * ld + c] : 0.0;
                double a1 = (two && has_b && inb(q + 1, g.n_x)) ? X[(int64_t)(q + 1) * ld + c] : 0.0;
                if (warp_any(two)) {
                    block_sub<true, CMASK>(g.col, vals, rp, rpv, 0, n, X, ld, c, a0, a1, cmask, g.n_x);
                    if (EXT) {
                        stx(X, q, ld, c, a0, g.n_x);
                        if (two) stx(X, q + 1, ld, c, a1, g.n_x);
                    } else {
                        fwd_finish<SCALE, true>(g, vals, X, ld, c, q, two, rpv + n, a0, a1);
                    }
                } else {
                    block_sub<false, CMASK>(g.col, vals, rp, rpv, 0, n, X, ld, c, a0, a1, cmask, g.n_x);
                    if (EXT) stx(X, q, ld, c, a0, g.n_x);
                    else fwd_finish<SCALE, false>(g, vals, X, ld, c, q, two, rpv + n, a0, a1);
                }
                if (mask) mask_bus(mask, g.bparent[q]);
            }
        } else {
            // narrow level: each row split over ks adjacent lanes, summed by shuffles
            const int total = nb * D * ks;
            const int lane = (int)(threadIdx.x & 31);
            for (int w0 = (int)threadIdx.x - lane; w0 < total; w0 += blockDim.x) {     // warp-uniform
                const int it = w0 + lane, sli = it & (ks - 1), item = it / ks;
                const bool valid = it < total;
                const int bi = valid ? item / D : 0, d = valid ? item - bi * D : 0;
                const int4 sl = valid ? slots[bi] : make_int4(0, 0, 0, -1);
                const int q = sl.x, rp = sl.z;
                const bool two = sl.w >= 0;
                const int rpv = two ? sl.w : rp;
                const bool act = valid && !(mask && !(inb(q, g.n_x) && mask_get(mask, q)));
                const int n = act ? part_len(sl.y, rp, rpv, g.nnz) : 0;
                const int64_t c = c0 + d;
                const bool fin = act && sli == 0;          // the lane that finishes the item
                const bool has_b = fin && (!seed || mask_get(seed, q));
                const double b0 = (has_b && inb(q, g.n_x)) ? X[(int64_t)q * ld + c] : 0.0;
                const double b1 = (two && has_b && inb(q + 1, g.n_x)) ? X[(int64_t)(q + 1) * ld + c] : 0.0;
                const bool wtwo = __any_sync(0xffffffffu, two);   // every lane of the warp is here
                double s0 = 0.0, s1 = 0.0;
                if (wtwo) strided_sub<true, CMASK>(g.col, vals, rp, rpv, sli, n, ks, X, ld, c, s0, s1, cmask, g.n_x);
                else strided_sub<false, CMASK>(g.col, vals, rp, rpv, sli, n, ks, X, ld, c, s0, s1, cmask, g.n_x);
                split_sum(ks, wtwo, s0, s1);
                if (!fin) continue;
                const double a0 = b0 + s0, a1 = b1 + s1;
                if (EXT) {
                    stx(X, q, ld, c, a0, g.n_x);
                    if (two) stx(X, q + 1, ld, c, a1, g.n_x);
                } else if (two) {
                    fwd_finish<SCALE, true>(g, vals, X, ld, c, q, two, rpv + n, a0, a1);
                } else {
                    fwd_finish<SCALE, false>(g, vals, X, ld, c, q, two, rpv + n, a0, a1);
                }
                if (mask) mask_bus(mask, g.bparent[q]);
            }
        }
        __syncthreads();
    }
}

// backward sweep over the U pattern: x_q = (b_q - sum_{c>q} v_qc x_c) [* 1/u_qq]
template <bool SCALE, bool TWO>
__device__ __forceinline__ void bwd_finish(const DirGrid& g, const double* __restrict__ vals, double* X, int64_t ld,
                                           int64_t c, int q, bool two, int pos_tv, double a0, double a1) {
    if constexpr (TWO) {
        const double i1 = (SCALE && two) ? g.invdiag[q + 1] : 1.0;
        const double x1 = SCALE ? a1 * i1 : a1;
        if (two) stx(X, q + 1, ld, c, x1, g.n_x);
        a0 = fma(-vals[pos_tv], two ? x1 : 0.0, a0);
    }
    stx(X, q, ld, c, SCALE ? a0 * g.invdiag[q] : a0, g.n_x);
}

// rmask (optional): right-hand side rows whose bit is clear are zero and are not read
template <bool SCALE>
__device__ void sweep_bwd(const DirGrid& g, const LevelSet& ls, const double* __restrict__ vals, double* X,
                          int64_t ld, int c0, int D, double* part, const unsigned* rmask = nullptr) {
    for (int lev = 0; lev < ls.n_lev; lev++) {
        const int b0 = ls.ptr[lev], nb = ls.ptr[lev + 1] - b0;
        const int4* __restrict__ slots = ls.slots + b0;
        const int ks = split_lanes(nb, D, ls.maxext[lev], g.ks_cap);
        if (ks == 1) {
            const int items = nb * D;
            int it = threadIdx.x;
            int bi = it / D;
            int4 nxt = it < items ? slots[bi] : make_int4(0, 0, 0, -1);
            for (; it < items; it += blockDim.x) {
                const int4 sl = nxt;
                const int d = it - bi * D;
                const int it2 = it + blockDim.x, bi2 = it2 / D;
                if (it2 < items) nxt = slots[bi2];
                const int q = sl.x, ue0 = sl.z;
                const bool two = sl.w >= 0;
                const int ue1 = two ? sl.w : ue0;
                const int n = part_len(sl.y, ue0 - 1, ue1, g.nnz);
                const int64_t c = c0 + d;
                const bool has_b = !rmask || mask_get(rmask, q);
                double a0 = (has_b && inb(q, g.n_x)) ? X[(int64_t)q * ld + c] : 0.0;
                double a1 = (two && has_b && inb(q + 1, g.n_x)) ? X[(int64_t)(q + 1) * ld + c] : 0.0;
                if (warp_any(two)) {
                    block_sub<true>(g.col, vals, ue0, ue1, 0, n, X, ld, c, a0, a1, nullptr, g.n_x);
                    bwd_finish<SCALE, true>(g, vals, X, ld, c, q, two, ue0 - 1, a0, a1);
                } else {
                    block_sub<false>(g.col, vals, ue0, ue1, 0, n, X, ld, c, a0, a1, nullptr, g.n_x);
                    bwd_finish<SCALE, false>(g, vals, X, ld, c, q, two, ue0 - 1, a0, a1);
                }
                bi = bi2;
            }
        } else {
            // narrow level: each row split over ks adjacent lanes, summed by shuffles
            const int total = nb * D * ks;
            const int lane = (int)(threadIdx.x & 31);
            for (int w0 = (int)threadIdx.x - lane; w0 < total; w0 += blockDim.x) {     // warp-uniform
                const int it = w0 + lane, sli = it & (ks - 1), item = it / ks;
                const bool valid = it < total;
                const int bi = valid ? item / D : 0, d = valid ? item - bi * D : 0;
                const int4 sl = valid ? slots[bi] : make_int4(0, 0, 0, -1);
                const int q = sl.x, ue0 = sl.z;
                const bool two = sl.w >= 0;
                const int ue1 = two ? sl.w : ue0;
                const int n = valid ? part_len(sl.y, ue0 - 1, ue1, g.nnz) : 0;
                const int64_t c = c0 + d;
                const bool fin = valid && sli == 0;
                const bool has_b = fin && (!rmask || mask_get(rmask, q));
                const double b0 = (has_b && inb(q, g.n_x)) ? X[(int64_t)q * ld + c] : 0.0;
                const double b1 = (two && has_b && inb(q + 1, g.n_x)) ? X[(int64_t)(q + 1) * ld + c] : 0.0;
                const bool wtwo = __any_sync(0xffffffffu, two);   // every lane of the warp is here
                double s0 = 0.0, s1 = 0.0;
                if (wtwo) strided_sub<true, false>(g.col, vals, ue0, ue1, sli, n, ks, X, ld, c, s0, s1, nullptr, g.n_x);
                else strided_sub<false, false>(g.col, vals, ue0, ue1, sli, n, ks, X, ld, c, s0, s1, nullptr, g.n_x);
                split_sum(ks, wtwo, s0, s1);
                if (!fin) continue;
                if (two) bwd_finish<SCALE, true>(g, vals, X, ld, c, q, two, ue0 - 1, b0 + s0, b1 + s1);
                else bwd_finish<SCALE, false>(g, vals, X, ld, c, q, two, ue0 - 1, b0 + s0, b1 + s1);
            }
        }
        __syncthreads();
    }
}

// Dense trailing block [t0, t0 + T) of a sweep, column-oriented in shared memory.
// xt[i * D + d] holds row t0 + i of the CTA's directions; tri_g is the packed
// strictly-triangular block (column j contiguous), columns pre-scaled by 1/u_jj
// for the scaled sweeps, so each column step is y_i -= tri_ij y_j and the
// result is x_i = y_i [* 1/u_ii].  One barrier per column.  With tri != NULL the
// triangle is first staged in shared memory (one CTA per SM); with tri == NULL
// it is read through L1, where it is shared by all the CTAs of the SM.
__device__ __forceinline__ int lpack_off(int j, int T) { return j * (T - 1) - j * (j - 1) / 2; }  // rows j+1..T-1
__device__ __forceinline__ int upack_off(int j) { return j * (j - 1) / 2; }                      // rows 0..j-1

// The solve runs over blocks of kTailB columns with two barriers per block:
// the block's diagonal part is solved inside warps (16 lanes hold the block's
// rows of one direction and pass each finished value along with a shuffle),
// then every row below (above, for the backward solve) takes the block's
// contribution in one CTA-wide pass.
constexpr int kTailB = 16;

__device__ __forceinline__ double tri_l(const double* src, int T, int i, int j) { return src[lpack_off(j, T) + (i - j - 1)]; }
__device__ __forceinline__ double tri_u(const double* src, int i, int j) { return src[upack_off(j) + i]; }

template <bool SCALE>
__device__ void tail_fwd(const DirGrid& g, const double* __restrict__ tri_g, double* X, int64_t ld, int c0, int D,
                         double* xt, double* tri) {
    const int T = g.T, t0 = g.t0;
    const int ntri = T * (T - 1) / 2;
    if (tri)
        for (int i = threadIdx.x; i < ntri; i += blockDim.x) tri[i] = tri_g[i];
    const double* src = tri ? tri : tri_g;
    for (int it = threadIdx.x; it < T * D; it += blockDim.x) {
        int i = it / D, d = it - i * D;
        xt[it] = X[(int64_t)(t0 + i) * ld + c0 + d];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, l = lane & 15;
    const int hw = (int)(threadIdx.x >> 4), nhw = (int)(blockDim.x >> 4);
    const unsigned hmask = (lane < 16) ? 0x0000ffffu : 0xffff0000u;
    for (int b0 = 0; b0 < T; b0 += kTailB) {
        const int bn = min(kTailB, T - b0);
        // (1) diagonal block: rows b0 + l of direction d, one half-warp per direction
        if (hw < D) {
            double a[kTailB];
#pragma unroll
            for (int m = 0; m < kTailB; m++) a[m] = (m < l && l < bn) ? tri_l(src, T, b0 + l, b0 + m) : 0.0;
            for (int d = hw; d < D; d += nhw) {
                double v = l < bn ? xt[(b0 + l) * D + d] : 0.0;
#pragma unroll
                for (int m = 0; m < kTailB - 1; m++) {
                    const double ym = __shfl_sync(hmask, v, m, 16);
                    v = fma(-a[m], ym, v);
                }
                if (l < bn) xt[(b0 + l) * D + d] = v;
            }
        }
        __syncthreads();
        // (2) rows below the block take its contribution
        const int n = (T - b0 - bn) * D;
        for (int it = threadIdx.x; it < n; it += blockDim.x) {
            const int i = b0 + bn + it / D, d = it % D;
            double v = xt[i * D + d];
            for (int m = 0; m < bn; m++) v = fma(-tri_l(src, T, i, b0 + m), xt[(b0 + m) * D + d], v);
            xt[i * D + d] = v;
        }
        __syncthreads();
    }
    for (int it = threadIdx.x; it < T * D; it += blockDim.x) {
        int i = it / D, d = it - i * D;
        double v = xt[it];
        X[(int64_t)(t0 + i) * ld + c0 + d] = SCALE ? v * g.invdiag[t0 + i] : v;
    }
    __syncthreads();
}

template <bool SCALE>
__device__ void tail_bwd(const DirGrid& g, const double* __restrict__ tri_g, double* X, int64_t ld, int c0, int D,
                         double* xt, double* tri) {
    const int T = g.T, t0 = g.t0;
    const int ntri = T * (T - 1) / 2;
    if (tri)
        for (int i = threadIdx.x; i < ntri; i += blockDim.x) tri[i] = tri_g[i];
    const double* src = tri ? tri : tri_g;
    for (int it = threadIdx.x; it < T * D; it += blockDim.x) {
        int i = it / D, d = it - i * D;
        xt[it] = X[(int64_t)(t0 + i) * ld + c0 + d];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, l = lane & 15;
    const int hw = (int)(threadIdx.x >> 4), nhw = (int)(blockDim.x >> 4);
    const unsigned hmask = (lane < 16) ? 0x0000ffffu : 0xffff0000u;
    for (int be = T; be > 0; be -= kTailB) {
        const int b0 = be > kTailB ? be - kTailB : 0, bn = be - b0;
        // (1) diagonal block, bottom-up: row b0 + l takes the finished values of the rows after it
        if (hw < D) {
            double a[kTailB];
#pragma unroll
            for (int m = 0; m < kTailB; m++) a[m] = (l < m && m < bn) ? tri_u(src, b0 + l, b0 + m) : 0.0;
            for (int d = hw; d < D; d += nhw) {
                double v = l < bn ? xt[(b0 + l) * D + d] : 0.0;
#pragma unroll
                for (int m = kTailB - 1; m > 0; m--) {
                    const double ym = __shfl_sync(hmask, v, m, 16);
                    v = fma(-a[m], ym, v);
                }
                if (l < bn) xt[(b0 + l) * D + d] = v;
            }
        }
        __syncthreads();
        // (2) rows above the block take its contribution
        const int n = b0 * D;
        for (int it = threadIdx.x; it < n; it += blockDim.x) {
            const int i = it / D, d = it - i * D;
            double v = xt[i * D + d];
            for (int m = 0; m < bn; m++) v = fma(-tri_u(src, i, b0 + m), xt[(b0 + m) * D + d], v);
            xt[i * D + d] = v;
        }
        __syncthreads();
    }
    for (int it = threadIdx.x; it < T * D; it += blockDim.x) {
        int i = it / D, d = it - i * D;
        double v = xt[it];
        X[(int64_t)(t0 + i) * ld + c0 + d] = SCALE ? v * g.invdiag[t0 + i] : v;
    }
    __syncthreads();
}

// Projection (eq. 11/13): y = [lambda^T Hess g + Hess f] v for v = (z, w).
// Gathered bus by bus over the incident branches (no atomics, deterministic):
//   y_v(b)  = d2_b dv_b + A_b dth_b + sum_e ( K_e dv_j - a_e dth_j )
//   y_th(b) = A_b dv_b  + C_b dth_b + sum_e ( b_e dv_j - c_e dth_j )
// plus c''_slack (grad P_slack . v) grad P_slack and c''_k w_Pg_k.
__device__ __forceinline__ double flip_sign(double v, bool flip) {
    // negation through the sign bit (an integer operation, not an FP64 instruction)
    return __longlong_as_double(__double_as_longlong(v) ^ (flip ? (long long)0x8000000000000000ULL : 0LL));
}

// Buses are visited in the order tp_bus (degree descending), so the lanes of a
// warp mostly share their incidence count; each output is one FMA chain; the
// slack-neighbour and Pg terms, which few buses have, are only issued by warps
// that hold such a bus (a predicated FP64 instruction costs its issue slot).
// fold_ut: the launch runs the U'^T sweep over the sparse levels next; its level 0
// (buses without L entries outside their block, so x_theta = b_theta and, for a PQ
// bus, x_v = b_v - u'_tv x_theta) is done here and the sweep starts at level 1.
__device__ void tproj(const DirGrid& g, const double* V, double* T, int64_t ld, int c0, int D, double* sref,
                      bool fold_ut) {
    double c2r = *g.c2ref;
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        double s = 0.0;
        for (int e = 0; e < g.n_gref; e++)
            if (inb(g.gref_row[e], g.zero_row + 1)) s = fma(g.gref_val[e], V[(int64_t)g.gref_row[e] * ld + c0 + d], s);
        sref[d] = c2r * s;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < g.n_bus * D; it += blockDim.x) {
        int bi = it / D, d = it - bi * D;
        int b = g.tp_bus[bi];
        int64_t c = c0 + d;
        int rth = g.uth[b], rv = g.uv[b];
        const int rows = g.zero_row + 1;
        double dth = inb(rth, rows) ? V[(int64_t)rth * ld + c] : 0.0, dv = inb(rv, rows) ? V[(int64_t)rv * ld + c] : 0.0;
        double ab = g.asum[b];
        double yv = fma(g.d2[b], dv, ab * dth);
        double yth = fma(ab, dv, g.csum[b] * dth);
        int e = g.inc_ptr[b];
        const int e1 = g.inc_ptr[b + 1];
        for (; e + 2 <= e1; e += 2) {
            const int t0 = g.inc_uth[e], v0 = g.inc_uv[e], t1 = g.inc_uth[e + 1], v1 = g.inc_uv[e + 1];
            const double dthj0 = inb(t0, rows) ? V[(int64_t)t0 * ld + c] : 0.0;
            const double dvj0 = inb(v0, rows) ? V[(int64_t)v0 * ld + c] : 0.0;
            const double dthj1 = inb(t1, rows) ? V[(int64_t)t1 * ld + c] : 0.0;
            const double dvj1 = inb(v1, rows) ? V[(int64_t)v1 * ld + c] : 0.0;
            const double4_32a cf0 = g.inc_coef[e], cf1 = g.inc_coef[e + 1];
            yv = fma(cf0.x, dvj0, yv);
            yv = fma(cf0.y, dthj0, yv);
            yth = fma(cf0.z, dvj0, yth);
            yth = fma(cf0.w, dthj0, yth);
            yv = fma(cf1.x, dvj1, yv);
            yv = fma(cf1.y, dthj1, yv);
            yth = fma(cf1.z, dvj1, yth);
            yth = fma(cf1.w, dthj1, yth);
        }
        if (warp_any(e < e1)) {
            if (e < e1) {
                const double4_32a cf = g.inc_coef[e];
                const double dthj = inb(g.inc_uth[e], rows) ? V[(int64_t)g.inc_uth[e] * ld + c] : 0.0;
                const double dvj = inb(g.inc_uv[e], rows) ? V[(int64_t)g.inc_uv[e] * ld + c] : 0.0;
                yv = fma(cf.x, dvj, yv);
                yv = fma(cf.y, dthj, yv);
                yth = fma(cf.z, dvj, yth);
                yth = fma(cf.w, dthj, yth);
            }
        }
        const bool hg = g.has_gref[b];
        if (warp_any(hg)) {
            if (hg) {
                yv = fma(sref[d], g.gref_v[b], yv);
                yth = fma(sref[d], g.gref_th[b], yth);
            }
        }
        if (rth != g.zero_row && inb(rth, rows)) T[(int64_t)rth * ld + c] = flip_sign(yth, true);
        const int l0 = fold_ut ? g.tp_l0[b] : -1;
        if (warp_any(l0 >= 0)) {
            if (l0 >= 0) yv = fma(-g.Atd[l0], yth, yv);   // T_v = -yv + u'_tv yth
        }
        if (inb(rv, rows)) T[(int64_t)rv * ld + c] = flip_sign(yv, rv < g.n_x);
        const int pr = g.pg_row[b];
        if (warp_any(pr >= 0)) {
            if (pr >= 0 && inb(pr, rows)) T[(int64_t)pr * ld + c] = g.pg_curv[b] * V[(int64_t)pr * ld + c];
        }
    }
}

// identity W: the column of direction j of the launch (and of its HW, relative to col0)
__device__ __forceinline__ int id_col(const DirLaunch& L, int j) { return L.colmap ? L.colmap[L.col0 + j] : L.col0 + j; }

// HW = Y_p + J_p^T Psi (Algorithm 2, SpMulAdd): one lane per p row k, directions
// blocked W at a time, so a warp's stores of one direction are consecutive.
template <int W>
__device__ __forceinline__ void muladd_row(const DirGrid& g, const DirLaunch& L, const double* T, int64_t ld, int c0,
                                           int d0, int k) {
    double h[W];
#pragma unroll
    for (int w = 0; w < W; w++) h[w] = T[(int64_t)(g.n_x + k) * ld + d0 + w];
    const int t1 = g.jpt_ptr[k + 1];
    for (int t = g.jpt_ptr[k]; t < t1; t++) {
        const double v = g.jptvd[t];
        if (!inb(g.jpt_row[t], g.n_x)) continue;
        const double* pr = T + (int64_t)g.jpt_row[t] * ld + d0;
#pragma unroll
        for (int w = 0; w < W; w++) h[w] = fma(v, pr[w], h[w]);
    }
#pragma unroll
    for (int w = 0; w < W; w++) L.HW[(int64_t)(id_col(L, c0 + d0 + w) - L.col0) * L.ldhw + k] = h[w];
}

// Algorithm 2 for the directions owned by CTA `cta` of launch L on grid g.
__device__ __forceinline__ void dirs_body(const DirGrid& g, const DirLaunch& L, const int cta, double* part,
                                          double* sref, unsigned* mask_smem) {
    const int c0 = (int)((int64_t)cta * L.N / L.n_cta);
    const int c1 = (int)((int64_t)(cta + 1) * L.N / L.n_cta);
    const int D = c1 - c0;
    if (D <= 0) return;
    // this CTA's directions: row r, local direction d at base[r * ld + d]
    const int64_t ld = L.ld;
    {
        // the CTA's last element lies in the buffers (bounds build; the condition is
        // the same for every thread of the CTA, so leaving here skips no barrier)
        const int64_t first = L.cta_stride ? (int64_t)cta * L.cta_stride : (int64_t)c0;
        const int64_t last = first + (int64_t)g.zero_row * ld + D - 1;
        if (!inb((L.cta_stride ? 0 : c0) + D - 1, ld) || (L.ws_elems > 0 && !inb(last, L.ws_elems))) return;
    }
    const int64_t base = L.cta_stride ? (int64_t)cta * L.cta_stride : (int64_t)c0;
    double* V = L.V + base;
    double* T = L.T + base;
    if (L.phases & PH_WLOAD) {
        for (int it = threadIdx.x; it < g.n_p * D; it += blockDim.x) {
            int k = it / D, d = it - k * D;
            int64_t c = c0 + d;
            double w = L.W ? L.W[c * L.ldw + k] : (k == id_col(L, (int)c) ? 1.0 : 0.0);
            V[(int64_t)(g.n_x + k) * ld + d] = w;
        }
        for (int d = threadIdx.x; d < D; d += blockDim.x) V[(int64_t)g.zero_row * ld + d] = 0.0;
        __syncthreads();
    }
    unsigned* seed = nullptr;
    if ((L.phases & PH_SPMUL) && !L.W && L.use_reach) {
        // identity W with the reach-restricted forward sweep: only the buses of this
        // CTA's J_p columns (all their rows, every direction) and the dense tail are
        // zeroed before the scatter; the forward sweep writes the other rows of the
        // reach, and the rows outside it are zero and never read
        seed = mask_smem + (g.n_x + 31) / 32;
        for (int i = threadIdx.x; i < (g.n_x + 31) / 32; i += blockDim.x) seed[i] = 0u;
        for (int it = threadIdx.x; it < g.T * D; it += blockDim.x) {
            const int i = it / D, d = it - i * D;
            V[(int64_t)(g.t0 + i) * ld + d] = 0.0;
        }
        __syncthreads();
        for (int d = threadIdx.x / 8; d < D; d += blockDim.x / 8) {
            const int k = id_col(L, c0 + d);
            for (int t = g.jpt_ptr[k] + (threadIdx.x & 7); t < g.jpt_ptr[k + 1]; t += 8) {
                const int qb = g.qtheta[g.jpt_row[t]];
                const bool two = qb + 1 < g.n_x && g.qtheta[qb + 1] == qb;
                mask_set(seed, qb);
                if (two) mask_set(seed, qb + 1);
                for (int e = 0; e < D; e++) {
                    V[(int64_t)qb * ld + e] = 0.0;
                    if (two) V[(int64_t)(qb + 1) * ld + e] = 0.0;
                }
            }
        }
        __syncthreads();
        for (int d = threadIdx.x / 8; d < D; d += blockDim.x / 8) {
            const int k = id_col(L, c0 + d);
            for (int t = g.jpt_ptr[k] + (threadIdx.x & 7); t < g.jpt_ptr[k + 1]; t += 8)
                V[(int64_t)g.jpt_row[t] * ld + d] = -g.jptvd[t];
        }
        __syncthreads();
    } else if ((L.phases & PH_SPMUL) && !L.W) {
        // identity W: -B column c is minus column col0 + c of J_p; zero the x rows
        // (stores only), then scatter the few entries of each column
        const int rstep = (int)blockDim.x / D;
        if (threadIdx.x < rstep * D) {
            const int d = threadIdx.x % D;
            for (int r = threadIdx.x / D; r < g.n_x; r += rstep) V[(int64_t)r * ld + d] = 0.0;
        }
        __syncthreads();
        for (int d = threadIdx.x / 8; d < D; d += blockDim.x / 8) {
            const int k = id_col(L, c0 + d);
            for (int t = g.jpt_ptr[k] + (threadIdx.x & 7); t < g.jpt_ptr[k + 1]; t += 8)
                V[(int64_t)g.jpt_row[t] * ld + d] = -g.jptvd[t];
        }
        __syncthreads();
    } else if (L.phases & PH_SPMUL) {
        // rows of J_p without entries: -B is zero there (stores only, no loads)
        for (int it = threadIdx.x; it < g.n_jp_zero * D; it += blockDim.x) {
            int r = it / D, d = it - r * D;
            V[(int64_t)g.jp_zero_rows[r] * ld + d] = 0.0;
        }
        for (int it = threadIdx.x; it < g.n_jp_rows * D; it += blockDim.x) {
            int r = it / D, d = it - r * D;
            const int q = g.jp_rows[r];
            double s = 0.0;
            for (int t = g.jp_ptr[q]; t < g.jp_ptr[q + 1]; t++)
                s = fma(g.jpv[t], V[(int64_t)(g.n_x + g.jp_col[t]) * ld + d], s);
            V[(int64_t)q * ld + d] = -s * g.invdiag[q];     // D^-1 B for the unit-diagonal factors
        }
        __syncthreads();
    }
    if (L.use_tail) {
        // identity W: the reach of B's columns (one bit per row; L, U and the tail's
        // external phase in this launch); rows outside it are zero in Z's forward sweep
        unsigned* mask = nullptr;
        if ((L.phases & PH_L) && L.use_reach) {
            mask = mask_smem;
            if (L.reach) {
                const int words = L.reach->words;
                const unsigned* m = L.reach->masks + (int64_t)cta * words;
                for (int i = threadIdx.x; i < words; i += blockDim.x) mask[i] = m[i];
            } else if (seed) {
                for (int i = threadIdx.x; i < (g.n_x + 31) / 32; i += blockDim.x) mask[i] = seed[i];
            } else {
                for (int i = threadIdx.x; i < (g.n_x + 31) / 32; i += blockDim.x) mask[i] = 0u;
                __syncthreads();
                for (int d = threadIdx.x / 8; d < D; d += blockDim.x / 8) {
                    const int k = id_col(L, c0 + d);
                    for (int t = g.jpt_ptr[k] + (threadIdx.x & 7); t < g.jpt_ptr[k + 1]; t += 8) {
                        const int qb = g.qtheta[g.jpt_row[t]];
                        mask_set(mask, qb);
                        if (qb + 1 < g.n_x && g.qtheta[qb + 1] == qb) mask_set(mask, qb + 1);
                    }
                }
            }
            __syncthreads();
        }
        if (L.phases & PH_L) {
            if (mask && L.reach) {
                // the CTA's reach, level by level, precomputed: nothing to skip or grow
                const ReachSched& R = *L.reach;
                const int m0 = R.lev0[cta];
                const LevelSet rs = {R.nlev[cta], R.ptr + m0 + cta, R.slots, R.maxext + m0};
                sweep_fwd<false, false, true>(g, rs, g.Ad, V, ld, 0, D, part, nullptr, seed, mask);
                sweep_fwd<false, true, true>(g, g.ef, g.Ad, V, ld, 0, D, part, nullptr, nullptr, mask);
            } else if (mask) {
                sweep_fwd<false, false, true>(g, g.sf, g.Ad, V, ld, 0, D, part, mask, seed, mask);
                sweep_fwd<false, true, true>(g, g.ef, g.Ad, V, ld, 0, D, part, nullptr, nullptr, mask);
            } else {
                sweep_fwd<false>(g, g.sf, g.Ad, V, ld, 0, D, part);
                sweep_fwd<false, true>(g, g.ef, g.Ad, V, ld, 0, D, part);
            }
            tail_fwd<false>(g, g.triLd, V, ld, 0, D, part, nullptr);
        }
        if (L.phases & PH_U) {
            tail_bwd<false>(g, g.triUd, V, ld, 0, D, part, nullptr);
            sweep_bwd<false>(g, g.sb, g.Ad, V, ld, 0, D, part, mask);
        }
    } else {
        if (L.phases & PH_L) sweep_fwd<false>(g, g.lf, g.Ad, V, ld, 0, D, part);
        if (L.phases & PH_U) sweep_bwd<false>(g, g.lb, g.Ad, V, ld, 0, D, part);
    }
    const bool fold_ut = (L.phases & PH_TPROJ) && (L.phases & PH_UT) && L.use_tail && g.sf.n_lev > 0;
    if (L.phases & PH_TPROJ) {
        tproj(g, V, T, ld, 0, D, sref, fold_ut);
        __syncthreads();
    }
    if (L.use_tail) {
        if (L.phases & PH_UT) {
            LevelSet sf = g.sf;
            if (fold_ut) {   // level 0 was done by the projection
                sf.n_lev -= 1;
                sf.ptr += 1;
                sf.maxext += 1;
            }
            sweep_fwd<false>(g, sf, g.Atd, T, ld, 0, D, part);
            sweep_fwd<false, true>(g, g.ef, g.Atd, T, ld, 0, D, part);
            tail_fwd<false>(g, g.triUtd, T, ld, 0, D, part, nullptr);
        }
        if (L.phases & PH_LT) {
            // psi is only read by SpMulAdd here: rows outside J_p and its ancestors are skipped
            tail_bwd<false>(g, g.triLtd, T, ld, 0, D, part, nullptr);
            sweep_bwd<false>(g, (L.phases & PH_MULADD) ? g.sbr : g.sb, g.Atd, T, ld, 0, D, part);
        }
    } else {
        if (L.phases & PH_UT) sweep_fwd<false>(g, g.lf, g.Atd, T, ld, 0, D, part);
        if (L.phases & PH_LT) sweep_bwd<false>(g, g.lb, g.Atd, T, ld, 0, D, part);
    }
    if (L.phases & PH_MULADD) {
        for (int k = threadIdx.x; k < g.n_p; k += blockDim.x) {
            int d0 = 0;
            for (; d0 + 8 <= D; d0 += 8) muladd_row<8>(g, L, T, ld, c0, d0, k);
            if (d0 + 4 <= D) { muladd_row<4>(g, L, T, ld, c0, d0, k); d0 += 4; }
            if (d0 + 2 <= D) { muladd_row<2>(g, L, T, ld, c0, d0, k); d0 += 2; }
            if (d0 < D) muladd_row<1>(g, L, T, ld, c0, d0, k);
        }
    }
}

__global__ void __launch_bounds__(kDirThreads, kDirCtasPerSm) k_dirs(DirGrid g, DirLaunch L) {
    __shared__ double part[kPartCap];
    __shared__ double sref[kDMax];
    extern __shared__ unsigned mask_smem[];
    dirs_body(g, L, blockIdx.x, part, sref, mask_smem);
}

// Several (grid, W block) items in one launch: CTA b belongs to the item i with
// cta_ptr[i] <= b < cta_ptr[i + 1]; the item descriptors travel in the kernel
// parameters and are copied to shared memory.
template <int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_dirs_batch(DirBatch B) {
    __shared__ double part[kPartCap];
    __shared__ double sref[kDMax];
    __shared__ DirGrid sg;
    __shared__ DirLaunch sl;
    int item = 0;
    while (item + 1 < B.n_items && (int)blockIdx.x >= B.cta_ptr[item + 1]) item++;
    if (threadIdx.x == 0) {
        sg = B.g[item];
        sl = B.l[item];
    }
    __syncthreads();
    dirs_body(sg, sl, (int)blockIdx.x - B.cta_ptr[item], part, sref, nullptr);
}

// Sweeps of a single right-hand side held in shared memory (k_solve1).  There
// is nothing to coalesce, so each bus block of a level takes a group of G
// lanes (G a power of two, G * nb <= blockDim): the lanes stride over the row
// and combine their sums with warp shuffles in log2(G) steps, and lane 0 of the
// group finishes the block.  One barrier per level.  (Spreading a level over a
// thread-block cluster with x replicated through distributed shared memory was
// slower: a level's cost is its chain of dependent loads, which more CTAs do not
// shorten, and a cluster barrier costs more than a CTA barrier.)
__device__ __forceinline__ int group_size(int nb, int maxext, int threads) {
    int G = 1;
    while (G < 32 && 2 * G * nb <= threads && G < maxext) G *= 2;
    return G;
}

// s0 -= sum v0[e] x[col[e]], s1 likewise, over e = e0, e0 + G, ... < n; unrolled by
// 4 so that four independent index/value loads (L2: read once per solve) are in
// flight per lane.
__device__ __forceinline__ void row1_sub(const int* __restrict__ col, const double* __restrict__ vals, int r0, int r1,
                                         int e0, int n, int G, const double* X, bool two, double& s0, double& s1) {
    int e = e0;
    for (; e + 3 * G < n; e += 4 * G) {
        const int i0 = col[r0 + e], i1 = col[r0 + e + G], i2 = col[r0 + e + 2 * G], i3 = col[r0 + e + 3 * G];
        const double u0 = vals[r0 + e], u1 = vals[r0 + e + G], u2 = vals[r0 + e + 2 * G], u3 = vals[r0 + e + 3 * G];
        double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
        if (two) {
            w0 = vals[r1 + e];
            w1 = vals[r1 + e + G];
            w2 = vals[r1 + e + 2 * G];
            w3 = vals[r1 + e + 3 * G];
        }
        const double x0 = X[i0], x1 = X[i1], x2 = X[i2], x3 = X[i3];
        s0 = fma(-u0, x0, s0);
        s0 = fma(-u1, x1, s0);
        s0 = fma(-u2, x2, s0);
        s0 = fma(-u3, x3, s0);
        if (two) {
            s1 = fma(-w0, x0, s1);
            s1 = fma(-w1, x1, s1);
            s1 = fma(-w2, x2, s1);
            s1 = fma(-w3, x3, s1);
        }
    }
    for (; e < n; e += G) {
        const double xv = X[col[r0 + e]];
        s0 = fma(-vals[r0 + e], xv, s0);
        if (two) s1 = fma(-vals[r1 + e], xv, s1);
    }
}

// sum of s over the G lanes of a group (G <= 32; groups are whole and aligned in
// the warp)
__device__ __forceinline__ void group_sum(int it, int items, int G, double& s0, double& s1) {
    if (G == 1) return;
    const int live = items - (it - (int)(threadIdx.x & 31));      // lanes of this warp holding an item
    const unsigned m = live >= 32 ? 0xffffffffu : ((1u << live) - 1u);
    for (int off = G / 2; off > 0; off >>= 1) {
        s0 += __shfl_down_sync(m, s0, off, G);
        s1 += __shfl_down_sync(m, s1, off, G);
    }
}

// The first item of a level for one thread, with everything it needs that does
// not depend on x: its slot, the first four (column, value) pairs of its share
// of the row and the finishing data.  Loaded for the next level before the
// barrier that ends the current one, so that after the barrier only the
// shared-memory reads of x and the FMAs remain on the critical path (for rows
// whose share is longer than four entries the rest is loaded as before).
struct Pf1 {
    int4 sl;
    int i[4];
    double u[4], w[4];
    double inv0, inv1, vt;
    bool valid;
};

template <bool FWD, bool SCALE, bool FIN>
__device__ __forceinline__ void pf1_load(const DirGrid& g, const int4* __restrict__ slots,
                                         const double* __restrict__ vals, int b0, int nb, int G, int it, Pf1& p) {
    p.valid = it < nb * G;
    if (!p.valid) return;
    const int bi = it / G, li = it - bi * G;
    p.sl = slots[b0 + bi];
    const int n = p.sl.y, r0 = p.sl.z;
    const bool two = p.sl.w >= 0;
    const int r1 = two ? p.sl.w : r0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int e = li + k * G;
        const bool in = e < n;
        p.i[k] = in ? g.col[r0 + e] : -1;
        p.u[k] = in ? vals[r0 + e] : 0.0;
        p.w[k] = (in && two) ? vals[r1 + e] : 0.0;
    }
    if (FIN && li == 0) {
        const int q = p.sl.x;
        p.inv0 = SCALE ? g.invdiag[q] : 1.0;
        p.inv1 = (SCALE && two) ? g.invdiag[q + 1] : 1.0;
        p.vt = two ? vals[FWD ? r1 + n : r0 - 1] : 0.0;
    }
}

// row share of one item: the prefetched first chunk, then the rest of the row
__device__ __forceinline__ void pf1_sum(const DirGrid& g, const double* __restrict__ vals, const Pf1& p, int li,
                                        int G, const double* X, double& s0, double& s1) {
    const int n = p.sl.y, r0 = p.sl.z;
    const bool two = p.sl.w >= 0;
    const int r1 = two ? p.sl.w : r0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        if (p.i[k] >= 0) {
            const double xv = X[p.i[k]];
            s0 = fma(-p.u[k], xv, s0);
            if (two) s1 = fma(-p.w[k], xv, s1);
        }
    }
    row1_sub(g.col, vals, r0, r1, li + 4 * G, n, G, X, two, s0, s1);
}

template <bool SCALE, bool EXT>
__device__ void sweep1_fwd(const DirGrid& g, const LevelSet& ls, const double* __restrict__ vals, double* X) {
    const int TT = (int)blockDim.x, gt = (int)threadIdx.x;
    if (ls.n_lev <= 0) return;
    int b0 = ls.ptr[0], nb = ls.ptr[1] - b0, G = group_size(nb, ls.maxext[0], TT);
    Pf1 cur;
    pf1_load<true, SCALE, !EXT>(g, ls.slots, vals, b0, nb, G, gt, cur);
    for (int lev = 0; lev < ls.n_lev; lev++) {
        int b0n = 0, nbn = 0, Gn = 1;
        if (lev + 1 < ls.n_lev) {
            b0n = ls.ptr[lev + 1];
            nbn = ls.ptr[lev + 2] - b0n;
            Gn = group_size(nbn, ls.maxext[lev + 1], TT);
        }
        for (int it = gt; it < nb * G; it += TT) {
            Pf1 p = cur;
            if (it != gt) pf1_load<true, SCALE, !EXT>(g, ls.slots, vals, b0, nb, G, it, p);
            const int li = it - (it / G) * G;
            const int q = p.sl.x;
            const bool two = p.sl.w >= 0;
            double s0 = 0.0, s1 = 0.0;
            pf1_sum(g, vals, p, li, G, X, s0, s1);
            group_sum(it, nb * G, G, s0, s1);
            if (li == 0) {
                const double a0 = X[q] + s0;
                double a1 = two ? X[q + 1] + s1 : 0.0;
                if (EXT) {
                    X[q] = a0;
                    if (two) X[q + 1] = a1;
                } else {
                    const double x0 = SCALE ? a0 * p.inv0 : a0;
                    X[q] = x0;
                    if (two) {
                        a1 = fma(-p.vt, x0, a1);
                        X[q + 1] = SCALE ? a1 * p.inv1 : a1;
                    }
                }
            }
        }
        if (lev + 1 < ls.n_lev) pf1_load<true, SCALE, !EXT>(g, ls.slots, vals, b0n, nbn, Gn, gt, cur);
        __syncthreads();
        b0 = b0n;
        nb = nbn;
        G = Gn;
    }
}

template <bool SCALE>
__device__ void sweep1_bwd(const DirGrid& g, const LevelSet& ls, const double* __restrict__ vals, double* X) {
    const int TT = (int)blockDim.x, gt = (int)threadIdx.x;
    if (ls.n_lev <= 0) return;
    int b0 = ls.ptr[0], nb = ls.ptr[1] - b0, G = group_size(nb, ls.maxext[0], TT);
    Pf1 cur;
    pf1_load<false, SCALE, true>(g, ls.slots, vals, b0, nb, G, gt, cur);
    for (int lev = 0; lev < ls.n_lev; lev++) {
        int b0n = 0, nbn = 0, Gn = 1;
        if (lev + 1 < ls.n_lev) {
            b0n = ls.ptr[lev + 1];
            nbn = ls.ptr[lev + 2] - b0n;
            Gn = group_size(nbn, ls.maxext[lev + 1], TT);
        }
        for (int it = gt; it < nb * G; it += TT) {
            Pf1 p = cur;
            if (it != gt) pf1_load<false, SCALE, true>(g, ls.slots, vals, b0, nb, G, it, p);
            const int li = it - (it / G) * G;
            const int q = p.sl.x;
            const bool two = p.sl.w >= 0;
            double s0 = 0.0, s1 = 0.0;
            pf1_sum(g, vals, p, li, G, X, s0, s1);
            group_sum(it, nb * G, G, s0, s1);
            if (li == 0) {
                double a0 = X[q] + s0;
                if (two) {
                    const double a1 = X[q + 1] + s1;
                    const double x1 = SCALE ? a1 * p.inv1 : a1;
                    X[q + 1] = x1;
                    a0 = fma(-p.vt, x1, a0);
                }
                X[q] = SCALE ? a0 * p.inv0 : a0;
            }
        }
        if (lev + 1 < ls.n_lev) pf1_load<false, SCALE, true>(g, ls.slots, vals, b0n, nbn, Gn, gt, cur);
        __syncthreads();
        b0 = b0n;
        nb = nbn;
        G = Gn;
    }
}

// One right-hand side, one CTA, x held in shared memory for the whole sweep
// (Newton steps and the first-order adjoint).  Dynamic shared memory holds
// X[n_x] | the packed tail triangle (use_tail) | kSolve1Part doubles of scratch
// (the tail's right-hand side).  With the tail, the dense top block is solved
// column by column in shared memory, as in k_dirs, instead of as one sparse
// level per variable.
constexpr int kSolve1Part = 2048;
constexpr int kSolve1Threads = 768;   // 85 registers per thread: room for the prefetched level data
__device__ __forceinline__ void k_solve1_body(DirGrid g, double* x, unsigned phases, int use_tail) {
    extern __shared__ double X[];
    double* tri = X + g.n_x;
    double* part = tri + (use_tail ? (size_t)g.T * (g.T - 1) / 2 : 0);
    for (int q = threadIdx.x; q < g.n_x; q += blockDim.x) X[q] = x[q];
    __syncthreads();
    if (use_tail) {
        if (phases & PH_L) {
            sweep1_fwd<false, false>(g, g.sf, g.A, X);
            sweep1_fwd<false, true>(g, g.ef, g.A, X);
            tail_fwd<false>(g, g.triL, X, 1, 0, 1, part, tri);
        }
        if (phases & PH_U) {
            tail_bwd<true>(g, g.triU, X, 1, 0, 1, part, tri);
            sweep1_bwd<true>(g, g.sb, g.A, X);
        }
        if (phases & PH_UT) {
            sweep1_fwd<true, false>(g, g.sf, g.At, X);
            sweep1_fwd<true, true>(g, g.ef, g.At, X);
            tail_fwd<true>(g, g.triUt, X, 1, 0, 1, part, tri);
        }
        if (phases & PH_LT) {
            tail_bwd<false>(g, g.triLt, X, 1, 0, 1, part, tri);
            sweep1_bwd<false>(g, g.sb, g.At, X);
        }
    } else {
        if (phases & PH_L) sweep1_fwd<false, false>(g, g.lf, g.A, X);
        if (phases & PH_U) sweep1_bwd<true>(g, g.lb, g.A, X);
        if (phases & PH_UT) sweep1_fwd<true, false>(g, g.lf, g.At, X);
        if (phases & PH_LT) sweep1_bwd<false>(g, g.lb, g.At, X);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < g.n_x; q += blockDim.x) x[q] = X[q];
}
__global__ void __launch_bounds__(kSolve1Threads, 1) k_solve1(DirGrid g, double* x, unsigned phases, int use_tail) { k_solve1_body(g, x, phases, use_tail); }

// ---------------------------------------------------------------------------
// adjoint (eq. 7) and the per-state second-order coefficients
// ---------------------------------------------------------------------------

// Single thread: the slack cost derivatives, grad P_slack, the right-hand side
// -grad_x f = -c'_slack grad_x P_slack of the adjoint system, and F.
__global__ void k_adjoint_rhs(PfGrid g, PfState s, AdjData a) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int r = g.ref;
    const double S = g.base_mva;
    double vr = s.vm[r], Pr = s.P[r];
    double pg_ref = Pr + s.pd[r];
    double cref = 2.0 * g.c2[r] * S * S * pg_ref + g.c1[r] * S;
    *a.cref = cref;
    *a.c2ref = 2.0 * g.c2[r] * S * S;
    int n = 0;
    for (int t = g.yp[r]; t < g.yp[r + 1]; t++) {
        int j = g.yj[t];
        if (j == r) {
            double dv = Pr / vr + g.G[t] * vr;
            a.gref_v[r] = dv;
            a.gref_th[r] = 0.0;
            a.gref_row[n] = a.uv[r];
            a.gref_val[n++] = dv;
            continue;
        }
        double sn, cs;
        sincos(s.va[r] - s.va[j], &sn, &cs);
        double vj = s.vm[j];
        double dth = vr * vj * (g.G[t] * sn - g.B[t] * cs);
        double dv = vr * (g.G[t] * cs + g.B[t] * sn);
        a.gref_th[j] = dth;
        a.gref_v[j] = dv;
        a.gref_row[n] = a.uth[j];
        a.gref_val[n++] = dth;
        a.gref_row[n] = a.uv[j];
        a.gref_val[n++] = dv;
        a.rhs[g.qth[j]] = -cref * dth;
        if (g.qv[j] >= 0) a.rhs[g.qv[j]] = -cref * dv;
    }
}

// F = sum over generators of c2 (S Pg)^2 + c1 S Pg, one block, fixed reduction order.
__global__ void k_objective(PfGrid g, PfState s, double* F) {
    __shared__ double red[256];
    const double S = g.base_mva;
    double acc = 0.0;
    for (int i = threadIdx.x; i < g.n_bus; i += blockDim.x) {
        if (g.qv[i] >= 0) continue;  // PQ bus: no generator
        double pg = (i == g.ref) ? s.P[i] + s.pd[i] : s.pg[i];
        double P = S * pg;
        acc += g.c2[i] * P * P + g.c1[i] * P;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *F = red[0];
}

// One thread per bus: bus weights mu, nu from lambda (mu_slack = c'_slack) and
// the coefficients of every incident branch for the gathered projection.
// With alpha = G(mu_i + mu_j) - B(nu_i + nu_j), beta = B(mu_i - mu_j) + G(nu_i - nu_j),
// t = theta_i - theta_j, the branch term of sum mu P + nu Q is
// v_i v_j (alpha cos t + beta sin t); K = alpha cos t + beta sin t,
// M = dK/dt, a = v_j M, b = v_i M, c = -v_i v_j K.
__global__ void k_adjoint_coef(PfGrid g, PfState s, const double* lam, const double* crefp, const int* inc_ptr,
                               const int* inc_nb, double4_32a* coef, double* d2, double* asum, double* csum,
                               double* pg_curv) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_bus) return;
    double cref = *crefp;
    double mu_i = g.qth[i] >= 0 ? lam[g.qth[i]] : cref;
    double nu_i = g.qv[i] >= 0 ? lam[g.qv[i]] : 0.0;
    double vi = s.vm[i];
    d2[i] = 2.0 * (mu_i * g.G[g.ydiag[i]] - nu_i * g.B[g.ydiag[i]]);
    double sa = 0.0, sc = 0.0;
    int e = inc_ptr[i];
    for (int t = g.yp[i]; t < g.yp[i + 1]; t++) {
        int j = g.yj[t];
        if (j == i) continue;
        double mu_j = g.qth[j] >= 0 ? lam[g.qth[j]] : cref;
        double nu_j = g.qv[j] >= 0 ? lam[g.qv[j]] : 0.0;
        double Gij = g.G[t], Bij = g.B[t];
        double alpha = Gij * (mu_i + mu_j) - Bij * (nu_i + nu_j);
        double beta = Bij * (mu_i - mu_j) + Gij * (nu_i - nu_j);
        double sn, cs;
        sincos(s.va[i] - s.va[j], &sn, &cs);
        double K = alpha * cs + beta * sn;
        double M = -alpha * sn + beta * cs;
        double vj = s.vm[j];
        double a = vj * M, bb = vi * M, c = -vi * vj * K;
        coef[e] = make_double4_32a(K, -a, bb, -c);
        sa += a;
        sc += c;
        e++;
    }
    asum[i] = sa;
    csum[i] = sc;
    pg_curv[i] = g.ip_pg[i] >= 0 ? 2.0 * g.c2[i] * g.base_mva * g.base_mva : 0.0;
}

// grad F = grad_p f + J_p^T lambda, one thread per bus (its v and Pg entries).
__global__ void k_gradient(PfGrid g, PfState s, const int* jpt_ptr, const int* jpt_row, const double* jptv,
                           const double* lam, const double* crefp, const double* gref_v, double* grad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n_bus) return;
    double cref = *crefp;
    int kv = g.ip_v[i];
    if (kv >= 0) {
        double h = cref * gref_v[i];
        for (int t = jpt_ptr[kv]; t < jpt_ptr[kv + 1]; t++) h = fma(jptv[t], lam[jpt_row[t]], h);
        grad[kv] = h;
    }
    int kp = g.ip_pg[i];
    if (kp >= 0) {
        double S = g.base_mva;
        double h = 2.0 * g.c2[i] * S * S * s.pg[i] + g.c1[i] * S;
        for (int t = jpt_ptr[kp]; t < jpt_ptr[kp + 1]; t++) h = fma(jptv[t], lam[jpt_row[t]], h);
        grad[kp] = h;
    }
}

// external column-major <-> internal row-major with a row map
__global__ void k_scatter_rows(int n_rows, int N, const int* map, const double* src, int64_t lds, double* dst,
                               int64_t ldd, double scale_x, int n_x) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= (int64_t)n_rows * N) return;
    int c = (int)(it / n_rows), r = (int)(it - (int64_t)c * n_rows);
    double v = src[(int64_t)c * lds + r];
    dst[(int64_t)map[r] * ldd + c] = r < n_x ? scale_x * v : v;
}

__global__ void k_gather_rows(int n_rows, int N, const int* map, const double* src, int64_t lds, double* dst,
                              int64_t ldd, double scale_x, int n_x) {
    int64_t it = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= (int64_t)n_rows * N) return;
    int c = (int)(it / n_rows), r = (int)(it - (int64_t)c * n_rows);
    double v = src[(int64_t)map[r] * lds + c];
    dst[(int64_t)c * ldd + r] = r < n_x ? scale_x * v : v;
}

int blocks_for(int64_t n, int t) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------------------
// Newton power flow over several grids of one topology: item blockIdx.y
// ---------------------------------------------------------------------------
__global__ void k_pf_eval_batch(PfBatch B) {
    const PfBatchItem& it = B.it[blockIdx.y];
    k_pf_eval_body(it.g, it.s, it.x, it.A, it.jpv, it.umax, it.umax + 1, 1);
}
__global__ void k_pf_prep_batch(PfBatch B) {
    const PfBatchItem& it = B.it[blockIdx.y];
    pf_prep_body(it.g, it.s, it.A, it.umax, nullptr, 1);
}
__global__ void __launch_bounds__(32 * kPfWarps) k_pf_eval_warp_batch(PfBatch B) {
    const PfBatchItem& it = B.it[blockIdx.y];
    pf_eval_warp_body(it.g, it.s, it.x, it.A, it.jpv, it.umax, it.umax + 1, 1);
}

__global__ void k_batch_status(PfBatch B, double* out) {
    const int i = threadIdx.x;
    if (i >= B.n) return;
    out[2 * i] = __longlong_as_double((long long)B.it[i].umax[0]);
    out[2 * i + 1] = (double)B.it[i].err[0];
}

__global__ void k_newton_update_batch(PfBatch B) {
    const PfBatchItem& it = B.it[blockIdx.y];
    k_newton_update_body(it.g, it.s, it.x);
}

__global__ void k_rf_update_batch(RfBatch B, int64_t t0, int64_t nt, int j0, int njob) {
    pdl_wait();
    k_rf_update_body(B.g[blockIdx.y], t0, nt, j0, njob);
}
__global__ void k_rf_leaf_piv_batch(RfBatch B, int njob) {
    pdl_wait();
    k_rf_leaf_piv_body(B.g[blockIdx.y], njob);
}
__global__ void k_rf_pivot_batch(RfBatch B) {
    pdl_wait();
    k_rf_pivot_body(B.g[blockIdx.y]);
}
__global__ void k_tail_gather_batch(RfBatch B) {
    pdl_wait();
    k_tail_gather_body(B.g[blockIdx.y]);
}
__global__ void __launch_bounds__(256) k_tail_step_batch(RfBatch B, int k) {
    pdl_wait();
    k_tail_step_body(B.g[blockIdx.y], k);
}
__global__ void k_tail_scatter_batch(RfBatch B) {
    pdl_wait();
    k_tail_scatter_body(B.g[blockIdx.y]);
}

// the single solves' tail triangles: L (unit lower) and U with column j scaled by 1/u_jj
__global__ void k_tail_tri_batch(TriBatch B) {
    const int i = blockIdx.y, T = B.T;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= T * T) return;
    const int r = idx / T, c = idx - r * T;
    if (r == c) return;
    const int p = B.pos[i][idx];
    const double a = p >= 0 ? B.A[i][p] : 0.0;
    if (r > c) B.triL[i][c * (T - 1) - c * (c - 1) / 2 + (r - c - 1)] = a;
    else B.triU[i][c * (c - 1) / 2 + r] = a * B.invdiag[i][B.t0 + c];
}

__global__ void __launch_bounds__(kSolve1Threads, 1) k_solve1_batch(Solve1Batch B, unsigned phases, int use_tail) {
    k_solve1_body(B.g[blockIdx.x], B.x[blockIdx.x], phases, use_tail);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------

void launch_injections(const PfGrid& g, const PfState& s, cudaStream_t st) {
    if (g.n_bus > 0) k_injections<<<blocks_for(g.n_bus, 128), 128, 0, st>>>(g, s);
}

static unsigned prep_blocks(const PfGrid& g) {
    const int64_t n = g.nnz_a > g.n_bus ? g.nnz_a : g.n_bus;
    const int64_t b = (n + 1023) / 1024;             // four entries per thread
    return (unsigned)(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}
void launch_pf_prep(const PfGrid& g, const PfState& s, double* A, unsigned long long* umax, int* err, bool zero,
                    cudaStream_t st) {
    k_pf_prep<<<prep_blocks(g), 256, 0, st>>>(g, s, A, umax, err, zero ? 1 : 0);
}
void launch_pf_prep_batch(const PfBatch& B, cudaStream_t st) {
    if (B.n > 0) k_pf_prep_batch<<<dim3(prep_blocks(B.it[0].g), (unsigned)B.n), 256, 0, st>>>(B);
}

void launch_pf_eval(const PfGrid& g, const PfState& s, double* gres, double* A, double* jpv,
                    unsigned long long* gmax, unsigned long long* jmax, bool want_jac, cudaStream_t st) {
    if (g.n_pfw > 0)
        k_pf_eval_warp<<<(g.n_pfw + kPfWarps - 1) / kPfWarps, 32 * kPfWarps, 0, st>>>(g, s, gres, A, jpv, gmax, jmax,
                                                                                   want_jac);
    else if (g.n_bus > 0)
        k_pf_eval<<<blocks_for(g.n_bus, 64), 64, 0, st>>>(g, s, gres, A, jpv, gmax, jmax, want_jac);
}

cudaError_t launch_jac_ad(const PfGrid& g, const PfState& s, const int* col_th, const int* col_v, const int* col_pg,
                          int n_colors, double* A, double* jpv, unsigned long long* jmax, cudaStream_t st) {
    constexpr int CH = 8;
    if (g.n_bus == 0 || n_colors == 0) return cudaSuccess;
    dim3 grid((unsigned)blocks_for(g.n_bus, 128), (unsigned)((n_colors + CH - 1) / CH));
    k_jac_ad<CH><<<grid, 128, 0, st>>>(g, s, col_th, col_v, col_pg, A, jpv, jmax);
    return cudaGetLastError();
}

void launch_newton_update(const PfGrid& g, const PfState& s, const double* dx, cudaStream_t st) {
    if (g.n_bus > 0) k_newton_update<<<blocks_for(g.n_bus, 128), 128, 0, st>>>(g, s, dx);
}

// L2 prefetch of read-only arrays: one bulk prefetch of up to kPrefetchChunk bytes
// per thread (TMA units of many SMs at once).  The refactorisation's level data
// (tens of MB on the 9241-bus grid) is otherwise read from HBM level by level,
// after the direction sweeps of the previous state evicted it from L2.
constexpr unsigned long long kPrefetchChunk = 4096;
__global__ void k_prefetch_l2(PrefetchList L) {
    const unsigned long long c = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (L.n <= 0 || c >= L.first[L.n]) return;
    int a = 0;
    while (a + 1 < L.n && c >= L.first[a + 1]) a++;
    const unsigned long long off = (c - L.first[a]) * kPrefetchChunk;
    if (off >= L.bytes[a]) return;
    unsigned long long n = L.bytes[a] - off;
    if (n > kPrefetchChunk) n = kPrefetchChunk;
    n &= ~15ull;
    if (n)
        asm volatile("{\n\t.reg .u64 ga;\n\tcvta.to.global.u64 ga, %0;\n\tcp.async.bulk.prefetch.L2.global [ga], %1;\n\t}"
                     :: "l"(L.p[a] + off), "r"((unsigned)n) : "memory");
}

void launch_prefetch_l2(const PrefetchList& in, cudaStream_t st) {
    PrefetchList L = in;
    L.first[0] = 0;
    for (int a = 0; a < L.n; a++) L.first[a + 1] = L.first[a] + (L.bytes[a] + kPrefetchChunk - 1) / kPrefetchChunk;
    const unsigned long long nc = L.n > 0 ? L.first[L.n] : 0;
    if (nc > 0) k_prefetch_l2<<<(unsigned)((nc + 31) / 32), 32, 0, st>>>(L);
}

cudaError_t launch_refactor(const RfGrid& g, const int* lev_ptr_host, const int64_t* tgt_lev_ptr_host,
                            const int* piv_lev_ptr_host, int n_lev, cudaStream_t st) {
    (void)lev_ptr_host;
    cudaError_t e = cudaSuccess;
    bool pdl = false;   // the first launch follows an event wait
    auto chk = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
        pdl = true;
    };
    if (n_lev > 0 && piv_lev_ptr_host[0] > 0)
        chk(launch_pdl(pdl, k_rf_leaf_piv, dim3(blocks_for(piv_lev_ptr_host[0], 128)), dim3(128), 0, st, g,
                       piv_lev_ptr_host[0]));
    for (int lev = 0; lev < n_lev; lev++) {
        const int64_t t0 = tgt_lev_ptr_host[lev], nt = tgt_lev_ptr_host[lev + 1] - t0;
        const int j0 = piv_lev_ptr_host[lev], njob = piv_lev_ptr_host[lev + 1] - j0;
        if (nt > 0) chk(launch_pdl(pdl, k_rf_update, dim3(blocks_for(nt, 256)), dim3(256), 0, st, g, t0, nt, j0, njob));
    }
    if (g.n_piv + g.n_pe > 0)
        chk(launch_pdl(pdl, k_rf_pivot, dim3(blocks_for((int64_t)g.n_piv + g.n_pe, 256)), dim3(256), 0, st, g));
    if (g.T > 0) {
        const int TT = g.T * g.T, nt = (g.T + kTailTB - 1) / kTailTB;
        chk(launch_pdl(pdl, k_tail_gather, dim3(blocks_for(TT, 256)), dim3(256), 0, st, g));
        for (int k = -1; k < nt; k++) {
            const int c = k + 1, U = c < nt ? nt - c - 1 : 0;
            const int grid = 2 * U + (k >= 0 ? 1 + U * U : 0);
            if (grid > 0) chk(launch_pdl(pdl, k_tail_step, dim3(grid), dim3(kTailTB * kTailTB), 0, st, g, k));
        }
        chk(launch_pdl(pdl, k_tail_scatter, dim3(blocks_for(TT, 256)), dim3(256), 0, st, g));
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

// The dynamic shared-memory limit is a per-kernel attribute of each device's
// context: raise it on every device once, to that device's maximum (minus the
// kernel's static shared memory), for every kernel that can need more than the
// 48 KB default.  The SM count is cached per device too.
constexpr int kMaxDevices = 64;
std::mutex g_dev_mu;
bool g_prepared[kMaxDevices];
int g_n_sm[kMaxDevices];

cudaError_t prepare_kernels() {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (g_prepared[dev]) return cudaSuccess;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    const void* fns[3] = {(const void*)k_dirs, (const void*)k_solve1, (const void*)k_solve1_batch};
    for (const void* f : fns) {
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, f);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    // the batched direction kernel's shapes: shared memory before L1, so that the
    // shape's resident CTAs fit an SM (6 x 35 KB for 128 threads)
    const void* shapes[4] = {(const void*)k_dirs_batch<128, 6>, (const void*)k_dirs_batch<192, 4>,
                             (const void*)k_dirs_batch<256, 3>, (const void*)k_dirs_batch<kDirThreads, kDirCtasPerSm>};
    for (const void* f : shapes) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
    }
    g_prepared[dev] = true;
    return cudaSuccess;
}

void launch_transpose_values(int nnz, const int* tpos, const int* arow, const int* col, const int* diagpos,
                             const double* A, const double* invdiag, double* At, double* Ad, double* Atd, int nnz_jp,
                             const int* jpt_src, const int* jpt_row, const double* jpv, double* jptv, double* jptvd,
                             cudaStream_t st) {
    int n = nnz > nnz_jp ? nnz : nnz_jp;
    if (n > 0)
        k_transpose_values<<<blocks_for(n, 256), 256, 0, st>>>(nnz, tpos, arow, col, diagpos, A, invdiag, At, Ad, Atd,
                                                               nnz_jp, jpt_src, jpt_row, jpv, jptv, jptvd);
}

// SMs of the current device (1 if the query fails)
static int num_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return 1;
    std::lock_guard<std::mutex> lock(g_dev_mu);
    if (g_n_sm[dev] == 0) {
        int n = 0;
        g_n_sm[dev] = (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0) ? n : 1;
    }
    return g_n_sm[dev];
}

int dirs_cta_slots_for(int n_sm) { return kDirCtasPerSm * n_sm; }

int dirs_ctas_for(int N, int slots) {
    int G = N < slots ? N : slots;
    int need = (N + kDMax - 1) / kDMax;
    if (G < need) G = need;
    return G < 1 ? 1 : G;
}

int dirs_default_ctas(int N) { return dirs_ctas_for(N, kDirCtasPerSm * num_sms()); }

bool dirs_tail_fits(int T, int N, int n_cta) {
    if (T <= 1 || n_cta <= 0) return false;
    int dmax = (N + n_cta - 1) / n_cta;
    return (int64_t)T * dmax <= kPartCap;      // the tail rows of the CTA's directions sit in `part`
}

void launch_dirs(const DirGrid& g, const DirLaunch& L, cudaStream_t st) {
    if (L.N <= 0 || L.n_cta <= 0) return;
    // active and seed masks, one bit per row each
    size_t smem = (L.use_tail && L.use_reach) ? 2 * (((size_t)g.n_x + 127) / 128 * 16) : 0;
    k_dirs<<<L.n_cta, kDirThreads, smem, st>>>(g, L);
}

// Compiled CTA shapes of the batched direction kernel: threads x resident CTAs per
// SM, 768 threads an SM each (the register bound of the 384 x 2 shape); the
// static shared memory (dense-tail rows, reference row, item descriptors) is
// about 35 KB a CTA, 210 KB an SM at 6 CTAs.
int dirs_batch_ctas_per_sm(int threads) {
    switch (threads) {
        case 128: return 6;
        case 192: return 4;
        case 256: return 3;
        case 384: return 2;
        default: return 0;
    }
}
bool dirs_batch_shape_ok(int threads) { return dirs_batch_ctas_per_sm(threads) > 0; }

void launch_dirs_batch(const DirBatch& B, int threads, cudaStream_t st) {
    const int n = B.n_items > 0 ? B.cta_ptr[B.n_items] : 0;
    if (n <= 0) return;
    switch (threads) {
        case 128: k_dirs_batch<128, 6><<<n, 128, 0, st>>>(B); break;
        case 192: k_dirs_batch<192, 4><<<n, 192, 0, st>>>(B); break;
        case 256: k_dirs_batch<256, 3><<<n, 256, 0, st>>>(B); break;
        default: k_dirs_batch<kDirThreads, kDirCtasPerSm><<<n, kDirThreads, 0, st>>>(B); break;
    }
}

void launch_scale_rows(int n, int N, const double* s, double* x, int64_t ld, cudaStream_t st) {
    if ((int64_t)n * N > 0) k_scale_rows<<<blocks_for((int64_t)n * N, 256), 256, 0, st>>>(n, N, s, x, ld);
}

void launch_build_tail(int T, int t0, const int* pos, const double* A, const double* invdiag, double* triL,
                       double* triU, double* triUt, double* triLt, double* triLd, double* triUd, double* triUtd,
                       double* triLtd, cudaStream_t st) {
    if (T > 1)
        k_build_tail<<<blocks_for((int64_t)T * T, 256), 256, 0, st>>>(T, t0, pos, A, invdiag, triL, triU, triUt, triLt,
                                                                      triLd, triUd, triUtd, triLtd);
}

void launch_adjoint_rhs(const PfGrid& g, const PfState& s, const AdjData& a, cudaStream_t st) {
    k_adjoint_rhs<<<1, 32, 0, st>>>(g, s, a);
    k_objective<<<1, 256, 0, st>>>(g, s, a.F);
}

static size_t solve1_smem(int n_x, int T, bool tail) {
    return ((size_t)n_x + (tail ? (size_t)T * (T - 1) / 2 : 0) + kSolve1Part) * sizeof(double);
}

int solve1_mode(int n_x, int T) {
    const size_t cap = 227 * 1024;
    if (T > 1 && T <= kSolve1Part && solve1_smem(n_x, T, true) <= cap) return 2;
    return solve1_smem(n_x, T, false) <= cap ? 1 : 0;
}

cudaError_t launch_solve1(const DirGrid& g, double* x, unsigned phases, bool use_tail, cudaStream_t st) {
    k_solve1<<<1, kSolve1Threads, solve1_smem(g.n_x, g.T, use_tail), st>>>(g, x, phases, use_tail ? 1 : 0);
    return cudaGetLastError();
}

int dirs_cta_slots() { return kDirCtasPerSm * num_sms(); }
int dirs_batch_slots(int threads) { return dirs_batch_ctas_per_sm(threads) * num_sms(); }

void launch_adjoint_coef(const PfGrid& g, const PfState& s, const double* lambda_int, const double* cref,
                         const int* inc_ptr, const int* inc_nb, double4_32a* inc_coef, double* d2, double* asum,
                         double* csum, double* pg_curv, cudaStream_t st) {
    if (g.n_bus > 0)
        k_adjoint_coef<<<blocks_for(g.n_bus, 128), 128, 0, st>>>(g, s, lambda_int, cref, inc_ptr, inc_nb, inc_coef,
                                                                 d2, asum, csum, pg_curv);
}

void launch_gradient(const PfGrid& g, const PfState& s, int n_p, const int* jpt_ptr, const int* jpt_row,
                     const double* jptv, const double* lambda_int, const double* cref, const double* gref_v,
                     double* grad, cudaStream_t st) {
    (void)n_p;
    if (g.n_bus > 0)
        k_gradient<<<blocks_for(g.n_bus, 128), 128, 0, st>>>(g, s, jpt_ptr, jpt_row, jptv, lambda_int, cref, gref_v,
                                                             grad);
}

void launch_scatter_rows(int n_rows, int N, const int* map, const double* src, int64_t lds, double* dst,
                         int64_t ldd, double scale_x, int n_x, cudaStream_t st) {
    int64_t n = (int64_t)n_rows * N;
    if (n > 0) k_scatter_rows<<<blocks_for(n, 256), 256, 0, st>>>(n_rows, N, map, src, lds, dst, ldd, scale_x, n_x);
}

void launch_pf_eval_batch(const PfBatch& B, cudaStream_t st) {
    if (B.n > 0 && B.it[0].g.n_pfw > 0)
        k_pf_eval_warp_batch<<<dim3((unsigned)((B.it[0].g.n_pfw + kPfWarps - 1) / kPfWarps), (unsigned)B.n),
                               32 * kPfWarps, 0, st>>>(B);
    else if (B.n > 0 && B.max_bus > 0)
        k_pf_eval_batch<<<dim3((unsigned)blocks_for(B.max_bus, 64), (unsigned)B.n), 64, 0, st>>>(B);
}

void launch_batch_status(const PfBatch& B, double* out, cudaStream_t st) {
    if (B.n > 0) k_batch_status<<<1, 32, 0, st>>>(B, out);
}

void launch_newton_update_batch(const PfBatch& B, cudaStream_t st) {
    if (B.n > 0 && B.max_bus > 0)
        k_newton_update_batch<<<dim3((unsigned)blocks_for(B.max_bus, 128), (unsigned)B.n), 128, 0, st>>>(B);
}

cudaError_t launch_refactor_batch(const RfBatch& B, const int* lev_ptr_host, const int64_t* tgt_lev_ptr_host,
                                  const int* piv_lev_ptr_host, int n_lev, cudaStream_t st) {
    if (B.n <= 0) return cudaSuccess;
    const unsigned n = (unsigned)B.n;
    (void)lev_ptr_host;
    cudaError_t e = cudaSuccess;
    bool pdl = false;   // the first launch follows an event wait
    auto chk = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
        pdl = true;
    };
    if (n_lev > 0 && piv_lev_ptr_host[0] > 0)
        chk(launch_pdl(pdl, k_rf_leaf_piv_batch, dim3((unsigned)blocks_for(piv_lev_ptr_host[0], 128), n), dim3(128), 0, st,
                       B, piv_lev_ptr_host[0]));
    for (int lev = 0; lev < n_lev; lev++) {
        const int64_t t0 = tgt_lev_ptr_host[lev], nt = tgt_lev_ptr_host[lev + 1] - t0;
        const int j0 = piv_lev_ptr_host[lev], njob = piv_lev_ptr_host[lev + 1] - j0;
        if (nt > 0)
            chk(launch_pdl(pdl, k_rf_update_batch, dim3((unsigned)blocks_for(nt, 256), n), dim3(256), 0, st, B, t0, nt, j0,
                           njob));
    }
    const int64_t np = (int64_t)B.g[0].n_piv + B.g[0].n_pe;
    if (np > 0) chk(launch_pdl(pdl, k_rf_pivot_batch, dim3((unsigned)blocks_for(np, 256), n), dim3(256), 0, st, B));
    const int T = B.g[0].T;
    if (T > 0) {
        const int TT = T * T, nt = (T + kTailTB - 1) / kTailTB;
        chk(launch_pdl(pdl, k_tail_gather_batch, dim3((unsigned)blocks_for(TT, 256), n), dim3(256), 0, st, B));
        for (int k = -1; k < nt; k++) {
            const int c = k + 1, U = c < nt ? nt - c - 1 : 0;
            const int grid = 2 * U + (k >= 0 ? 1 + U * U : 0);
            if (grid > 0)
                chk(launch_pdl(pdl, k_tail_step_batch, dim3((unsigned)grid, n), dim3(kTailTB * kTailTB), 0, st, B, k));
        }
        chk(launch_pdl(pdl, k_tail_scatter_batch, dim3((unsigned)blocks_for(TT, 256), n), dim3(256), 0, st, B));
    }
    return e != cudaSuccess ? e : cudaGetLastError();
}

void launch_tail_tri_batch(const TriBatch& B, cudaStream_t st) {
    if (B.n > 0 && B.T > 1)
        k_tail_tri_batch<<<dim3((unsigned)blocks_for((int64_t)B.T * B.T, 256), (unsigned)B.n), 256, 0, st>>>(B);
}

cudaError_t launch_solve1_batch(const Solve1Batch& B, unsigned phases, bool use_tail, int n_x, int T,
                                cudaStream_t st) {
    if (B.n <= 0) return cudaSuccess;
    k_solve1_batch<<<B.n, kSolve1Threads, solve1_smem(n_x, T, use_tail), st>>>(B, phases, use_tail ? 1 : 0);
    return cudaGetLastError();
}

void launch_gather_rows(int n_rows, int N, const int* map, const double* src, int64_t lds, double* dst,
                        int64_t ldd, double scale_x, int n_x, cudaStream_t st) {
    int64_t n = (int64_t)n_rows * N;
    if (n > 0) k_gather_rows<<<blocks_for(n, 256), 256, 0, st>>>(n_rows, N, map, src, lds, dst, ldd, scale_x, n_x);
}

}  // namespace rh

// Whether this build checks indices (-DRH_BOUNDS), and the error word of `device`,
// which the call reads and clears.
extern "C" rh_status rh_bounds_check(int32_t device, int32_t* enabled, uint32_t* errors) {
    if (!enabled || !errors) return RH_EINVAL;
    *errors = 0;
#ifdef RH_BOUNDS
    *enabled = 1;
    if (cudaSetDevice(device) != cudaSuccess) return RH_ECUDA;
    unsigned int e = 0, z = 0;
    if (cudaMemcpyFromSymbol(&e, rh::g_bounds_err, sizeof(e)) != cudaSuccess) return RH_ECUDA;
    if (cudaMemcpyToSymbol(rh::g_bounds_err, &z, sizeof(z)) != cudaSuccess) return RH_ECUDA;
    *errors = e;
#else
    (void)device;
    *enabled = 0;
#endif
    return RH_OK;
}
