// Host check of the refactorisation schedule that the library's symbolic phase
// builds (test infrastructure: compiled and run by tests/test_rf_schedule.py).
//
// Reads a grid (binary: n_bus, n_branch int32; order_level_cost int64; from, to
// int32[n_branch]; r, x, b float64[n_branch]; bus type int8[n_bus]), runs
// build_symbolic with the given dense-tail bound, then emulates on the host, with
// random diagonally dominant values on the pattern of A:
//   (a) every level's updates with each group forming bus k's pivot quantities
//       from k's raw block (two divisions per group);
//   (b) the library's schedule: the leaves' pivot jobs first, every level's
//       updates reading the quantities of its buses, then the level's pivot jobs
//       from its quads (the entries the level updates, the others from A);
//   and then the pivot steps per bus (c) and by entry as the library lists them (d).
// It checks that (a) and (b) give the same factors bit for bit, that (c) and (d)
// do, that every sparse bus has exactly one pivot job, written in a launch before
// any group reads it, that a quad's lane holds only its own block entry, and that
// the quads fit in their level.  Prints one line; exit status 0 when all hold.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_2201_00241_gb300/csrc/rh_internal.h"

namespace {

struct Piv {
    double it = NAN, lvt = NAN, iv = NAN, utv = NAN;
};

// pivot quantities from a block (a_tt, a_tv, a_vt, a_vv) as the library forms them:
// 1/u_tt, l_vt = a_vt / u_tt, 1/u_vv = a_tt / det
Piv block_piv(double att, double atv, double avt, double avv, bool two) {
    Piv p;
    p.it = 1.0 / att;
    p.lvt = 0.0;
    p.iv = 0.0;
    p.utv = 0.0;
    if (two) {
        p.utv = atv;
        p.lvt = avt * p.it;
        p.iv = att * (1.0 / std::fma(att, avv, -(avt * atv)));
    }
    return p;
}

double group(const std::vector<double>& A, const int* g6, const Piv& p, double acc) {
    if (g6[2] < 0) return acc;
    const double lt = A[g6[2]] * p.it;
    const double ut = A[g6[3]];
    if (g6[1] >= 0) {
        const double lv = std::fma(-lt, p.utv, A[g6[4]]) * p.iv;
        const double uv = std::fma(-p.lvt, ut, A[g6[5]]);
        acc = std::fma(lt, ut, acc);
        return std::fma(lv, uv, acc);
    }
    return std::fma(lt, ut, acc);
}

}  // namespace

int main(int argc, char** argv) {
    if (argc < 3) {
        std::fprintf(stderr, "usage: rf_schedule_check grid.bin max_tail\n");
        return 2;
    }
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    int32_t nb = 0, ne = 0;
    int64_t lc = 0;
    bool ok = std::fread(&nb, 4, 1, f) == 1 && std::fread(&ne, 4, 1, f) == 1 && std::fread(&lc, 8, 1, f) == 1;
    std::vector<int32_t> fr(ne), to(ne);
    std::vector<double> r(ne), x(ne), b(ne);
    std::vector<int8_t> ty(nb);
    ok = ok && std::fread(fr.data(), 4, ne, f) == (size_t)ne && std::fread(to.data(), 4, ne, f) == (size_t)ne &&
         std::fread(r.data(), 8, ne, f) == (size_t)ne && std::fread(x.data(), 8, ne, f) == (size_t)ne &&
         std::fread(b.data(), 8, ne, f) == (size_t)ne && std::fread(ty.data(), 1, nb, f) == (size_t)nb;
    std::fclose(f);
    if (!ok) return 2;
    rh::Symbolic S;
    const std::string msg = rh::build_symbolic(nb, ne, fr.data(), to.data(), r.data(), x.data(), b.data(), ty.data(),
                                               lc, S, std::atoi(argv[2]));
    if (!msg.empty()) {
        std::fprintf(stderr, "%s\n", msg.c_str());
        return 2;
    }
    const int nnz = (int)S.col.size(), nsp = S.tail_bus0, nl = S.rf_n_lev;
    std::mt19937_64 rng(7);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    std::vector<double> A0(nnz);
    for (int q = 0; q < S.n_x; q++)
        for (int t = S.rowptr[q]; t < S.rowptr[q + 1]; t++) A0[t] = S.col[t] == q ? 20.0 + U(rng) : U(rng);
    auto raw_piv = [&](const std::vector<double>& A, int k) {
        const int qt = S.q0[k], dt = S.diagpos[qt];
        const bool two = S.nv[k] == 2;
        const int dv = two ? S.diagpos[qt + 1] : -1;
        return block_piv(A[dt], two ? A[dt + 1] : 0.0, two ? A[dv - 1] : 0.0, two ? A[dv] : 0.0, two);
    };

    // (a) per-group form
    std::vector<double> Aa = A0;
    for (int l = 0; l < nl; l++) {
        std::vector<std::pair<int, double>> st;
        for (int64_t t = S.rf_tgt_lev_ptr[l]; t < S.rf_tgt_lev_ptr[l + 1]; t++) {
            const int p = S.rf_tgt_pos[t];
            if (p < 0) continue;
            double acc = 0.0;
            const int* g = &S.rf_grp[6 * t];
            if (g[2] >= 0) acc = group(Aa, g, raw_piv(Aa, g[0]), acc);
            for (int64_t c = S.rf_xptr[t]; c < S.rf_xptr[t + 1]; c++) {
                const int* gx = &S.rf_xgrp[6 * c];
                acc = group(Aa, gx, raw_piv(Aa, gx[0]), acc);
            }
            st.push_back({p, Aa[p] - acc});
        }
        for (auto& e : st) Aa[e.first] = e.second;
    }

    // (b) the schedule with pivot jobs
    std::vector<double> Ab = A0;
    std::vector<Piv> piv(nsp);
    std::vector<int> written(nsp, -2);        // launch that wrote bus k's quantities (-1: leaves)
    long order_errors = 0, lane_errors = 0, fit_errors = 0, repeat = 0;
    for (int q = 0; q < S.rf_piv_lev_ptr[0]; q++) {
        const int* pp = &S.rf_piv_pos[4 * q];
        double v[4];
        for (int e = 0; e < 4; e++) v[e] = pp[e] >= 0 ? Ab[pp[e]] : 0.0;
        const int j = S.rf_piv_bus[q];
        if (written[j] != -2) repeat++;
        piv[j] = block_piv(v[0], v[1], v[2], v[3], pp[3] >= 0);
        written[j] = -1;
    }
    for (int l = 0; l < nl; l++) {
        const int64_t t0 = S.rf_tgt_lev_ptr[l], nt = S.rf_tgt_lev_ptr[l + 1] - t0;
        const int j0 = S.rf_piv_lev_ptr[l], nj = S.rf_piv_lev_ptr[l + 1] - j0;
        if (4LL * nj > nt) fit_errors++;
        std::vector<double> nv(nt, 0.0);
        std::vector<std::pair<int, double>> st;
        for (int64_t tl = 0; tl < nt; tl++) {
            const int p = S.rf_tgt_pos[t0 + tl];
            if (p < 0) continue;
            auto use = [&](const int* g, double acc) {
                if (g[2] < 0) return acc;
                if (written[g[0]] == -2 || written[g[0]] >= l) order_errors++;
                return group(Ab, g, piv[g[0]], acc);
            };
            double acc = use(&S.rf_grp[6 * (t0 + tl)], 0.0);
            for (int64_t c = S.rf_xptr[t0 + tl]; c < S.rf_xptr[t0 + tl + 1]; c++) acc = use(&S.rf_xgrp[6 * c], acc);
            nv[tl] = Ab[p] - acc;
            st.push_back({p, nv[tl]});
        }
        for (auto& e : st) Ab[e.first] = e.second;
        for (int q = 0; q < nj && 4LL * q + 3 < nt; q++) {
            const int* pp = &S.rf_piv_pos[4 * (j0 + q)];
            double v[4];
            for (int e = 0; e < 4; e++) {
                const int p = S.rf_tgt_pos[t0 + 4 * q + e];
                if (p >= 0 && p != pp[e]) lane_errors++;
                v[e] = p >= 0 ? nv[4 * q + e] : (pp[e] >= 0 ? Ab[pp[e]] : 0.0);
            }
            const int j = S.rf_piv_bus[j0 + q];
            if (written[j] != -2) repeat++;
            piv[j] = block_piv(v[0], v[1], v[2], v[3], pp[3] >= 0);
            written[j] = l;
        }
    }
    long missing = 0, diff = 0;
    for (int j = 0; j < nsp; j++)
        if (written[j] == -2) missing++;
    for (int i = 0; i < nnz; i++)
        if (std::memcmp(&Aa[i], &Ab[i], sizeof(double)) != 0) diff++;

    // (c) pivot steps per bus against (d) the library's by-entry list
    std::vector<double> Pc = Ab, Pd = Ab;
    for (int k = 0; k < nsp; k++) {
        const int qt = S.q0[k], dt = S.diagpos[qt];
        const bool two = S.nv[k] == 2;
        const Piv p = raw_piv(Pc, k);
        int dv = 0;
        if (two) {
            dv = S.diagpos[qt + 1];
            const double uvv = std::fma(-p.lvt, p.utv, Pc[dv]);
            Pc[dv - 1] = p.lvt;
            Pc[dv] = uvv;
        }
        const int ut0 = dt + (two ? 2 : 1), uv0 = dv + 1, n = S.rowptr[qt + 1] - ut0;
        for (int e = 0; e < n; e++) {
            if (two) Pc[uv0 + e] = std::fma(-p.lvt, Pc[ut0 + e], Pc[uv0 + e]);
            const int pt = S.tpos[ut0 + e];
            const double lt = Pc[pt] * p.it;
            Pc[pt] = lt;
            if (two) {
                const int pv = S.tpos[uv0 + e];
                Pc[pv] = std::fma(-lt, p.utv, Pc[pv]) * p.iv;
            }
        }
    }
    for (int k = 0; k < nsp; k++) {
        if (S.nv[k] != 2) continue;
        const int dv = S.diagpos[S.q0[k] + 1];
        const double uvv = std::fma(-piv[k].lvt, piv[k].utv, Pd[dv]);
        Pd[dv - 1] = piv[k].lvt;
        Pd[dv] = uvv;
    }
    for (size_t e = 0; e < S.rf_pe_bus.size(); e++) {
        const Piv& p = piv[S.rf_pe_bus[e]];
        const int* pos = &S.rf_pe_ut[4 * e];
        const double lt = Pd[pos[2]] * p.it;
        Pd[pos[2]] = lt;
        if (pos[1] >= 0) {
            Pd[pos[1]] = std::fma(-p.lvt, Pd[pos[0]], Pd[pos[1]]);
            Pd[pos[3]] = std::fma(-lt, p.utv, Pd[pos[3]]) * p.iv;
        }
    }
    long pdiff = 0;
    for (int i = 0; i < nnz; i++)
        if (std::memcmp(&Pc[i], &Pd[i], sizeof(double)) != 0) pdiff++;

    std::printf("levels=%d sparse_buses=%d tail_vars=%d targets=%lld missing=%ld repeated=%ld order_errors=%ld "
                "lane_errors=%ld fit_errors=%ld diff_updates=%ld diff_pivot_steps=%ld\n",
                nl, nsp, S.n_x - S.t0, (long long)S.rf_tgt_pos.size(), missing, repeat, order_errors, lane_errors,
                fit_errors, diff, pdiff);
    return (missing || repeat || order_errors || lane_errors || fit_errors || diff || pdiff) ? 1 : 0;
}
