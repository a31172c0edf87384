// symbolic.cpp -- host symbolic phase of librh (once per topology).
//
// The paper factors J_x once on the host and hands the fixed pattern to a
// device refactorisation (section 5.2).  Here the host does only the symbolic
// work: admittance pattern, a static fill-reducing order, the pattern of
// L + U, the bus-level schedules and the index maps used by the kernels.
// Numerical work (Jacobian values, LU values, solves) runs on the device.
#include <algorithm>
#include <array>
#include <cmath>
#include <functional>
#include <queue>
#include <tuple>
#include <utility>

#include "rh_internal.h"

namespace rh {
namespace {

// Exact minimum degree on the bus graph: repeatedly eliminate the remaining
// bus of smallest degree in the current elimination graph (ties: smallest bus
// id); the neighbours of an eliminated bus become a clique.  Adjacency lists
// are kept sorted; a min-heap with lazy invalidation finds the next bus.
// colpat_bus[k] receives the neighbour set (bus ids) of the k-th eliminated bus.
void minimum_degree(int n_bus, const std::vector<std::vector<int>>& adj0, const std::vector<char>& active,
                    std::vector<int>& order, std::vector<std::vector<int>>& colpat_bus) {
    std::vector<std::vector<int>> adj = adj0;
    std::vector<char> alive = active;
    using Key = std::pair<int, int>;  // (degree, bus id)
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
    for (int i = 0; i < n_bus; i++)
        if (alive[i]) heap.push({(int)adj[i].size(), i});
    std::vector<int> merged;
    while (!heap.empty()) {
        auto [d, e] = heap.top();
        heap.pop();
        if (!alive[e] || d != (int)adj[e].size()) continue;  // stale entry
        alive[e] = 0;
        std::vector<int> nb = std::move(adj[e]);
        adj[e].clear();
        for (int a : nb) {
            // adj[a] <- (adj[a] U nb) \ {a, e}
            merged.clear();
            std::set_union(adj[a].begin(), adj[a].end(), nb.begin(), nb.end(), std::back_inserter(merged));
            adj[a].clear();
            for (int v : merged)
                if (v != a && v != e) adj[a].push_back(v);
            heap.push({(int)adj[a].size(), a});
        }
        order.push_back(e);
        colpat_bus.push_back(std::move(nb));
    }
}

// Cost of an elimination order for choosing between the two orders below: the
// factor entries outside the bus blocks (sum over buses of w_k times the weight
// of the neighbours it has when eliminated) times the directions of a full
// reduced Hessian, plus level_cost per forward level (each level of the four
// direction sweeps costs a barrier and a chain of dependent loads; the caller
// passes what one level costs in entry-direction FMAs).
int64_t order_cost(int n_bus, const std::vector<int>& order, const std::vector<std::vector<int>>& colpat_bus,
                   const std::vector<int>& w, int64_t n_dirs, int64_t level_cost) {
    std::vector<int> pos(n_bus, -1), lev(order.size(), 0);
    for (size_t k = 0; k < order.size(); k++) pos[order[k]] = (int)k;
    int64_t entries = 0;
    int n_lev = 0;
    for (size_t k = 0; k < order.size(); k++) {
        int64_t s = 0;
        for (int c : colpat_bus[k]) {
            s += w[c];
            lev[pos[c]] = std::max(lev[pos[c]], lev[k] + 1);
        }
        entries += (int64_t)w[order[k]] * s;
        n_lev = std::max(n_lev, lev[k] + 1);
    }
    return entries * n_dirs + level_cost * n_lev;
}

// Minimum weighted fill on the bus graph.  Eliminating bus e joins its remaining
// neighbours into a clique: every pair (a, b) of them that is not yet adjacent
// adds w_a * w_b entries to L (and as many to U), w = variables per bus (1 for a
// PV bus, 2 for a PQ bus).  Repeatedly eliminate the bus that adds the fewest
// (ties: the smallest weighted degree, i.e. sum of w over its remaining
// neighbours, then the smallest bus id).  An elimination changes the score of
// the buses within two steps of it only; those are rescored and pushed again on
// a min-heap with lazy invalidation.  Adjacency lists are kept sorted.
// colpat_bus[k] receives the neighbour set (bus ids) of the k-th eliminated bus.
void minimum_fill(int n_bus, const std::vector<std::vector<int>>& adj0, const std::vector<char>& active,
                  const std::vector<int>& w, std::vector<int>& order, std::vector<std::vector<int>>& colpat_bus) {
    std::vector<std::vector<int>> adj = adj0;
    std::vector<char> alive = active;
    std::vector<int> mark(n_bus, -1);
    int stamp = 0;
    using Key = std::tuple<int64_t, int64_t, int>;   // (weighted fill, weighted degree, bus id)
    auto key = [&](int v) {
        stamp++;
        int64_t sw = 0, sw2 = 0, adj2 = 0;
        for (int c : adj[v]) {
            mark[c] = stamp;
            sw += w[c];
            sw2 += (int64_t)w[c] * w[c];
        }
        for (int a : adj[v])
            for (int c : adj[a])
                if (mark[c] == stamp) adj2 += (int64_t)w[a] * w[c];   // each adjacent pair twice
        return Key{(sw * sw - sw2) / 2 - adj2 / 2, sw, v};
    };
    std::vector<Key> cur(n_bus);
    std::priority_queue<Key, std::vector<Key>, std::greater<Key>> heap;
    for (int i = 0; i < n_bus; i++)
        if (alive[i]) heap.push(cur[i] = key(i));
    std::vector<int> merged, touched;
    std::vector<int> seen(n_bus, -1);
    while (!heap.empty()) {
        const Key k = heap.top();
        heap.pop();
        const int e = std::get<2>(k);
        if (!alive[e] || k != cur[e]) continue;  // stale entry
        alive[e] = 0;
        std::vector<int> nb = std::move(adj[e]);
        adj[e].clear();
        for (int a : nb) {
            // adj[a] <- (adj[a] U nb) \ {a, e}
            merged.clear();
            std::set_union(adj[a].begin(), adj[a].end(), nb.begin(), nb.end(), std::back_inserter(merged));
            adj[a].clear();
            for (int v : merged)
                if (v != a && v != e) adj[a].push_back(v);
        }
        // rescore the buses within two steps of e
        touched.clear();
        for (int a : nb) {
            if (seen[a] != e) { seen[a] = e; touched.push_back(a); }
            for (int c : adj[a])
                if (seen[c] != e) { seen[c] = e; touched.push_back(c); }
        }
        for (int v : touched)
            if (alive[v]) heap.push(cur[v] = key(v));
        order.push_back(e);
        colpat_bus.push_back(std::move(nb));
    }
}

int find_in_row(const std::vector<int>& rowptr, const std::vector<int>& col, int row, int c) {
    auto b = col.begin() + rowptr[row], e = col.begin() + rowptr[row + 1];
    auto it = std::lower_bound(b, e, c);
    if (it == e || *it != c) return -1;
    return (int)(it - col.begin());
}

// Greedy column colouring from row -> column lists: columns in ascending
// order, each taking the smallest colour that no earlier column sharing one of
// its rows holds.  Returns the number of colours.
int greedy_columns(int n_cols, const std::vector<std::vector<int>>& row_cols, std::vector<int>& colour) {
    std::vector<std::vector<int>> col_rows(n_cols);
    for (int r = 0; r < (int)row_cols.size(); r++)
        for (int c : row_cols[r]) col_rows[c].push_back(r);
    colour.assign(n_cols, -1);
    std::vector<int> stamp(n_cols + 1, -1);
    int n_colours = 0;
    for (int c = 0; c < n_cols; c++) {
        for (int r : col_rows[c])
            for (int d : row_cols[r])
                if (d < c) stamp[colour[d]] = c;
        int k = 0;
        while (stamp[k] == c) k++;
        colour[c] = k;
        n_colours = std::max(n_colours, k + 1);
    }
    return n_colours;
}

}  // namespace

std::string build_symbolic(int n_bus, int n_branch, const int32_t* fr, const int32_t* to,
                           const double* r, const double* x, const double* b,
                           const int8_t* type, int64_t level_cost, Symbolic& S, int max_tail) {
    if (n_bus < 1 || n_branch < 0) return "n_bus must be >= 1 and n_branch >= 0";
    if (level_cost < 0) return "order_level_cost must be >= 0";
    S.n_bus = n_bus;
    S.n_branch = n_branch;
    int n_ref = 0;
    for (int i = 0; i < n_bus; i++) {
        if (type[i] != kRef && type[i] != kPV && type[i] != kPQ) return "bus_type must be 0, 1 or 2";
        if (type[i] == kRef) { n_ref++; S.ref = i; }
        if (type[i] == kPV) S.n_pv++;
        if (type[i] == kPQ) S.n_pq++;
    }
    if (n_ref != 1) return "the grid needs exactly one slack bus (bus_type 0)";
    S.n_gen = 1 + S.n_pv;
    S.n_x = S.n_pv + 2 * S.n_pq;
    S.n_p = 2 * S.n_gen - 1;

    // ---- admittance matrix (pi model) -------------------------------------
    std::vector<std::vector<std::tuple<int, double, double>>> yrow(n_bus);
    std::vector<double> gd(n_bus, 0.0), bd(n_bus, 0.0);
    for (int e = 0; e < n_branch; e++) {
        int i = fr[e], j = to[e];
        if (i < 0 || j < 0 || i >= n_bus || j >= n_bus || i == j) return "branch with a bad or repeated end bus";
        double den = r[e] * r[e] + x[e] * x[e];
        if (!(den > 0.0) || !std::isfinite(den)) return "branch with zero or non-finite impedance";
        double gs = r[e] / den, bs = -x[e] / den;
        gd[i] += gs; bd[i] += bs + 0.5 * b[e];
        gd[j] += gs; bd[j] += bs + 0.5 * b[e];
        yrow[i].emplace_back(j, -gs, -bs);
        yrow[j].emplace_back(i, -gs, -bs);
    }
    S.yp.assign(n_bus + 1, 0);
    S.ydiag.assign(n_bus, -1);
    for (int i = 0; i < n_bus; i++) {
        auto& rw = yrow[i];
        rw.emplace_back(i, gd[i], bd[i]);
        std::sort(rw.begin(), rw.end(), [](auto& a, auto& c) { return std::get<0>(a) < std::get<0>(c); });
        for (size_t k = 0; k < rw.size(); k++) {
            int j = std::get<0>(rw[k]);
            if (!S.yj.empty() && (int)S.yj.size() > S.yp[i] && S.yj.back() == j) {
                S.G.back() += std::get<1>(rw[k]);
                S.B.back() += std::get<2>(rw[k]);
            } else {
                if (j == i) S.ydiag[i] = (int)S.yj.size();
                S.yj.push_back(j);
                S.G.push_back(std::get<1>(rw[k]));
                S.B.push_back(std::get<2>(rw[k]));
            }
        }
        S.yp[i + 1] = (int)S.yj.size();
    }

    // ---- external index maps ------------------------------------------------
    S.ix_th.assign(n_bus, -1); S.ix_v.assign(n_bus, -1); S.ip_v.assign(n_bus, -1); S.ip_pg.assign(n_bus, -1);
    {
        int kpv = 0, kpq = 0, kg = 0;
        for (int i = 0; i < n_bus; i++) {
            if (type[i] == kPV) { S.ix_th[i] = kpv; S.ip_pg[i] = S.n_gen + kpv; kpv++; }
            if (type[i] == kPQ) { S.ix_th[i] = S.n_pv + kpq; S.ix_v[i] = S.n_pv + S.n_pq + kpq; kpq++; }
            if (type[i] != kPQ) S.ip_v[i] = kg++;
        }
    }

    // ---- ordering -------------------------------------------------------------
    std::vector<std::vector<int>> adj(n_bus);
    std::vector<char> active(n_bus, 0);
    for (int i = 0; i < n_bus; i++) active[i] = type[i] != kRef;
    for (int i = 0; i < n_bus; i++) {
        if (!active[i]) continue;
        for (int s = S.yp[i]; s < S.yp[i + 1]; s++) {
            int j = S.yj[s];
            if (j != i && active[j]) adj[i].push_back(j);   // yj is sorted and unique
        }
    }
    // Two candidate orders: exact minimum degree (fewer levels on small grids) and
    // minimum weighted fill (fewer factor entries); the cheaper by order_cost wins
    // (ties: minimum degree).
    std::vector<int> wbus(n_bus);
    for (int i = 0; i < n_bus; i++) wbus[i] = type[i] == kPQ ? 2 : 1;
    std::vector<int> order_md, order_mf;
    std::vector<std::vector<int>> colpat_md, colpat_mf;
    minimum_degree(n_bus, adj, active, order_md, colpat_md);
    minimum_fill(n_bus, adj, active, wbus, order_mf, colpat_mf);
    const int64_t n_dirs = S.n_p;
    const bool mf = order_cost(n_bus, order_mf, colpat_mf, wbus, n_dirs, level_cost) <
                    order_cost(n_bus, order_md, colpat_md, wbus, n_dirs, level_cost);
    S.order_mf = mf;
    S.ebus = mf ? std::move(order_mf) : std::move(order_md);
    std::vector<std::vector<int>> colpat_bus = mf ? std::move(colpat_mf) : std::move(colpat_md);
    S.n_elim = (int)S.ebus.size();
    S.epos.assign(n_bus, -1);
    for (int k = 0; k < S.n_elim; k++) S.epos[S.ebus[k]] = k;
    S.q0.assign(S.n_elim, 0);
    S.nv.assign(S.n_elim, 1);
    S.qth.assign(n_bus, -1);
    S.qv.assign(n_bus, -1);
    S.perm.assign(S.n_x, -1);
    {
        int q = 0;
        for (int k = 0; k < S.n_elim; k++) {
            int bus = S.ebus[k];
            S.q0[k] = q;
            S.qth[bus] = q;
            S.perm[q++] = S.ix_th[bus];
            if (type[bus] == kPQ) {
                S.nv[k] = 2;
                S.qv[bus] = q;
                S.perm[q++] = S.ix_v[bus];
            }
        }
    }

    // ---- bus-level patterns and levels ----------------------------------------
    S.colpat.assign(S.n_elim, {});
    S.rowpat.assign(S.n_elim, {});
    for (int k = 0; k < S.n_elim; k++) {
        for (int bus : colpat_bus[k]) S.colpat[k].push_back(S.epos[bus]);
        std::sort(S.colpat[k].begin(), S.colpat[k].end());
        for (int c : S.colpat[k]) S.rowpat[c].push_back(k);        // k ascending -> sorted
    }
    // Forward level: the height of the bus above the leaves of the elimination tree.
    // Backward level: the same height counted from the top (a bus comes after all
    // its ancestors, whose heights are larger).  Levels by height hold buses of
    // equal height, whose rows have similar lengths, and both sweeps get the same
    // number of levels; levels by depth from the root mixed leaves with interior
    // buses (94 against 74 sparse levels on the 9241-bus grid, lanes 86 % against
    // 94 % busy, in a host count of the direction kernel's FP64 instructions).
    S.flevel.assign(S.n_elim, 0);
    S.blevel.assign(S.n_elim, 0);
    int h_max = 0;
    for (int k = 0; k < S.n_elim; k++) {
        for (int c : S.rowpat[k]) S.flevel[k] = std::max(S.flevel[k], S.flevel[c] + 1);
        h_max = std::max(h_max, S.flevel[k]);
    }
    for (int k = 0; k < S.n_elim; k++) S.blevel[k] = h_max - S.flevel[k];
    auto ext_len = [&](const std::vector<int>& pat) {
        int n = 0;
        for (int c : pat) n += S.nv[c];
        return n;
    };
    auto group = [&](const std::vector<int>& lev, const std::vector<std::vector<int>>& pat, int& nlev,
                     std::vector<int>& ptr, std::vector<int>& bus, std::vector<int>& maxext) {
        nlev = 0;
        for (int k = 0; k < S.n_elim; k++) nlev = std::max(nlev, lev[k] + 1);
        ptr.assign(nlev + 1, 0);
        maxext.assign(nlev, 0);
        for (int k = 0; k < S.n_elim; k++) ptr[lev[k] + 1]++;
        for (int l = 0; l < nlev; l++) ptr[l + 1] += ptr[l];
        bus.assign(S.n_elim, 0);
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (int k = 0; k < S.n_elim; k++) bus[fill[lev[k]]++] = k;
        // within a level: PQ buses first, then longer rows first (balance, less divergence)
        for (int l = 0; l < nlev; l++) {
            std::stable_sort(bus.begin() + ptr[l], bus.begin() + ptr[l + 1], [&](int a, int c) {
                int la = ext_len(pat[a]), lc = ext_len(pat[c]);
                if (S.nv[a] != S.nv[c]) return S.nv[a] > S.nv[c];
                return la > lc;
            });
            for (int t = ptr[l]; t < ptr[l + 1]; t++) maxext[l] = std::max(maxext[l], ext_len(pat[bus[t]]));
        }
    };
    group(S.flevel, S.rowpat, S.n_flev, S.flev_ptr, S.flev_bus, S.flev_maxext);
    group(S.blevel, S.colpat, S.n_blev, S.blev_ptr, S.blev_bus, S.blev_maxext);

    // ---- variable-level CSR of A = L + U -------------------------------------
    S.rowptr.assign(S.n_x + 1, 0);
    S.diagpos.assign(S.n_x, 0);
    for (int k = 0; k < S.n_elim; k++) {
        for (int t = 0; t < S.nv[k]; t++) {
            int q = S.q0[k] + t;
            S.rowptr[q] = (int)S.col.size();
            for (int c : S.rowpat[k])
                for (int u = 0; u < S.nv[c]; u++) S.col.push_back(S.q0[c] + u);
            if (t == 1) S.col.push_back(S.q0[k]);                 // (v, theta) of the bus
            S.diagpos[q] = (int)S.col.size();
            S.col.push_back(q);
            if (t == 0 && S.nv[k] == 2) S.col.push_back(q + 1);   // (theta, v) of the bus
            for (int c : S.colpat[k])
                for (int u = 0; u < S.nv[c]; u++) S.col.push_back(S.q0[c] + u);
        }
    }
    S.rowptr[S.n_x] = (int)S.col.size();
    S.nnz_l = 0;
    for (int q = 0; q < S.n_x; q++) S.nnz_l += S.diagpos[q] - S.rowptr[q];
    S.nnz_u = (int64_t)S.col.size() - S.nnz_l;
    S.tpos.assign(S.col.size(), -1);
    for (int q = 0; q < S.n_x; q++)
        for (int s = S.rowptr[q]; s < S.rowptr[q + 1]; s++) {
            int t = find_in_row(S.rowptr, S.col, S.col[s], q);
            if (t < 0) return "internal error: pattern of L + U is not symmetric";
            S.tpos[s] = t;
        }

    // ---- refactorisation schedule -------------------------------------------
    // default bound: the top separator of a near-planar grid has about sqrt(n_x)
    // variables; rounded to the 16-column tiles of the tail's LU (at least one tile)
    if (max_tail <= 0) max_tail = 16 * std::max(1, (int)std::lround(std::sqrt((double)S.n_x) / 16.0));
    S.max_tail = max_tail;
    S.tail_bus0 = S.n_elim;
    while (S.tail_bus0 > 0 && S.n_x - S.q0[S.tail_bus0 - 1] <= max_tail) S.tail_bus0--;
    S.t0 = S.tail_bus0 < S.n_elim ? S.q0[S.tail_bus0] : S.n_x;
    {
        std::vector<std::vector<int>> by_lev(S.n_flev);
        for (int t = 0; t < S.n_elim; t++) {
            int k = S.flev_bus[t];
            if (k < S.tail_bus0) by_lev[S.flevel[k]].push_back(k);
        }
        S.rf_lev_ptr.assign(1, 0);
        S.rf_lev_bus.clear();
        S.rf_tgt_lev_ptr.assign(1, 0);
        S.rf_tgt_gptr.assign(1, 0);
        S.rf_grp.clear();
        S.rf_updates = 0;
        // (target, bus order, {dt, dv, lt, ut, lv, uv}): one group per target and bus
        using Grp = std::tuple<int, int, std::array<int, 6>>;
        std::vector<Grp> grp;
        for (auto& v : by_lev) {
            if (v.empty()) continue;
            grp.clear();
            int order = 0;
            for (int k : v) {
                S.rf_lev_bus.push_back(k);
                int qt = S.q0[k];
                bool two = S.nv[k] == 2;
                int dt = S.diagpos[qt], dv = two ? S.diagpos[qt + 1] : -1;
                int ut0 = dt + (two ? 2 : 1);
                int uv0 = two ? dv + 1 : -1;
                int n = S.rowptr[qt + 1] - ut0;
                for (int a = 0; a < n; a++) {
                    int i = S.col[ut0 + a];
                    int lt = S.tpos[ut0 + a], lv = two ? S.tpos[uv0 + a] : -1;
                    for (int bb = 0; bb < n; bb++) {
                        int j = S.col[ut0 + bb];
                        int tg = find_in_row(S.rowptr, S.col, i, j);
                        if (tg < 0) return "internal error: fill pattern not closed";
                        grp.emplace_back(tg, order, std::array<int, 6>{k, dv, lt, ut0 + bb, lv, two ? uv0 + bb : -1});
                        S.rf_updates += two ? 2 : 1;
                    }
                }
                order++;
            }
            std::sort(grp.begin(), grp.end(),
                      [](const Grp& x, const Grp& y) { return std::tie(std::get<0>(x), std::get<1>(x)) <
                                                             std::tie(std::get<0>(y), std::get<1>(y)); });
            for (size_t t = 0; t < grp.size(); t++) {
                int tg = std::get<0>(grp[t]);
                if (t == 0 || std::get<0>(grp[t - 1]) != tg) {
                    if (t > 0) S.rf_tgt_gptr.push_back((int64_t)(S.rf_grp.size() / 6));
                    S.rf_tgt_pos.push_back(tg);
                }
                for (int x : std::get<2>(grp[t])) S.rf_grp.push_back(x);
            }
            if (!grp.empty()) S.rf_tgt_gptr.push_back((int64_t)(S.rf_grp.size() / 6));
            S.rf_lev_ptr.push_back((int)S.rf_lev_bus.size());
            S.rf_tgt_lev_ptr.push_back((int64_t)S.rf_tgt_pos.size());
        }
        S.rf_n_lev = (int)S.rf_lev_ptr.size() - 1;

        // Pivot jobs.  The pivot quantities of sparse bus j (1/u_tt, l_vt, 1/u_vv, u_tv)
        // depend on its 2x2 block only, which is final after the last level that
        // updates it (m_j).  Level m_j computes them right after its updates: the
        // block's four entries sit in four adjacent lanes at the front of the level (a
        // quad; entries the level does not update are read from A), and the quad's
        // first lane stores them.  The leaves (no update: m_j = -1) are computed by a
        // launch of their own before the first level.  Every level then reads them
        // instead of forming them from the block with two divisions.
        const int n_sp = S.tail_bus0;
        std::vector<int> pos_job(S.col.size(), -1);              // position -> 4 * bus + entry
        for (int j = 0; j < n_sp; j++) {
            const int qt = S.q0[j], dt = S.diagpos[qt];
            pos_job[dt] = 4 * j;
            if (S.nv[j] == 2) {
                const int dv = S.diagpos[qt + 1];
                pos_job[dt + 1] = 4 * j + 1;
                pos_job[dv - 1] = 4 * j + 2;
                pos_job[dv] = 4 * j + 3;
            }
        }
        std::vector<int> mj(n_sp, -1);
        for (int l = 0; l < S.rf_n_lev; l++)
            for (int64_t t = S.rf_tgt_lev_ptr[l]; t < S.rf_tgt_lev_ptr[l + 1]; t++) {
                const int pj = pos_job[S.rf_tgt_pos[t]];
                if (pj >= 0) mj[pj / 4] = l;
            }
        // new target order per level: the quads, then the other targets in position order
        std::vector<int> npos;
        std::vector<int> ngrp, nxgrp;
        std::vector<int64_t> nlev(1, 0), nxptr(1, 0);
        S.rf_piv_bus.clear();
        S.rf_piv_pos.clear();
        auto add_job = [&](int j) {
            const int qt = S.q0[j], dt = S.diagpos[qt];
            const bool two = S.nv[j] == 2;
            const int dv = two ? S.diagpos[qt + 1] : -1;
            S.rf_piv_bus.push_back(j);
            for (int e : {dt, two ? dt + 1 : -1, two ? dv - 1 : -1, dv}) S.rf_piv_pos.push_back(e);
        };
        std::vector<std::vector<int>> jobs(S.rf_n_lev);
        for (int j = 0; j < n_sp; j++) {
            if (mj[j] >= 0) jobs[mj[j]].push_back(j);
            else add_job(j);                                  // leaves first
        }
        S.rf_piv_lev_ptr.assign(1, (int)S.rf_piv_bus.size());
        auto put = [&](int64_t t) {            // target t of the old order (-1: an empty lane)
            npos.push_back(t < 0 ? -1 : S.rf_tgt_pos[t]);
            const int64_t g0 = t < 0 ? 0 : S.rf_tgt_gptr[t], g1 = t < 0 ? 0 : S.rf_tgt_gptr[t + 1];
            for (int x = 0; x < 6; x++) ngrp.push_back(g1 > g0 ? S.rf_grp[6 * g0 + x] : -1);
            for (int64_t c = g0 + 1; c < g1; c++)
                for (int x = 0; x < 6; x++) nxgrp.push_back(S.rf_grp[6 * c + x]);
            nxptr.push_back((int64_t)(nxgrp.size() / 6));
        };
        for (int l = 0; l < S.rf_n_lev; l++) {
            const int64_t a = S.rf_tgt_lev_ptr[l], b = S.rf_tgt_lev_ptr[l + 1];
            std::vector<int64_t> lane(4 * jobs[l].size(), -1);
            std::vector<char> in_quad(b - a, 0);
            for (int64_t t = a; t < b; t++) {
                const int pj = pos_job[S.rf_tgt_pos[t]];
                if (pj < 0 || mj[pj / 4] != l) continue;
                const int64_t q = std::lower_bound(jobs[l].begin(), jobs[l].end(), pj / 4) - jobs[l].begin();
                lane[4 * q + pj % 4] = t;
                in_quad[t - a] = 1;
            }
            for (size_t q = 0; q < jobs[l].size(); q++) {
                add_job(jobs[l][q]);
                for (int e = 0; e < 4; e++) put(lane[4 * q + e]);
            }
            for (int64_t t = a; t < b; t++)
                if (!in_quad[t - a]) put(t);
            nlev.push_back((int64_t)npos.size());
            S.rf_piv_lev_ptr.push_back((int)S.rf_piv_bus.size());
        }
        S.rf_tgt_pos.swap(npos);
        S.rf_grp.swap(ngrp);
        S.rf_xgrp.swap(nxgrp);
        S.rf_xptr.swap(nxptr);
        S.rf_tgt_lev_ptr.swap(nlev);
        S.rf_tgt_gptr.clear();

        // Pivot steps, one thread per sparse bus (its block: l_vt, u_vv, 1/u_kk) and one
        // per entry of its U rows right of the block (u_vj, and l_jt, l_jv through the
        // transposed positions)
        S.rf_pe_ut.clear();
        S.rf_pe_bus.clear();
        for (int j = 0; j < n_sp; j++) {
            const int qt = S.q0[j], dt = S.diagpos[qt];
            const bool two = S.nv[j] == 2;
            const int ut0 = dt + (two ? 2 : 1), n = S.rowptr[qt + 1] - ut0;
            const int uv0 = two ? S.diagpos[qt + 1] + 1 : -1;
            for (int e = 0; e < n; e++) {
                S.rf_pe_bus.push_back(j);
                S.rf_pe_ut.push_back(ut0 + e);
                S.rf_pe_ut.push_back(two ? uv0 + e : -1);
                S.rf_pe_ut.push_back(S.tpos[ut0 + e]);
                S.rf_pe_ut.push_back(two ? S.tpos[uv0 + e] : -1);
            }
        }
    }

    // ---- J_p pattern and the assembly destinations -------------------------
    std::vector<std::vector<int>> jprow(S.n_x);
    for (int i = 0; i < n_bus; i++) {
        int rows[2] = {S.qth[i], S.qv[i]};
        for (int s = S.yp[i]; s < S.yp[i + 1]; s++) {
            int j = S.yj[s];
            if (S.qv[j] >= 0) continue;                       // v_j in x
            for (int rr : rows)
                if (rr >= 0) jprow[rr].push_back(S.ip_v[j]);
        }
        if (S.ip_pg[i] >= 0) jprow[S.qth[i]].push_back(S.ip_pg[i]);
    }
    S.jp_ptr.assign(S.n_x + 1, 0);
    for (int q = 0; q < S.n_x; q++) {
        std::sort(jprow[q].begin(), jprow[q].end());
        jprow[q].erase(std::unique(jprow[q].begin(), jprow[q].end()), jprow[q].end());
        for (int c : jprow[q]) S.jp_col.push_back(c);
        S.jp_ptr[q + 1] = (int)S.jp_col.size();
    }
    auto jp_slot = [&](int row, int pc) { return find_in_row(S.jp_ptr, S.jp_col, row, pc); };
    S.jac_dst.assign(4 * S.yj.size(), -1);
    S.nnz_jx = 0;
    for (int i = 0; i < n_bus; i++) {
        int rP = S.qth[i], rQ = S.qv[i];
        for (int s = S.yp[i]; s < S.yp[i + 1]; s++) {
            int j = S.yj[s];
            int cth = S.qth[j];
            int rows[2] = {rP, rQ};
            for (int a = 0; a < 2; a++) {
                int rr = rows[a];
                if (rr < 0) continue;
                if (cth >= 0) {
                    int t = find_in_row(S.rowptr, S.col, rr, cth);
                    if (t < 0) return "internal error: J_x entry outside the LU pattern";
                    S.jac_dst[4 * s + 2 * a + 0] = t;
                    S.nnz_jx++;
                }
                if (S.qv[j] >= 0) {
                    int t = find_in_row(S.rowptr, S.col, rr, S.qv[j]);
                    if (t < 0) return "internal error: J_x entry outside the LU pattern";
                    S.jac_dst[4 * s + 2 * a + 1] = t;
                    S.nnz_jx++;
                } else {
                    int t = jp_slot(rr, S.ip_v[j]);
                    if (t < 0) return "internal error: J_p entry missing";
                    S.jac_dst[4 * s + 2 * a + 1] = -(t + 2);
                }
            }
        }
    }
    S.pg_slot.assign(n_bus, -1);
    for (int i = 0; i < n_bus; i++)
        if (S.ip_pg[i] >= 0) S.pg_slot[i] = jp_slot(S.qth[i], S.ip_pg[i]);
    // ---- column colouring of J_x and J_p (coloured forward-mode AD) --------
    {
        std::vector<std::vector<int>> xrows(S.n_x), prows(S.n_x);   // row (x index) -> columns
        for (int i = 0; i < n_bus; i++) {
            int rows[2] = {S.qth[i], S.qv[i]};
            for (int a = 0; a < 2; a++) {
                if (rows[a] < 0) continue;
                int r = S.perm[rows[a]];
                for (int s = S.yp[i]; s < S.yp[i + 1]; s++) {
                    int j = S.yj[s];
                    if (S.qth[j] >= 0) xrows[r].push_back(S.perm[S.qth[j]]);
                    if (S.qv[j] >= 0) xrows[r].push_back(S.perm[S.qv[j]]);
                    else if (S.ip_v[j] >= 0) prows[r].push_back(S.ip_v[j]);
                }
                if (a == 0 && S.ip_pg[i] >= 0) prows[r].push_back(S.ip_pg[i]);
            }
        }
        S.n_colors_x = greedy_columns(S.n_x, xrows, S.colors_x);
        S.n_colors_p = greedy_columns(S.n_p, prows, S.colors_p);
        S.col_th.assign(n_bus, -1);
        S.col_v.assign(n_bus, -1);
        S.col_pg.assign(n_bus, -1);
        for (int j = 0; j < n_bus; j++) {
            if (S.qth[j] >= 0) S.col_th[j] = S.colors_x[S.perm[S.qth[j]]];
            if (S.qv[j] >= 0) S.col_v[j] = S.colors_x[S.perm[S.qv[j]]];
            else if (S.ip_v[j] >= 0) S.col_v[j] = S.n_colors_x + S.colors_p[S.ip_v[j]];
            if (S.ip_pg[j] >= 0) S.col_pg[j] = S.n_colors_x + S.colors_p[S.ip_pg[j]];
        }
        // structural J_x entries for export, sorted by (row, column) in x indices
        std::vector<std::tuple<int, int, int>> e;
        e.reserve((size_t)S.nnz_jx);
        for (int i = 0; i < n_bus; i++) {
            int rows[2] = {S.qth[i], S.qv[i]};
            for (int s = S.yp[i]; s < S.yp[i + 1]; s++) {
                int j = S.yj[s];
                for (int a = 0; a < 2; a++)
                    for (int u = 0; u < 2; u++) {
                        int dst = S.jac_dst[4 * s + 2 * a + u];
                        int cq = u == 0 ? S.qth[j] : S.qv[j];
                        if (dst >= 0) e.emplace_back(S.perm[rows[a]], S.perm[cq], dst);
                    }
            }
        }
        std::sort(e.begin(), e.end());
        S.jx_row.resize(e.size());
        S.jx_col.resize(e.size());
        S.jx_slot.resize(e.size());
        for (size_t k = 0; k < e.size(); k++) {
            S.jx_row[k] = std::get<0>(e[k]);
            S.jx_col[k] = std::get<1>(e[k]);
            S.jx_slot[k] = std::get<2>(e[k]);
        }
        S.jp_xrow.resize(S.n_x);
        for (int q = 0; q < S.n_x; q++) S.jp_xrow[q] = S.perm[q];
    }
    // transpose of J_p: rows = p index
    S.jpt_ptr.assign(S.n_p + 1, 0);
    for (int c : S.jp_col) S.jpt_ptr[c + 1]++;
    for (int k = 0; k < S.n_p; k++) S.jpt_ptr[k + 1] += S.jpt_ptr[k];
    S.jpt_row.assign(S.jp_col.size(), 0);
    S.jpt_src.assign(S.jp_col.size(), 0);
    {
        std::vector<int> fill(S.jpt_ptr.begin(), S.jpt_ptr.end() - 1);
        for (int q = 0; q < S.n_x; q++)
            for (int s = S.jp_ptr[q]; s < S.jp_ptr[q + 1]; s++) {
                int d = fill[S.jp_col[s]]++;
                S.jpt_row[d] = q;
                S.jpt_src[d] = s;
            }
    }

    // warps of the power-flow evaluation: consecutive buses whose admittance rows
    // together hold at most 32 entries, one entry per lane (empty if some row is
    // longer than a warp: the evaluation then takes one thread per bus)
    S.pf_wb.assign(1, 0);
    S.yrow.assign(S.yj.size(), 0);
    for (int i = 0; i < n_bus; i++)
        for (int s = S.yp[i]; s < S.yp[i + 1]; s++) S.yrow[s] = i;
    for (int i = 0; i < n_bus; i++) {
        if (S.yp[i + 1] - S.yp[i] > 32) {
            S.pf_wb.clear();
            break;
        }
        if (S.yp[i + 1] - S.yp[S.pf_wb.back()] > 32) S.pf_wb.push_back(i);
    }
    if (!S.pf_wb.empty()) S.pf_wb.push_back(n_bus);
    return "";
}

}  // namespace rh
