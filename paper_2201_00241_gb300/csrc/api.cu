// api.cu -- extern "C" entry points of librh (declared in include/rh.h).
//
// Host code only: argument checks, device memory, the Newton and setup
// sequencing, copies for host-pointer calls.  Every numerical step runs in the
// kernels of kernels.cu.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <memory>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/rh.h"
#include "rh_internal.h"
#include "rh_kernels.h"

namespace {

thread_local std::string g_last_error;

rh_status fail(rh_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

#define RH_CUDA(call)                                                                           \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? RH_ENOMEM : RH_ECUDA,                 \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                    \
    } while (0)

template <typename T>
struct DevArr {
    T* p = nullptr;
    size_t n = 0;
};

}  // namespace

struct rh_grid {
    int device = 0;
    rh::Symbolic S;
    double base_mva = 100.0;
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;

    // --- device: topology (static) --------------------------------------
    int *yp = nullptr, *yj = nullptr, *ydiag = nullptr, *yrow = nullptr, *pf_wb = nullptr;
    double* sc = nullptr;          // sin, cos per bus (the assembly's preparation)
    double *G = nullptr, *B = nullptr;
    int *qth = nullptr, *qv = nullptr, *ip_v = nullptr, *ip_pg = nullptr, *ix_th = nullptr, *ix_v = nullptr;
    int *pg_slot = nullptr, *jac_dst = nullptr;
    int *col_th = nullptr, *col_v = nullptr, *col_pg = nullptr;   // seed colours (coloured AD)
    int jac_method = RH_JAC_ANALYTIC;
    double *c2 = nullptr, *c1 = nullptr;
    int *rowptr = nullptr, *col = nullptr, *diagpos = nullptr, *tpos = nullptr, *q0 = nullptr;
    uint8_t* nv = nullptr;
    int *flev_ptr = nullptr, *flev_bus = nullptr, *flev_maxext = nullptr;
    int4 *fslot = nullptr, *bslot = nullptr;
    // sparse-part schedules and the tail's external phase (device), with host level pointers
    int *sf_ptr = nullptr, *sf_maxext = nullptr, *sb_ptr = nullptr, *sb_maxext = nullptr;
    int *ef_ptr = nullptr, *ef_maxext = nullptr;
    int4 *sf_slot = nullptr, *sb_slot = nullptr, *ef_slot = nullptr;
    int n_sf = 0, n_sb = 0, n_ef = 0;
    // backward schedule of the buses whose psi rows SpMulAdd reads (rows of J_p and
    // their ancestors): the L^T sweep of a launch that ends in SpMulAdd
    int *sbr_ptr = nullptr, *sbr_maxext = nullptr;
    int4* sbr_slot = nullptr;
    int n_sbr = 0;
    int* tail_pos = nullptr;
    int *qtheta = nullptr, *bparent = nullptr;
    int *jp_rows = nullptr, *jp_zero_rows = nullptr;
    int n_jp_rows = 0, n_jp_zero = 0;
    double *triL = nullptr, *triU = nullptr, *triUt = nullptr, *triLt = nullptr;
    // unit-diagonal factors of the direction kernel (J_x = D L'' U')
    double *Ad = nullptr, *Atd = nullptr, *jptvd = nullptr;
    int* arow = nullptr;   // row of every position of A
    double *triLd = nullptr, *triUd = nullptr, *triUtd = nullptr, *triLtd = nullptr;
    int *blev_ptr = nullptr, *blev_bus = nullptr, *blev_maxext = nullptr;
    int *rf_lev_bus = nullptr, *rf_tgt_pos = nullptr, *rf_grp = nullptr, *rf_xgrp = nullptr;
    int64_t* rf_xptr = nullptr;
    int *rf_piv_bus = nullptr, *rf_piv_pos = nullptr;
    double4_32a* rf_piv = nullptr;          // per sparse bus: 1/u_tt, l_vt, 1/u_vv, u_tv
    int *rf_pe_bus = nullptr, *rf_pe_pos = nullptr;
    int *jp_ptr = nullptr, *jp_col = nullptr, *jpt_ptr = nullptr, *jpt_row = nullptr, *jpt_src = nullptr;
    // identity W over all n_p columns: direction j takes column hcolmap[j], the columns in the
    // postorder of their generator buses in the elimination tree, so that the few
    // directions of a CTA share most of their reach; and the CTAs' reach, per CTA count
    int* hcolmap = nullptr;
    std::vector<int> colmap;                    // host copy
    std::map<int, rh::ReachSched*> reach_dev;   // device structs, keyed by the launch's CTA count
    int *tp_bus = nullptr, *uth = nullptr, *uv = nullptr, *inc_ptr = nullptr, *inc_nb = nullptr;
    int* tp_l0 = nullptr;   // per bus: position of (v, theta) in At for a PQ bus of forward level 0, else -1
    int *inc_uth = nullptr, *inc_uv = nullptr, *gref_row = nullptr, *pg_row = nullptr, *xmap = nullptr;
    uint8_t* has_gref = nullptr;
    int n_inc = 0, n_gref = 0;

    // --- device: state ----------------------------------------------------
    double *vm = nullptr, *va = nullptr, *pg = nullptr, *pd = nullptr, *qd = nullptr, *P = nullptr, *Q = nullptr;
    double *A = nullptr, *At = nullptr, *invdiag = nullptr, *jpv = nullptr, *jptv = nullptr;
    double *gres = nullptr, *lam = nullptr, *grad = nullptr, *v1 = nullptr;
    double4_32a* inc_coef = nullptr;
    double *d2 = nullptr, *asum = nullptr, *csum = nullptr, *pg_curv = nullptr, *gref_th = nullptr,
           *gref_v = nullptr, *gref_val = nullptr;
    double *tmp_bus = nullptr;     // 4 * n_bus scratch for rh_injections
    double *rto_y = nullptr;       // n_p: workspace of the tracking step's solve
    double *tailD = nullptr;       // T x T scratch of the dense tail LU
    double *pbuf = nullptr;        // n_p
    double *xbuf = nullptr;        // n_x
    // scalars: cref, c2ref, F
    double* dscal = nullptr;
    unsigned long long* umax = nullptr;  // gmax, jmax
    int* err = nullptr;

    // --- workspace for the direction kernel --------------------------------
    double *V = nullptr, *T = nullptr;
    size_t ws_elems = 0;
    double *stage_in = nullptr, *stage_out = nullptr;
    size_t stage_n = 0;

    bool adjoint_ready = false;
    // batched Newton (rh_batch_powerflow): the grid's identity and structure, the
    // captured per-iteration graphs of batches led by this grid, keyed by the items'
    // identities and the set of items still iterating, and a status buffer
    uint64_t uid = 0, topo_hash = 0;
    std::map<std::string, cudaGraphExec_t> pf_graphs;
    double *bstat_d = nullptr, *bstat_h = nullptr;
    cudaGraphExec_t adj_exec = nullptr;   // captured device work of rh_adjoint
    int adj_kernels = 0;                  // kernel nodes in that graph
    // rh_powerflow: a Newton iteration's device work as two graphs (the refactorisation
    // with its factor copies; the step, the update and the next assembly)
    cudaGraphExec_t nt_fac_exec = nullptr, nt_step_exec = nullptr;
    cudaEvent_t apply_done = nullptr;     // orders a tracking step's parameter update before later grid work

    // rh_reduced_hessian: its captured graph (for one H pointer, leading dimension and
    // workspace), the second stream and events of the fork and join, and the timing
    // events around the direction launches
    cudaGraphExec_t hess_exec = nullptr;
    const double* hess_H = nullptr;
    int64_t hess_ld = 0;
    const double *hess_V = nullptr, *hess_T = nullptr;
    int hess_kernels = 0;
    bool hess_timed = false;
    cudaStream_t stream2 = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_user = nullptr;
    cudaEvent_t ev_d0 = nullptr, ev_d1 = nullptr, ev_v = nullptr, ev_c = nullptr;   // timing
    cudaEvent_t ev_pf0 = nullptr, ev_pf1 = nullptr;   // fork / join of the L2 prefetch beside the assembly

    void drop_graphs() {
        for (cudaGraphExec_t e : {adj_exec, hess_exec, nt_fac_exec, nt_step_exec})
            if (e) cudaGraphExecDestroy(e);
        adj_exec = hess_exec = nt_fac_exec = nt_step_exec = nullptr;
        for (auto& kv : pf_graphs) cudaGraphExecDestroy(kv.second);
        pf_graphs.clear();
    }

    ~rh_grid() {
        drop_graphs();
        if (apply_done) cudaEventDestroy(apply_done);
        for (cudaEvent_t e : {ev_fork, ev_join, ev_user, ev_d0, ev_d1, ev_v, ev_c, ev_pf0, ev_pf1})
            if (e) cudaEventDestroy(e);
        if (stream2) cudaStreamDestroy(stream2);
        if (bstat_h) cudaFreeHost(bstat_h);
        for (void* p : allocs) cudaFree(p);
        if (V) cudaFree(V);
        if (T) cudaFree(T);
        if (stage_in) cudaFree(stage_in);
        if (stage_out) cudaFree(stage_out);
        if (stream) cudaStreamDestroy(stream);
    }

    template <typename T_>
    cudaError_t alloc(T_*& p, size_t n) {
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, (n ? n : 1) * sizeof(T_));
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        p = (T_*)q;
        return cudaMemset(q, 0, (n ? n : 1) * sizeof(T_));
    }
    template <typename T_>
    cudaError_t upload(T_*& p, const std::vector<T_>& v) {
        cudaError_t e = alloc(p, v.size());
        if (e != cudaSuccess || v.empty()) return e;
        return cudaMemcpy(p, v.data(), v.size() * sizeof(T_), cudaMemcpyHostToDevice);
    }

    rh::PfGrid pf() const {
        rh::PfGrid g;
        g.n_bus = S.n_bus;
        g.n_x = S.n_x;
        g.ref = S.ref;
        g.nnz_a = (int)S.col.size();
        g.nnz_jp = (int)S.jp_col.size();
        g.yp = yp; g.yj = yj; g.ydiag = ydiag; g.G = G; g.B = B;
        g.qth = qth; g.qv = qv; g.ip_v = ip_v; g.ip_pg = ip_pg;
        g.jac_dst = jac_dst; g.pg_slot = pg_slot;
        g.base_mva = base_mva; g.c2 = c2; g.c1 = c1;
        g.yrow = yrow; g.pf_wb = pf_wb; g.n_pfw = S.pf_wb.empty() ? 0 : (int)S.pf_wb.size() - 1;
        return g;
    }
    rh::PfState st() const {
        rh::PfState s;
        s.vm = vm; s.va = va; s.pg = pg; s.pd = pd; s.qd = qd; s.P = P; s.Q = Q; s.sc = sc;
        return s;
    }
    rh::DirGrid dir() const {
        rh::DirGrid g;
        g.n_x = S.n_x; g.n_p = S.n_p; g.zero_row = S.n_x + S.n_p;
        g.nnz = (int)S.col.size();
        g.col = col; g.A = A; g.At = At; g.invdiag = invdiag;
        g.lf = {S.n_flev, flev_ptr, fslot, flev_maxext};
        g.lb = {S.n_blev, blev_ptr, bslot, blev_maxext};
        g.sf = {n_sf, sf_ptr, sf_slot, sf_maxext};
        g.sb = {n_sb, sb_ptr, sb_slot, sb_maxext};
        g.sbr = {n_sbr, sbr_ptr, sbr_slot, sbr_maxext};
        g.ef = {n_ef, ef_ptr, ef_slot, ef_maxext};
        g.t0 = S.t0; g.T = S.n_x - S.t0;
        g.ks_cap = 32;
        g.triL = triL; g.triU = triU; g.triUt = triUt; g.triLt = triLt;
        g.Ad = Ad; g.Atd = Atd; g.jptvd = jptvd;
        g.triLd = triLd; g.triUd = triUd; g.triUtd = triUtd; g.triLtd = triLtd;
        g.qtheta = qtheta; g.bparent = bparent;
        g.jp_ptr = jp_ptr; g.jp_col = jp_col; g.jpv = jpv;
        g.n_jp_rows = n_jp_rows; g.n_jp_zero = n_jp_zero; g.jp_rows = jp_rows; g.jp_zero_rows = jp_zero_rows;
        g.jpt_ptr = jpt_ptr; g.jpt_row = jpt_row; g.jptv = jptv;
        g.n_bus = S.n_bus; g.tp_bus = tp_bus; g.uth = uth; g.uv = uv; g.tp_l0 = tp_l0;
        g.inc_ptr = inc_ptr; g.inc_uth = inc_uth; g.inc_uv = inc_uv; g.inc_coef = inc_coef;
        g.d2 = d2; g.asum = asum; g.csum = csum; g.has_gref = has_gref; g.gref_th = gref_th; g.gref_v = gref_v;
        g.n_gref = n_gref; g.gref_row = gref_row; g.gref_val = gref_val; g.c2ref = dscal + 1;
        g.pg_row = pg_row; g.pg_curv = pg_curv;
        return g;
    }
    rh::RfGrid rf() const {
        rh::RfGrid g;
        g.n_x = S.n_x; g.t0 = S.t0; g.T = S.n_x - S.t0;
        g.nnz = (int)S.col.size();
        g.rf_lev_bus = rf_lev_bus; g.q0 = q0; g.nv = nv;
        g.rowptr = rowptr; g.col = col; g.diagpos = diagpos; g.tpos = tpos;
        g.tgt_pos = rf_tgt_pos; g.grp = reinterpret_cast<const int2*>(rf_grp);
        g.xptr = rf_xptr; g.xgrp = reinterpret_cast<const int2*>(rf_xgrp);
        g.piv = rf_piv; g.n_piv = S.tail_bus0; g.piv_bus = rf_piv_bus; g.piv_pos = rf_piv_pos;
        g.n_pe = (int64_t)S.rf_pe_bus.size(); g.pe_bus = rf_pe_bus; g.pe_pos = reinterpret_cast<const int4*>(rf_pe_pos);
        g.A = A; g.invdiag = invdiag; g.jmax = umax + 1; g.err = err;
        g.tailD = tailD; g.tail_pos = tail_pos;
        return g;
    }
    int rows() const { return S.n_x + S.n_p + 1; }
};

namespace {

// The order of the identity columns in full-Hessian launches: by the lowest
// postorder, in the elimination tree, of the buses of a column's J_p rows (parent:
// the first later bus of a bus's pattern; children and roots visited in ascending
// position; ties keep the column order).  The directions of one CTA then come from
// one part of the tree and share most of their reach.
std::vector<int> tree_column_order(const rh::Symbolic& S) {
    const int ne = S.n_elim, np = S.n_p;
    std::vector<std::vector<int>> kids(ne);
    std::vector<int> roots, post(ne, 0), bpos(S.n_x);
    for (int k = 0; k < ne; k++) {
        if (S.colpat[k].empty()) roots.push_back(k);
        else kids[S.colpat[k][0]].push_back(k);
        for (int t = 0; t < S.nv[k]; t++) bpos[S.q0[k] + t] = k;
    }
    int cnt = 0;
    std::vector<std::pair<int, size_t>> stk;
    for (auto r = roots.rbegin(); r != roots.rend(); ++r) stk.emplace_back(*r, 0);
    while (!stk.empty()) {
        auto& top = stk.back();
        if (top.second < kids[top.first].size()) {
            const int c = kids[top.first][top.second++];
            stk.emplace_back(c, 0);
        } else {
            post[top.first] = cnt++;
            stk.pop_back();
        }
    }
    std::vector<int> anchor(np, ne), cm(np);
    for (int j = 0; j < np; j++) {
        for (int t = S.jpt_ptr[j]; t < S.jpt_ptr[j + 1]; t++) anchor[j] = std::min(anchor[j], post[bpos[S.jpt_row[t]]]);
        cm[j] = j;
    }
    std::stable_sort(cm.begin(), cm.end(), [&](int a, int b) { return anchor[a] < anchor[b]; });
    return cm;
}

rh_status set_device(const rh_grid* g) {
    if (g->device < 0) return fail(RH_ESTATE, "grid was created without a device (symbolic only)");
    RH_CUDA(cudaSetDevice(g->device));
    return RH_OK;
}

// V and T hold at least n doubles each
rh_status ensure_ws_elems(rh_grid* g, size_t n) {
    if (n <= g->ws_elems) return RH_OK;
    if (g->V) { cudaFree(g->V); g->V = nullptr; }
    if (g->T) { cudaFree(g->T); g->T = nullptr; }
    g->ws_elems = 0;
    RH_CUDA(cudaMalloc(&g->V, n * sizeof(double)));
    RH_CUDA(cudaMalloc(&g->T, n * sizeof(double)));
    g->ws_elems = n;
    return RH_OK;
}

rh_status ensure_ws(rh_grid* g, size_t cols) { return ensure_ws_elems(g, (size_t)g->rows() * cols); }

rh_status ensure_stage(rh_grid* g, size_t n) {
    if (n <= g->stage_n) return RH_OK;
    if (g->stage_in) { cudaFree(g->stage_in); g->stage_in = nullptr; }
    if (g->stage_out) { cudaFree(g->stage_out); g->stage_out = nullptr; }
    g->stage_n = 0;
    RH_CUDA(cudaMalloc(&g->stage_in, n * sizeof(double)));
    RH_CUDA(cudaMalloc(&g->stage_out, n * sizeof(double)));
    g->stage_n = n;
    return RH_OK;
}

rh_status check_err_flag(rh_grid* g) {
    int e = 0;
    RH_CUDA(cudaMemcpyAsync(&e, g->err, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    RH_CUDA(cudaStreamSynchronize(g->stream));
    if (e & 1) return fail(RH_ESINGULAR, "LU refactorisation: a static pivot is below 1e-14 max|J_x|");
    return RH_OK;
}

// Captures what `enqueue` puts on g->stream (and on streams it joins) into an
// executable graph, counting its kernel nodes.
template <class F>
rh_status capture_graph(rh_grid* g, F&& enqueue, cudaGraphExec_t* exec, int* kernels) {
    cudaGraph_t graph = nullptr;
    RH_CUDA(cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal));
    rh_status st = enqueue();
    cudaError_t ce = cudaStreamEndCapture(g->stream, &graph);
    if (st) { if (graph) cudaGraphDestroy(graph); return st; }
    if (ce != cudaSuccess) return fail(RH_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    size_t n_nodes = 0;
    if (cudaGraphGetNodes(graph, nullptr, &n_nodes) == cudaSuccess) {
        std::vector<cudaGraphNode_t> nodes(n_nodes);
        int k = 0;
        if (n_nodes && cudaGraphGetNodes(graph, nodes.data(), &n_nodes) == cudaSuccess)
            for (auto nd : nodes) {
                cudaGraphNodeType ty;
                if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) k++;
            }
        *kernels = k;
    }
    ce = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) { *exec = nullptr; return fail(RH_ECUDA, std::string("graph: ") + cudaGetErrorString(ce)); }
    return RH_OK;
}

// Injections, residual (when gres is given) and the values of J_x (into the
// slots of A, cleared first together with the maxima and the pivot flag) and J_p,
// by the analytic formulas or by coloured forward-mode AD (enqueue only).
rh_status assemble(rh_grid* g, int method, double* gres, cudaStream_t s) {
    const bool ad = (method == RH_JAC_COLORED_AD);
    rh::launch_pf_prep(g->pf(), g->st(), g->A, g->umax, g->err, true, s);
    rh::launch_pf_eval(g->pf(), g->st(), gres, g->A, g->jpv, g->umax, g->umax + 1, !ad, s);
    if (ad)
        RH_CUDA(rh::launch_jac_ad(g->pf(), g->st(), g->col_th, g->col_v, g->col_pg,
                                  g->S.n_colors_x + g->S.n_colors_p, g->A, g->jpv, g->umax + 1, s));
    RH_CUDA(cudaGetLastError());
    return RH_OK;
}

// Transposed values, the direction kernel's unit-diagonal factors and the dense
// tail's triangles from the current LU (enqueue only).
void enqueue_factor_copies(rh_grid* g, cudaStream_t s) {
    const auto& S = g->S;
    rh::launch_transpose_values((int)S.col.size(), g->tpos, g->arow, g->col, g->diagpos, g->A, g->invdiag, g->At,
                                g->Ad, g->Atd, (int)S.jp_col.size(), g->jpt_src, g->jpt_row, g->jpv, g->jptv,
                                g->jptvd, s);
    rh::launch_build_tail(S.n_x - S.t0, S.t0, g->tail_pos, g->A, g->invdiag, g->triL, g->triU, g->triUt, g->triLt,
                          g->triLd, g->triUd, g->triUtd, g->triLtd, s);
}

// L2 prefetch of the refactorisation's level data, read level by level after
// the Jacobian assembly: on stream2 beside the assembly, joined before the first
// update launch by enqueue_rf_prefetch_join (enqueue only)
void enqueue_rf_prefetch(rh_grid* g, cudaStream_t s) {
    const auto& S = g->S;
    rh::PrefetchList L{};
    auto add = [&](const void* p, size_t bytes) {
        if (p && bytes >= 16 && L.n < 8) {
            L.p[L.n] = (const char*)p;
            L.bytes[L.n++] = bytes;
        }
    };
    add(g->rf_tgt_pos, S.rf_tgt_pos.size() * sizeof(int));
    add(g->rf_grp, S.rf_grp.size() * sizeof(int));
    add(g->rf_xptr, S.rf_xptr.size() * sizeof(int64_t));
    add(g->rf_xgrp, S.rf_xgrp.size() * sizeof(int));
    add(g->rf_piv_pos, S.rf_piv_pos.size() * sizeof(int));
    add(g->rf_pe_pos, S.rf_pe_ut.size() * sizeof(int));
    add(g->rf_pe_bus, S.rf_pe_bus.size() * sizeof(int));
    if (cudaEventRecord(g->ev_pf0, s) == cudaSuccess && cudaStreamWaitEvent(g->stream2, g->ev_pf0, 0) == cudaSuccess) {
        rh::launch_prefetch_l2(L, g->stream2);
        cudaEventRecord(g->ev_pf1, g->stream2);
    } else {
        rh::launch_prefetch_l2(L, s);
        cudaEventRecord(g->ev_pf1, s);
    }
}
cudaError_t enqueue_rf_prefetch_join(rh_grid* g, cudaStream_t s) { return cudaStreamWaitEvent(s, g->ev_pf1, 0); }

// J_x, J_p at the current state, refactorisation, transposed copies (enqueue only).
rh_status enqueue_factor(rh_grid* g) {
    const auto& S = g->S;
    cudaStream_t s = g->stream;
    enqueue_rf_prefetch(g, s);
    rh_status st = assemble(g, g->jac_method, nullptr, s);
    if (st) return st;
    RH_CUDA(enqueue_rf_prefetch_join(g, s));
    RH_CUDA(rh::launch_refactor(g->rf(), S.rf_lev_ptr.data(), S.rf_tgt_lev_ptr.data(), S.rf_piv_lev_ptr.data(), S.rf_n_lev, s));
    enqueue_factor_copies(g, s);
    RH_CUDA(cudaGetLastError());
    return RH_OK;
}

rh_status assemble_and_factor(rh_grid* g) {
    rh_status st = enqueue_factor(g);
    if (st) return st;
    return check_err_flag(g);
}

// n_cta > 0 caps the CTA count (the default is one per slot of the device)
// The reach of every CTA of an identity-W launch of all n_p directions on n_cta CTAs
// (columns through hcolmap), built on the host once per CTA count: for CTA c, the
// buses of its J_p columns and their ancestors in the sparse part, as forward slots
// grouped by level (PQ buses first, then longer rows, like the full schedule), and
// the mask of their rows (seed rows in the dense tail included, as the run-time
// mask has them).  Must be called outside stream capture (it allocates and copies).
rh_status reach_schedule(rh_grid* g, int n_cta, rh::ReachSched** out) {
    *out = nullptr;
    auto f = g->reach_dev.find(n_cta);
    if (f != g->reach_dev.end()) {
        *out = f->second;
        return RH_OK;
    }
    const auto& S = g->S;
    const int np = S.n_p, ne = S.n_elim, words = (S.n_x + 31) / 32;
    const std::vector<int>& cm = g->colmap;
    std::vector<int> bpos(S.n_x);
    for (int k = 0; k < ne; k++)
        for (int t = 0; t < S.nv[k]; t++) bpos[S.q0[k] + t] = k;
    std::vector<int> nlev(n_cta), lev0(n_cta), ptr, mx;
    std::vector<int4> slots;
    std::vector<unsigned> masks((size_t)n_cta * words, 0u);
    std::vector<char> in(ne);
    std::vector<int> sel;
    for (int c = 0; c < n_cta; c++) {
        const int c0 = (int)((int64_t)c * np / n_cta), c1 = (int)((int64_t)(c + 1) * np / n_cta);
        std::fill(in.begin(), in.end(), 0);
        unsigned* m = masks.data() + (size_t)c * words;
        for (int j = c0; j < c1; j++)
            for (int t = S.jpt_ptr[cm[j]]; t < S.jpt_ptr[cm[j] + 1]; t++) {
                const int k = bpos[S.jpt_row[t]];
                in[k] = 1;
                for (int u = 0; u < S.nv[k]; u++) m[(S.q0[k] + u) >> 5] |= 1u << ((S.q0[k] + u) & 31);
            }
        sel.clear();
        for (int k = 0; k < S.tail_bus0; k++) {
            if (!in[k]) continue;
            sel.push_back(k);
            for (int u = 0; u < S.nv[k]; u++) m[(S.q0[k] + u) >> 5] |= 1u << ((S.q0[k] + u) & 31);
            if (!S.colpat[k].empty() && S.colpat[k][0] < S.tail_bus0) in[S.colpat[k][0]] = 1;
        }
        auto ext = [&](int k) { return S.diagpos[S.q0[k]] - S.rowptr[S.q0[k]]; };
        std::stable_sort(sel.begin(), sel.end(), [&](int a, int b) {
            if (S.flevel[a] != S.flevel[b]) return S.flevel[a] < S.flevel[b];
            if (S.nv[a] != S.nv[b]) return S.nv[a] > S.nv[b];
            return ext(a) > ext(b);
        });
        lev0[c] = (int)mx.size();
        int cur = -1;
        for (int k : sel) {
            if (S.flevel[k] != cur) {
                ptr.push_back((int)slots.size());
                mx.push_back(0);
                cur = S.flevel[k];
            }
            const int q = S.q0[k];
            slots.push_back(make_int4(q, ext(k), S.rowptr[q], S.nv[k] == 2 ? S.rowptr[q + 1] : -1));
            mx.back() = std::max(mx.back(), ext(k));
        }
        ptr.push_back((int)slots.size());
        nlev[c] = (int)mx.size() - lev0[c];
    }
    rh::ReachSched h;
    h.n_cta = n_cta;
    h.words = words;
    int *d_nlev, *d_lev0, *d_ptr, *d_mx;
    int4* d_slots;
    unsigned* d_masks;
    RH_CUDA(g->upload(d_nlev, nlev));
    RH_CUDA(g->upload(d_lev0, lev0));
    RH_CUDA(g->upload(d_ptr, ptr));
    RH_CUDA(g->upload(d_mx, mx));
    RH_CUDA(g->upload(d_slots, slots));
    RH_CUDA(g->upload(d_masks, masks));
    h.nlev = d_nlev; h.lev0 = d_lev0; h.ptr = d_ptr; h.maxext = d_mx; h.slots = d_slots; h.masks = d_masks;
    rh::ReachSched* d = nullptr;
    RH_CUDA(g->alloc(d, 1));
    RH_CUDA(cudaMemcpy(d, &h, sizeof(h), cudaMemcpyHostToDevice));
    g->reach_dev[n_cta] = d;
    *out = d;
    return RH_OK;
}

// CTAs of a direction launch: the fewest that keep the default grid's largest number of
// directions per CTA, so that every CTA holds the same number (all but the last).  On the
// 9241-bus grid, 304 CTAs of 9 or 10 directions left a few CTAs 10 % behind the rest every
// time, whatever their directions or workspace addresses; 289 CTAs of 10 did not, and
// ended the launch 0.1-0.3 ms sooner.
int balanced_ctas(int N) {
    const int grid = rh::dirs_default_ctas(N);
    const int per = (N + grid - 1) / grid;
    return std::max(1, (N + per - 1) / per);
}

rh_status dirs(rh_grid* g, int N, int64_t ld, double* V, double* T, const double* W, int64_t ldw, int col0,
               double* HW, int64_t ldhw, unsigned phases, cudaStream_t s, int n_cta = 0) {
    rh::DirLaunch L;
    L.N = N;
    L.n_cta = balanced_ctas(N);
    if (n_cta > 0 && n_cta < L.n_cta) L.n_cta = n_cta;
    L.ld = ld;
    L.cta_stride = 0;
    L.V = V;
    L.T = T;
    L.W = W;
    L.ldw = ldw;
    L.col0 = col0;
    L.HW = HW;
    L.ldhw = ldhw;
    L.phases = phases;
    L.ws_elems = V == g->V ? (int64_t)g->ws_elems : (V == g->v1 ? (int64_t)g->rows() : 0);
    L.use_tail = rh::dirs_tail_fits(g->S.n_x - g->S.t0, N, L.n_cta) ? 1 : 0;
    L.use_reach = (L.use_tail && !W && (phases & rh::PH_WLOAD) && (phases & rh::PH_L) && (phases & rh::PH_U)) ? 1 : 0;
    // all n_p identity columns: in the tree order of hcolmap, with each CTA's reach precomputed
    const bool all_cols = !W && col0 == 0 && N == g->S.n_p && g->hcolmap;
    L.colmap = (all_cols && (phases & (rh::PH_WLOAD | rh::PH_MULADD))) ? g->hcolmap : nullptr;
    L.reach = nullptr;
    if (all_cols && L.use_reach) {
        auto f = g->reach_dev.find(L.n_cta);
        if (f != g->reach_dev.end()) {
            L.reach = f->second;
        } else {
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            RH_CUDA(cudaStreamIsCapturing(s, &cs));
            if (cs == cudaStreamCaptureStatusNone) {
                rh::ReachSched* rs = nullptr;
                rh_status st = reach_schedule(g, L.n_cta, &rs);
                if (st) return st;
                L.reach = rs;
            }
        }
    }
    rh::launch_dirs(g->dir(), L, s);
    RH_CUDA(cudaGetLastError());
    return RH_OK;
}

// single right-hand side in g->v1 (internal order), in place.  beside_dirs: as
// one CTA of the direction kernel, which fits in the slot a direction launch of
// fewer CTAs than the device holds leaves free (k_solve1's shared-memory x
// needs a shared-memory carveout that an SM running k_dirs does not have).
rh_status solve_one(rh_grid* g, unsigned phases, cudaStream_t s, bool beside_dirs = false) {
    const int mode = beside_dirs ? 0 : rh::solve1_mode(g->S.n_x, g->S.n_x - g->S.t0);
    if (mode > 0) {
        RH_CUDA(rh::launch_solve1(g->dir(), g->v1, phases, mode == 2, s));
        return RH_OK;
    }
    // through k_dirs, whose factors are unit-diagonal (J_x = D L'' U'): the right-hand
    // side of J_x z = b enters as D^-1 b, and J_x^T's solution D psi leaves as psi
    if (phases & rh::PH_L) rh::launch_scale_rows(g->S.n_x, 1, g->invdiag, g->v1, 1, s);
    rh_status st = dirs(g, 1, 1, g->v1, g->v1, nullptr, 0, 0, nullptr, 0, phases, s);
    if (st) return st;
    if (phases & rh::PH_LT) rh::launch_scale_rows(g->S.n_x, 1, g->invdiag, g->v1, 1, s);
    return RH_OK;
}

__global__ void k_set_p(int n_bus, const int* ip_v, const int* ip_pg, const double* p, double* vm, double* pg) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_bus) return;
    if (ip_v[i] >= 0) vm[i] = p[ip_v[i]];
    pg[i] = ip_pg[i] >= 0 ? p[ip_pg[i]] : 0.0;
}

__global__ void k_set_x(int n_bus, const int* ix_th, const int* ix_v, const double* x, double* vm, double* va) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_bus) return;
    va[i] = ix_th[i] >= 0 ? x[ix_th[i]] : 0.0;
    if (ix_v[i] >= 0) vm[i] = x[ix_v[i]];
}

__global__ void k_get_x(int n_bus, const int* ix_th, const int* ix_v, const double* vm, const double* va, double* x) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_bus) return;
    if (ix_th[i] >= 0) x[ix_th[i]] = va[i];
    if (ix_v[i] >= 0) x[ix_v[i]] = vm[i];
}

// Tracking step (section 6.3): right-hand side -g, p_next = p + d, and the
// optional hand-over of p_next to the grid, which only happens when the
// factorisation reported no bad pivot.
__global__ void k_rto_rhs(int n, const double* grad, double* d) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = -grad[i];
}

__global__ void k_rto_next(int n, const double* p, const double* d, double* p_next) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p_next[i] = p[i] + d[i];
}

__global__ void k_rto_apply(int n_p, int n_bus, const int* info, const double* p_next, double* p, const int* ip_v,
                            const int* ip_pg, double* vm, double* pg) {
    if (*info != 0) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_p) p[i] = p_next[i];
    if (i < n_bus) {
        if (ip_v[i] >= 0) vm[i] = p_next[ip_v[i]];
        pg[i] = ip_pg[i] >= 0 ? p_next[ip_pg[i]] : 0.0;
    }
}

int nblk(int n, int t) { return (n + t - 1) / t; }

}  // namespace

extern "C" {

const char* rh_last_error(void) { return g_last_error.c_str(); }

rh_status rh_grid_create(const rh_grid_desc* d, int32_t device, rh_grid** out) {
    if (!out) return fail(RH_EINVAL, "out is NULL");
    *out = nullptr;
    if (!d || !d->from || !d->to || !d->r || !d->x || !d->b || !d->bus_type || !d->c2 || !d->c1)
        return fail(RH_EINVAL, "grid descriptor has a NULL array");
    if (!(d->base_mva > 0.0)) return fail(RH_EINVAL, "base_mva must be positive");
    if (d->max_tail != 0 && (d->max_tail < 2 || d->max_tail > 512))
        return fail(RH_EINVAL, "max_tail must be 0 or in [2, 512]");
    std::unique_ptr<rh_grid> g(new rh_grid());
    g->device = device;
    g->base_mva = d->base_mva;
    std::string msg = rh::build_symbolic(d->n_bus, d->n_branch, d->from, d->to, d->r, d->x, d->b, d->bus_type,
                                         d->order_level_cost, g->S, d->max_tail);
    if (!msg.empty()) return fail(RH_EINVAL, msg);
    {
        static std::atomic<uint64_t> next_uid{1};
        g->uid = next_uid++;
        // FNV-1a over the structure the batched refactorisation shares between grids
        uint64_t h = 1469598103934665603ull;
        auto mix = [&h](const void* p, size_t n) {
            const unsigned char* b = (const unsigned char*)p;
            for (size_t i = 0; i < n; i++) { h ^= b[i]; h *= 1099511628211ull; }
        };
        const auto& S = g->S;
        const int dims[4] = {S.n_bus, S.n_x, S.n_p, S.t0};
        mix(dims, sizeof dims);
        for (const std::vector<int>* v : {&S.ebus, &S.rowptr, &S.col, &S.rf_lev_ptr, &S.rf_lev_bus, &S.rf_tgt_pos,
                                          &S.rf_grp, &S.rf_xgrp, &S.rf_piv_lev_ptr, &S.rf_piv_bus, &S.rf_piv_pos,
                                          &S.rf_pe_bus, &S.rf_pe_ut,
                                          &S.jac_dst, &S.yp, &S.yj})
            mix(v->data(), v->size() * sizeof(int));
        mix(S.rf_tgt_lev_ptr.data(), S.rf_tgt_lev_ptr.size() * sizeof(int64_t));
        mix(S.rf_xptr.data(), S.rf_xptr.size() * sizeof(int64_t));
        g->topo_hash = h;
    }
    g->colmap = tree_column_order(g->S);
    const auto& S = g->S;
    if (device < 0) {  // symbolic phase only: no device state
        *out = g.release();
        return RH_OK;
    }
    RH_CUDA(cudaSetDevice(device));
    RH_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    RH_CUDA(cudaStreamCreateWithFlags(&g->stream2, cudaStreamNonBlocking));
    RH_CUDA(cudaEventCreateWithFlags(&g->ev_pf0, cudaEventDisableTiming));
    RH_CUDA(cudaEventCreateWithFlags(&g->ev_pf1, cudaEventDisableTiming));
    RH_CUDA(rh::prepare_kernels());
    int nb = S.n_bus, nx = S.n_x, np = S.n_p;
    int zero_row = nx + np;

    // projection structure
    std::vector<int> uth(nb), uv(nb), pg_row(nb, -1), inc_ptr(nb + 1, 0), inc_nb, inc_uth, inc_uv;
    std::vector<uint8_t> has_gref(nb, 0);
    for (int i = 0; i < nb; i++) {
        uth[i] = S.qth[i] >= 0 ? S.qth[i] : zero_row;
        uv[i] = S.qv[i] >= 0 ? S.qv[i] : nx + S.ip_v[i];
        if (S.ip_pg[i] >= 0) pg_row[i] = nx + S.ip_pg[i];
    }
    for (int i = 0; i < nb; i++) {
        for (int t = S.yp[i]; t < S.yp[i + 1]; t++) {
            int j = S.yj[t];
            if (j == i) continue;
            inc_nb.push_back(j);
            inc_uth.push_back(uth[j]);
            inc_uv.push_back(uv[j]);
        }
        inc_ptr[i + 1] = (int)inc_nb.size();
    }
    has_gref[S.ref] = 1;
    for (int t = S.yp[S.ref]; t < S.yp[S.ref + 1]; t++) has_gref[S.yj[t]] = 1;
    g->n_inc = (int)inc_nb.size();
    g->n_gref = 1 + 2 * (S.yp[S.ref + 1] - S.yp[S.ref] - 1);
    // projection order: degree descending, then buses with a Pg row, then elimination order, so
    // that the lanes of a warp share their incidence count and their branches
    std::vector<int> tp_bus(S.ebus);
    tp_bus.push_back(S.ref);
    std::stable_sort(tp_bus.begin(), tp_bus.end(), [&](int a, int b) {
        int da = inc_ptr[a + 1] - inc_ptr[a], db = inc_ptr[b + 1] - inc_ptr[b];
        if (da != db) return da > db;
        return (pg_row[a] >= 0) > (pg_row[b] >= 0);
    });
    std::vector<int> xmap(nx + np);
    for (int q = 0; q < nx; q++) xmap[S.perm[q]] = q;
    for (int k = 0; k < np; k++) xmap[nx + k] = nx + k;

    std::vector<double> c2v(d->c2, d->c2 + nb), c1v(d->c1, d->c1 + nb);
    std::vector<int> flev_ptr(S.flev_ptr), blev_ptr(S.blev_ptr);
    RH_CUDA(g->upload(g->yp, S.yp));
    RH_CUDA(g->upload(g->yj, S.yj));
    RH_CUDA(g->upload(g->yrow, S.yrow));
    RH_CUDA(g->alloc(g->sc, 2 * (size_t)S.n_bus));
    RH_CUDA(g->upload(g->pf_wb, S.pf_wb));
    RH_CUDA(g->upload(g->ydiag, S.ydiag));
    RH_CUDA(g->upload(g->G, S.G));
    RH_CUDA(g->upload(g->B, S.B));
    RH_CUDA(g->upload(g->qth, S.qth));
    RH_CUDA(g->upload(g->qv, S.qv));
    RH_CUDA(g->upload(g->ip_v, S.ip_v));
    RH_CUDA(g->upload(g->ip_pg, S.ip_pg));
    RH_CUDA(g->upload(g->ix_th, S.ix_th));
    RH_CUDA(g->upload(g->ix_v, S.ix_v));
    RH_CUDA(g->upload(g->pg_slot, S.pg_slot));
    RH_CUDA(g->upload(g->jac_dst, S.jac_dst));
    RH_CUDA(g->upload(g->col_th, S.col_th));
    RH_CUDA(g->upload(g->col_v, S.col_v));
    RH_CUDA(g->upload(g->col_pg, S.col_pg));
    RH_CUDA(g->upload(g->c2, c2v));
    RH_CUDA(g->upload(g->c1, c1v));
    RH_CUDA(g->upload(g->rowptr, S.rowptr));
    RH_CUDA(g->upload(g->col, S.col));
    RH_CUDA(g->upload(g->diagpos, S.diagpos));
    RH_CUDA(g->upload(g->tpos, S.tpos));
    {
        std::vector<int> arow(S.col.size());
        for (int q = 0; q < S.n_x; q++)
            for (int e = S.rowptr[q]; e < S.rowptr[q + 1]; e++) arow[e] = q;
        RH_CUDA(g->upload(g->arow, arow));
    }
    RH_CUDA(g->upload(g->q0, S.q0));
    RH_CUDA(g->upload(g->nv, S.nv));
    RH_CUDA(g->upload(g->flev_ptr, flev_ptr));
    RH_CUDA(g->upload(g->flev_bus, S.flev_bus));
    RH_CUDA(g->upload(g->flev_maxext, S.flev_maxext));
    RH_CUDA(g->upload(g->blev_ptr, blev_ptr));
    RH_CUDA(g->upload(g->blev_bus, S.blev_bus));
    RH_CUDA(g->upload(g->blev_maxext, S.blev_maxext));
    {
        std::vector<int4> fs(S.n_elim), bs(S.n_elim);
        for (int t = 0; t < S.n_elim; t++) {
            int k = S.flev_bus[t], q = S.q0[k];
            bool two = S.nv[k] == 2;
            fs[t] = make_int4(q, S.diagpos[q] - S.rowptr[q], S.rowptr[q], two ? S.rowptr[q + 1] : -1);
            k = S.blev_bus[t];
            q = S.q0[k];
            two = S.nv[k] == 2;
            int ue0 = S.diagpos[q] + (two ? 2 : 1);
            bs[t] = make_int4(q, S.rowptr[q + 1] - ue0, ue0, two ? S.diagpos[q + 1] + 1 : -1);
        }
        RH_CUDA(g->upload(g->fslot, fs));
        RH_CUDA(g->upload(g->bslot, bs));
        // schedules restricted to the sparse part (buses before the dense tail)
        auto restrict_set = [&](const std::vector<int>& order, const std::vector<int>& lev, const std::vector<int4>& src,
                                std::vector<int>& ptr, std::vector<int4>& sl, std::vector<int>& mx,
                                const std::vector<char>* keep = nullptr) {
            ptr.assign(1, 0);
            int cur = -1;
            for (int t = 0; t < S.n_elim; t++) {
                int k = order[t];
                if (k >= S.tail_bus0 || (keep && !(*keep)[k])) continue;
                if (lev[k] != cur) {
                    if (cur >= 0) ptr.push_back((int)sl.size());
                    cur = lev[k];
                    mx.push_back(0);
                }
                sl.push_back(src[t]);
                mx.back() = std::max(mx.back(), src[t].y);
            }
            if (cur >= 0) ptr.push_back((int)sl.size());
        };
        std::vector<int> sfp, sbp, sfm, sbm;
        std::vector<int4> sfs, sbs;
        restrict_set(S.flev_bus, S.flevel, fs, sfp, sfs, sfm);
        restrict_set(S.blev_bus, S.blevel, bs, sbp, sbs, sbm);
        g->n_sf = (int)sfp.size() - 1;
        g->n_sb = (int)sbp.size() - 1;
        // HW = Y_p + J_p^T psi reads psi only at the rows of J_p, and the L^T sweep
        // computes a row from the rows of its ancestors: the other buses' rows of that
        // last sweep are never read
        {
            std::vector<char> need(S.n_elim, 0);
            for (int k = 0; k < S.n_elim; k++)
                for (int t = 0; t < S.nv[k]; t++)
                    if (S.jp_ptr[S.q0[k] + t + 1] > S.jp_ptr[S.q0[k] + t]) need[k] = 1;
            for (int k = 0; k < S.n_elim; k++)      // ancestors come later: one ascending pass closes the set
                if (need[k])
                    for (int c : S.colpat[k]) need[c] = 1;
            std::vector<int> rp, rm;
            std::vector<int4> rs;
            restrict_set(S.blev_bus, S.blevel, bs, rp, rs, rm, &need);
            g->n_sbr = (int)rp.size() - 1;
            RH_CUDA(g->upload(g->sbr_ptr, rp));
            RH_CUDA(g->upload(g->sbr_slot, rs));
            RH_CUDA(g->upload(g->sbr_maxext, rm));
        }
        // the tail's external phase: one level of tail buses, columns left of t0 only
        std::vector<int> efp(1, 0), efm;
        std::vector<int4> efs;
        for (int k = S.tail_bus0; k < S.n_elim; k++) {
            int q = S.q0[k];
            int n = 0;
            for (int t = S.rowptr[q]; t < S.diagpos[q] && S.col[t] < S.t0; t++) n++;
            efs.push_back(make_int4(q, n, S.rowptr[q], S.nv[k] == 2 ? S.rowptr[q + 1] : -1));
        }
        if (!efs.empty()) {
            efp.push_back((int)efs.size());
            int m = 0;
            for (auto& e : efs) m = std::max(m, e.y);
            efm.push_back(m);
        }
        g->n_ef = (int)efp.size() - 1;
        RH_CUDA(g->upload(g->sf_ptr, sfp));
        RH_CUDA(g->upload(g->sf_slot, sfs));
        RH_CUDA(g->upload(g->sf_maxext, sfm));
        RH_CUDA(g->upload(g->sb_ptr, sbp));
        RH_CUDA(g->upload(g->sb_slot, sbs));
        RH_CUDA(g->upload(g->sb_maxext, sbm));
        RH_CUDA(g->upload(g->ef_ptr, efp));
        RH_CUDA(g->upload(g->ef_slot, efs));
        RH_CUDA(g->upload(g->ef_maxext, efm));
        // dense tail: position of (t0 + i, t0 + j) in A, -1 where structurally zero
        int T = S.n_x - S.t0;
        std::vector<int> tp((size_t)T * T, -1);
        for (int i = 0; i < T; i++)
            for (int t = S.rowptr[S.t0 + i]; t < S.rowptr[S.t0 + i + 1]; t++)
                if (S.col[t] >= S.t0) tp[(size_t)i * T + (S.col[t] - S.t0)] = t;
        RH_CUDA(g->upload(g->tail_pos, tp));
        // bus structure by theta row for the reach-restricted forward sweep
        std::vector<int> qth(nx, 0), bpar(nx, -1);
        for (int k = 0; k < S.n_elim; k++) {
            int q = S.q0[k];
            for (int t = 0; t < S.nv[k]; t++) qth[q + t] = q;
            if (k < S.tail_bus0 && !S.colpat[k].empty()) {
                int par = S.colpat[k][0];              // first later bus of the pattern: the tree parent
                if (par < S.tail_bus0) bpar[q] = 2 * S.q0[par] + (S.nv[par] == 2 ? 1 : 0);
            }
        }
        RH_CUDA(g->upload(g->qtheta, qth));
        RH_CUDA(g->upload(g->bparent, bpar));
        size_t ntri = T > 1 ? (size_t)T * (T - 1) / 2 : 1;
        RH_CUDA(g->alloc(g->triL, ntri));
        RH_CUDA(g->alloc(g->triU, ntri));
        RH_CUDA(g->alloc(g->triUt, ntri));
        RH_CUDA(g->alloc(g->triLt, ntri));
        RH_CUDA(g->alloc(g->triLd, ntri));
        RH_CUDA(g->alloc(g->triUd, ntri));
        RH_CUDA(g->alloc(g->triUtd, ntri));
        RH_CUDA(g->alloc(g->triLtd, ntri));
    }
    RH_CUDA(g->upload(g->rf_lev_bus, S.rf_lev_bus));
    RH_CUDA(g->upload(g->rf_tgt_pos, S.rf_tgt_pos));
    RH_CUDA(g->upload(g->rf_grp, S.rf_grp));
    RH_CUDA(g->upload(g->rf_xptr, S.rf_xptr));
    RH_CUDA(g->upload(g->rf_xgrp, S.rf_xgrp));
    RH_CUDA(g->upload(g->rf_piv_bus, S.rf_piv_bus));
    RH_CUDA(g->upload(g->rf_piv_pos, S.rf_piv_pos));
    RH_CUDA(g->alloc(g->rf_piv, (size_t)S.tail_bus0));
    RH_CUDA(g->upload(g->rf_pe_bus, S.rf_pe_bus));
    RH_CUDA(g->upload(g->rf_pe_pos, S.rf_pe_ut));
    RH_CUDA(g->upload(g->jp_ptr, S.jp_ptr));
    {
        std::vector<int> rows, zero;
        for (int q = 0; q < nx; q++) (S.jp_ptr[q + 1] > S.jp_ptr[q] ? rows : zero).push_back(q);
        g->n_jp_rows = (int)rows.size();
        g->n_jp_zero = (int)zero.size();
        RH_CUDA(g->upload(g->jp_rows, rows));
        RH_CUDA(g->upload(g->jp_zero_rows, zero));
    }
    RH_CUDA(g->upload(g->jp_col, S.jp_col));
    RH_CUDA(g->upload(g->jpt_ptr, S.jpt_ptr));
    RH_CUDA(g->upload(g->jpt_row, S.jpt_row));
    RH_CUDA(g->upload(g->jpt_src, S.jpt_src));
    RH_CUDA(g->upload(g->hcolmap, g->colmap));
    RH_CUDA(g->upload(g->tp_bus, tp_bus));
    {
        // a sparse bus of forward level 0 has no L entries outside its block; for a PQ
        // bus the v row's only L entry is (v, theta), the first of the row
        std::vector<int> l0(nb, -1);
        for (int k = 0; k < S.tail_bus0; k++)
            if (S.flevel[k] == 0 && S.nv[k] == 2) l0[S.ebus[k]] = S.rowptr[S.q0[k] + 1];
        RH_CUDA(g->upload(g->tp_l0, l0));
    }
    RH_CUDA(g->upload(g->uth, uth));
    RH_CUDA(g->upload(g->uv, uv));
    RH_CUDA(g->upload(g->inc_ptr, inc_ptr));
    RH_CUDA(g->upload(g->inc_nb, inc_nb));
    RH_CUDA(g->upload(g->inc_uth, inc_uth));
    RH_CUDA(g->upload(g->inc_uv, inc_uv));
    RH_CUDA(g->upload(g->has_gref, has_gref));
    RH_CUDA(g->upload(g->pg_row, pg_row));
    RH_CUDA(g->upload(g->xmap, xmap));
    RH_CUDA(g->alloc(g->gref_row, g->n_gref));
    // state
    std::vector<double> ones(nb, 1.0);
    RH_CUDA(g->upload(g->vm, ones));
    RH_CUDA(g->alloc(g->va, nb));
    RH_CUDA(g->alloc(g->pg, nb));
    RH_CUDA(g->alloc(g->pd, nb));
    RH_CUDA(g->alloc(g->qd, nb));
    RH_CUDA(g->alloc(g->P, nb));
    RH_CUDA(g->alloc(g->Q, nb));
    RH_CUDA(g->alloc(g->A, S.col.size()));
    RH_CUDA(g->alloc(g->At, S.col.size()));
    RH_CUDA(g->alloc(g->Ad, S.col.size()));
    RH_CUDA(g->alloc(g->Atd, S.col.size()));
    RH_CUDA(g->alloc(g->invdiag, nx));
    RH_CUDA(g->alloc(g->jpv, S.jp_col.size()));
    RH_CUDA(g->alloc(g->jptv, S.jp_col.size()));
    RH_CUDA(g->alloc(g->jptvd, S.jp_col.size()));
    RH_CUDA(g->alloc(g->gres, nx));
    RH_CUDA(g->alloc(g->lam, nx));
    RH_CUDA(g->alloc(g->grad, np));
    RH_CUDA(g->alloc(g->rto_y, np));
    RH_CUDA(g->alloc(g->tailD, (size_t)(S.n_x - S.t0) * (S.n_x - S.t0)));
    RH_CUDA(g->alloc(g->v1, g->rows()));
    RH_CUDA(g->alloc(g->inc_coef, g->n_inc));
    RH_CUDA(g->alloc(g->d2, nb));
    RH_CUDA(g->alloc(g->asum, nb));
    RH_CUDA(g->alloc(g->csum, nb));
    RH_CUDA(g->alloc(g->pg_curv, nb));
    RH_CUDA(g->alloc(g->gref_th, nb));
    RH_CUDA(g->alloc(g->gref_v, nb));
    RH_CUDA(g->alloc(g->gref_val, g->n_gref));
    RH_CUDA(g->alloc(g->tmp_bus, 4 * (size_t)nb));
    RH_CUDA(g->alloc(g->pbuf, np));
    RH_CUDA(g->alloc(g->xbuf, nx));
    RH_CUDA(g->alloc(g->dscal, 4));
    RH_CUDA(g->alloc(g->umax, 2));
    RH_CUDA(g->alloc(g->err, 1));
    RH_CUDA(cudaDeviceSynchronize());
    *out = g.release();
    return RH_OK;
}

void rh_grid_destroy(rh_grid* g) {
    if (!g) return;
    if (g->device >= 0) cudaSetDevice(g->device);
    delete g;
}

rh_status rh_grid_dims(const rh_grid* g, rh_dims* o) {
    if (!g || !o) return fail(RH_EINVAL, "NULL argument");
    const auto& S = g->S;
    o->n_bus = S.n_bus; o->n_branch = S.n_branch; o->n_gen = S.n_gen; o->n_pv = S.n_pv; o->n_pq = S.n_pq;
    o->n_x = S.n_x; o->n_p = S.n_p; o->n_levels_fwd = S.n_flev; o->n_levels_bwd = S.n_blev;
    o->nnz_jx = S.nnz_jx; o->nnz_jp = (int64_t)S.jp_col.size();
    o->nnz_l = S.nnz_l; o->nnz_u = S.nnz_u;
    o->refactor_updates = S.rf_updates;
    o->setup_kernels = g->adj_kernels;
    o->hessian_kernels = g->hess_kernels;
    o->max_tail = S.max_tail;
    o->tail_vars = S.n_x - S.t0;
    return RH_OK;
}

rh_status rh_grid_symbolic(const rh_grid* g, int32_t* perm, int32_t* bus_order, int32_t* level, int32_t* Lp,
                           int32_t* Lj, int32_t* Up, int32_t* Uj) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    const auto& S = g->S;
    if (perm) for (int q = 0; q < S.n_x; q++) perm[q] = S.perm[q];
    if (bus_order) for (int k = 0; k < S.n_elim; k++) bus_order[k] = S.ebus[k];
    if (level) for (int k = 0; k < S.n_elim; k++) level[k] = S.flevel[k];
    int64_t nl = 0, nu = 0;
    for (int q = 0; q < S.n_x; q++) {
        if (Lp) Lp[q] = (int32_t)nl;
        if (Up) Up[q] = (int32_t)nu;
        for (int s = S.rowptr[q]; s < S.diagpos[q]; s++) { if (Lj) Lj[nl] = S.col[s]; nl++; }
        for (int s = S.diagpos[q]; s < S.rowptr[q + 1]; s++) { if (Uj) Uj[nu] = S.col[s]; nu++; }
    }
    if (Lp) Lp[S.n_x] = (int32_t)nl;
    if (Up) Up[S.n_x] = (int32_t)nu;
    return RH_OK;
}

rh_status rh_injections(rh_grid* g, const double* vm, const double* va, double* P, double* Q) {
    if (!g || !vm || !va || !P || !Q) return fail(RH_EINVAL, "NULL argument");
    rh_status st = set_device(g);
    if (st) return st;
    int nb = g->S.n_bus;
    rh::PfState s = g->st();
    s.vm = g->tmp_bus; s.va = g->tmp_bus + nb; s.P = g->tmp_bus + 2 * nb; s.Q = g->tmp_bus + 3 * nb;
    RH_CUDA(cudaMemcpyAsync(s.vm, vm, nb * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    RH_CUDA(cudaMemcpyAsync(s.va, va, nb * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    rh::launch_injections(g->pf(), s, g->stream);
    RH_CUDA(cudaGetLastError());
    RH_CUDA(cudaMemcpyAsync(P, s.P, nb * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    RH_CUDA(cudaMemcpyAsync(Q, s.Q, nb * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    RH_CUDA(cudaStreamSynchronize(g->stream));
    return RH_OK;
}

rh_status rh_set_state(rh_grid* g, const double* p, const double* pd, const double* qd) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    rh_status st = set_device(g);
    if (st) return st;
    int nb = g->S.n_bus;
    if (p) RH_CUDA(cudaMemcpyAsync(g->pbuf, p, g->S.n_p * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    if (pd) RH_CUDA(cudaMemcpyAsync(g->pd, pd, nb * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    if (qd) RH_CUDA(cudaMemcpyAsync(g->qd, qd, nb * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    k_set_p<<<nblk(nb, 128), 128, 0, g->stream>>>(nb, g->ip_v, g->ip_pg, g->pbuf, g->vm, g->pg);
    RH_CUDA(cudaGetLastError());
    RH_CUDA(cudaStreamSynchronize(g->stream));
    g->adjoint_ready = false;
    return RH_OK;
}

rh_status rh_powerflow(rh_grid* g, const double* x0, double tol, int32_t max_iter, double* x_out, int32_t* iters,
                       double* resid) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    if (!(tol >= 0.0) || max_iter < 0) return fail(RH_EINVAL, "tol must be >= 0 and max_iter >= 0");
    rh_status st = set_device(g);
    if (st) return st;
    const auto& S = g->S;
    int nb = S.n_bus, nx = S.n_x;
    cudaStream_t s = g->stream;
    g->adjoint_ready = false;
    if (x0) {
        RH_CUDA(cudaMemcpyAsync(g->xbuf, x0, nx * sizeof(double), cudaMemcpyHostToDevice, s));
        k_set_x<<<nblk(nb, 128), 128, 0, s>>>(nb, g->ix_th, g->ix_v, g->xbuf, g->vm, g->va);
    }
    // An iteration's device work is replayed from two graphs captured once per grid
    // (a few dozen launches on the host otherwise): the refactorisation with its factor
    // copies, after which the host reads the pivot flag, and the Newton step, the update
    // and the next assembly, after which it reads the residual.  The assembly clears the
    // pivot flag, so the flag is read between the two.
    if (!g->nt_fac_exec) {
        int nk = 0;
        st = capture_graph(
            g,
            [&]() -> rh_status {
                RH_CUDA(rh::launch_refactor(g->rf(), S.rf_lev_ptr.data(), S.rf_tgt_lev_ptr.data(),
                                            S.rf_piv_lev_ptr.data(), S.rf_n_lev, g->stream));
                enqueue_factor_copies(g, g->stream);
                RH_CUDA(cudaGetLastError());
                return RH_OK;
            },
            &g->nt_fac_exec, &nk);
        if (st) return st;
    }
    if (!g->nt_step_exec) {
        int nk = 0;
        st = capture_graph(
            g,
            [&]() -> rh_status {
                RH_CUDA(cudaMemcpyAsync(g->v1, g->gres, nx * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
                rh_status ss = solve_one(g, rh::PH_L | rh::PH_U, g->stream);
                if (ss) return ss;
                rh::launch_newton_update(g->pf(), g->st(), g->v1, g->stream);
                return assemble(g, g->jac_method, g->gres, g->stream);
            },
            &g->nt_step_exec, &nk);
        if (st) return st;
    }
    auto read_residual = [&](double* r) -> rh_status {
        unsigned long long bits = 0;
        RH_CUDA(cudaMemcpyAsync(&bits, g->umax, sizeof(bits), cudaMemcpyDeviceToHost, s));
        RH_CUDA(cudaStreamSynchronize(s));
        std::memcpy(r, &bits, sizeof(*r));
        if (nx == 0) *r = 0.0;
        return RH_OK;
    };
    int it = 0;
    double res = INFINITY;
    rh_status out = RH_ENOCONV;
    st = assemble(g, g->jac_method, g->gres, s);
    if (st) return st;
    st = read_residual(&res);
    if (st) return st;
    for (;;) {
        if (res <= tol) { out = RH_OK; break; }
        if (it >= max_iter || !std::isfinite(res)) break;
        RH_CUDA(cudaGraphLaunch(g->nt_fac_exec, s));
        st = check_err_flag(g);
        if (st) return st;
        RH_CUDA(cudaGraphLaunch(g->nt_step_exec, s));
        st = read_residual(&res);
        if (st) return st;
        it++;
    }
    if (iters) *iters = it;
    if (resid) *resid = res;
    if (x_out) {
        k_get_x<<<nblk(nb, 128), 128, 0, s>>>(nb, g->ix_th, g->ix_v, g->vm, g->va, g->xbuf);
        RH_CUDA(cudaGetLastError());
        RH_CUDA(cudaMemcpyAsync(x_out, g->xbuf, nx * sizeof(double), cudaMemcpyDeviceToHost, s));
        RH_CUDA(cudaStreamSynchronize(s));
    }
    if (out != RH_OK) return fail(out, "Newton did not reach the tolerance");
    return RH_OK;
}

rh_status rh_refactor(rh_grid* g, double* A_out) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    rh_status st = set_device(g);
    if (st) return st;
    g->adjoint_ready = false;
    st = assemble_and_factor(g);
    if (st) return st;
    if (A_out) {
        RH_CUDA(cudaMemcpyAsync(A_out, g->A, sizeof(double) * g->S.col.size(), cudaMemcpyDeviceToHost, g->stream));
        RH_CUDA(cudaStreamSynchronize(g->stream));
    }
    return RH_OK;
}

// Device work of rh_adjoint: a1 (Jacobian), a2 (refactor), a3 (adjoint, gradient,
// projection coefficients).  Enqueue only; captured once per grid into a graph.
}  // extern "C"

namespace {

// The adjoint (eq. 7) on the current factors: right-hand side and F, the transposed
// single solve, lambda, the projection coefficients and grad F (enqueue only).
rh_status enqueue_adjoint_chain(rh_grid* g, cudaStream_t s, bool beside_dirs) {
    const auto& S = g->S;
    RH_CUDA(cudaMemsetAsync(g->v1, 0, sizeof(double) * g->rows(), s));
    rh::AdjData a;
    a.rhs = g->v1; a.cref = g->dscal; a.c2ref = g->dscal + 1; a.F = g->dscal + 2;
    a.gref_th = g->gref_th; a.gref_v = g->gref_v; a.gref_row = g->gref_row; a.gref_val = g->gref_val;
    a.n_gref = g->n_gref; a.uth = g->uth; a.uv = g->uv;
    rh::launch_adjoint_rhs(g->pf(), g->st(), a, s);
    rh_status st = solve_one(g, rh::PH_UT | rh::PH_LT, s, beside_dirs);
    if (st) return st;
    RH_CUDA(cudaMemcpyAsync(g->lam, g->v1, S.n_x * sizeof(double), cudaMemcpyDeviceToDevice, s));
    rh::launch_adjoint_coef(g->pf(), g->st(), g->lam, g->dscal, g->inc_ptr, g->inc_nb, g->inc_coef, g->d2, g->asum,
                            g->csum, g->pg_curv, s);
    rh::launch_gradient(g->pf(), g->st(), S.n_p, g->jpt_ptr, g->jpt_row, g->jptv, g->lam, g->dscal, g->gref_v,
                        g->grad, s);
    RH_CUDA(cudaGetLastError());
    return RH_OK;
}

rh_status enqueue_adjoint(rh_grid* g) {
    rh_status st = enqueue_factor(g);
    if (st) return st;
    return enqueue_adjoint_chain(g, g->stream, false);
}


// CTAs of rh_reduced_hessian's first direction launch: the fewest with the directions
// per CTA of a launch one slot short of full; the slots left over (7 SMs' worth for the
// 9241-bus grid) are the adjoint branch's
int first_launch_ctas(int np) {
    const int per = (np + rh::dirs_cta_slots() - 2) / (rh::dirs_cta_slots() - 1);
    return std::min(rh::dirs_default_ctas(np), std::max(1, (np + per - 1) / per));
}

// rh_reduced_hessian's device work.  After the factorisation the adjoint chain
// forks onto stream2 (its single solve as one direction CTA) while
// the direction kernel runs SpMul and the L and U sweeps on fewer CTAs than the
// device holds, so the two run at once; after the join a second direction launch
// runs the projection, the transposed sweeps and SpMulAdd.  The directions of the
// two launches are independent columns of V, so their CTA counts may differ.
rh_status enqueue_reduced_hessian(rh_grid* g, double* Hd, int64_t lh) {
    const int np = g->S.n_p;
    rh_status st = enqueue_factor(g);
    if (st) return st;
    RH_CUDA(cudaEventRecord(g->ev_fork, g->stream));
    RH_CUDA(cudaStreamWaitEvent(g->stream2, g->ev_fork, 0));
    st = enqueue_adjoint_chain(g, g->stream2, true);
    if (st) return st;
    RH_CUDA(cudaEventRecordWithFlags(g->ev_d0, g->stream, cudaEventRecordExternal));
    st = dirs(g, np, np, g->V, g->T, nullptr, 0, 0, Hd, lh, rh::PH_WLOAD | rh::PH_SPMUL | rh::PH_L | rh::PH_U,
              g->stream, first_launch_ctas(np));
    if (st) return st;
    RH_CUDA(cudaEventRecordWithFlags(g->ev_v, g->stream, cudaEventRecordExternal));
    RH_CUDA(cudaEventRecordWithFlags(g->ev_c, g->stream2, cudaEventRecordExternal));
    RH_CUDA(cudaEventRecord(g->ev_join, g->stream2));
    RH_CUDA(cudaStreamWaitEvent(g->stream, g->ev_join, 0));
    // the second launch on balanced CTAs (every CTA the same number of directions)
    st = dirs(g, np, np, g->V, g->T, nullptr, 0, 0, Hd, lh, rh::PH_TPROJ | rh::PH_UT | rh::PH_LT | rh::PH_MULADD,
              g->stream);
    if (st) return st;
    RH_CUDA(cudaEventRecordWithFlags(g->ev_d1, g->stream, cudaEventRecordExternal));
    return RH_OK;
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// One half of a batched Newton iteration for the items whose bit is set in `mask`
// (enqueue only, on items[0]'s stream).  Phase 0: zero A and the maxima, residual
// and Jacobians of every item, and their max |g| and pivot flags copied to the host.
// Phase 1: refactorisation, the single solves' tail triangles, the Newton step
// J_x dx = g and x -= dx.
rh_status enqueue_batch_newton(rh_grid* const* items, int n, uint32_t mask, int phase) {
    rh_grid* g0 = items[0];
    const auto& S = g0->S;
    cudaStream_t s = g0->stream;
    std::vector<rh_grid*> act;
    for (int i = 0; i < n; i++)
        if (mask & (1u << i)) act.push_back(items[i]);
    if (act.empty()) return RH_OK;
    std::unique_ptr<rh::PfBatch> B(new rh::PfBatch());
    B->n = (int)act.size();
    B->max_bus = S.n_bus;
    for (int k = 0; k < B->n; k++) {
        rh_grid* g = act[k];
        rh::PfBatchItem& it = B->it[k];
        it.g = g->pf();
        it.s = g->st();
        it.A = g->A;
        it.jpv = g->jpv;
        it.x = g->v1;
        it.umax = g->umax;
        it.err = g->err;
    }
    if (phase == 0) {
        rh::launch_pf_prep_batch(*B, s);
        rh::launch_pf_eval_batch(*B, s);
        rh::launch_batch_status(*B, g0->bstat_d, s);
        RH_CUDA(cudaMemcpyAsync(g0->bstat_h, g0->bstat_d, 2 * sizeof(double) * B->n, cudaMemcpyDeviceToHost, s));
        RH_CUDA(cudaGetLastError());
        return RH_OK;
    }
    for (rh_grid* g : act) RH_CUDA(cudaMemsetAsync(g->err, 0, sizeof(int), s));
    std::unique_ptr<rh::RfBatch> R(new rh::RfBatch());
    R->n = B->n;
    for (int k = 0; k < B->n; k++) R->g[k] = act[k]->rf();
    RH_CUDA(rh::launch_refactor_batch(*R, S.rf_lev_ptr.data(), S.rf_tgt_lev_ptr.data(), S.rf_piv_lev_ptr.data(), S.rf_n_lev, s));
    const int T = S.n_x - S.t0;
    const int mode = rh::solve1_mode(S.n_x, T);
    if (mode == 2) {
        std::unique_ptr<rh::TriBatch> tb(new rh::TriBatch());
        tb->n = B->n;
        tb->T = T;
        tb->t0 = S.t0;
        for (int k = 0; k < B->n; k++) {
            tb->pos[k] = act[k]->tail_pos;
            tb->A[k] = act[k]->A;
            tb->invdiag[k] = act[k]->invdiag;
            tb->triL[k] = act[k]->triL;
            tb->triU[k] = act[k]->triU;
        }
        rh::launch_tail_tri_batch(*tb, s);
    }
    if (mode > 0) {
        std::unique_ptr<rh::Solve1Batch> sb(new rh::Solve1Batch());
        sb->n = B->n;
        for (int k = 0; k < B->n; k++) {
            sb->g[k] = act[k]->dir();
            sb->x[k] = act[k]->v1;
        }
        RH_CUDA(rh::launch_solve1_batch(*sb, rh::PH_L | rh::PH_U, mode == 2, S.n_x, T, s));
    } else {
        // x does not fit in one CTA's shared memory: the direction kernel solves each item
        for (rh_grid* g : act) {
            enqueue_factor_copies(g, s);
            rh_status st = solve_one(g, rh::PH_L | rh::PH_U, s);
            if (st) return st;
        }
    }
    rh::launch_newton_update_batch(*B, s);
    RH_CUDA(cudaGetLastError());
    return RH_OK;
}

}  // namespace

extern "C" {

rh_status rh_batch_powerflow(int32_t n_items, rh_grid* const* grids, const double* const* x0, double tol,
                             int32_t max_iter, double* const* x_out, int32_t* iters, double* resid,
                             int32_t* status) {
    if (n_items < 0 || n_items > rh::kMaxPfBatch || (n_items > 0 && !grids))
        return fail(RH_EINVAL, "n_items must be in [0, 32] and grids non-NULL");
    if (!(tol >= 0.0) || max_iter < 0) return fail(RH_EINVAL, "tol must be >= 0 and max_iter >= 0");
    if (n_items == 0) return RH_OK;
    rh_grid* g0 = grids[0];
    for (int i = 0; i < n_items; i++) {
        if (!grids[i]) return fail(RH_EINVAL, "item " + std::to_string(i) + ": NULL grid");
        if (grids[i]->device < 0) return fail(RH_ESTATE, "item " + std::to_string(i) + ": symbolic-only grid");
        if (grids[i]->device != g0->device || grids[i]->topo_hash != g0->topo_hash)
            return fail(RH_EINVAL, "item " + std::to_string(i) + ": not the same topology and device as item 0");
        for (int j = 0; j < i; j++)
            if (grids[j] == grids[i]) return fail(RH_EINVAL, "a grid appears twice");
    }
    rh_status st = set_device(g0);
    if (st) return st;
    const auto& S = g0->S;
    cudaStream_t s = g0->stream;
    if (!g0->bstat_d) RH_CUDA(g0->alloc(g0->bstat_d, 2 * rh::kMaxPfBatch));
    if (!g0->bstat_h) RH_CUDA(cudaMallocHost(&g0->bstat_h, 2 * rh::kMaxPfBatch * sizeof(double)));
    // earlier work of every item is done; then the starting points and clean pivot flags
    for (int i = 0; i < n_items; i++) {
        rh_grid* g = grids[i];
        RH_CUDA(cudaStreamSynchronize(g->stream));
        g->adjoint_ready = false;
        if (x0 && x0[i]) {
            RH_CUDA(cudaMemcpyAsync(g->xbuf, x0[i], S.n_x * sizeof(double), cudaMemcpyHostToDevice, s));
            k_set_x<<<nblk(S.n_bus, 128), 128, 0, s>>>(S.n_bus, g->ix_th, g->ix_v, g->xbuf, g->vm, g->va);
        }
        RH_CUDA(cudaMemsetAsync(g->err, 0, sizeof(int), s));
    }
    RH_CUDA(cudaGetLastError());
    std::vector<int> it(n_items, 0), stat(n_items, RH_ENOCONV);
    std::vector<double> res(n_items, INFINITY);
    uint32_t mask = n_items == 32 ? 0xffffffffu : ((1u << n_items) - 1u);
    // the graph of one phase for one set of items, captured once and replayed
    auto run = [&](uint32_t m, int phase) -> rh_status {
        std::string key = std::to_string(phase) + ":" + std::to_string(m);
        for (int i = 0; i < n_items; i++) key += ":" + std::to_string(grids[i]->uid);
        auto f = g0->pf_graphs.find(key);
        if (f == g0->pf_graphs.end()) {
            cudaGraphExec_t ex = nullptr;
            int nk = 0;
            rh_status cs = capture_graph(g0, [&] { return enqueue_batch_newton(grids, n_items, m, phase); }, &ex, &nk);
            if (cs) return cs;
            f = g0->pf_graphs.emplace(key, ex).first;
        }
        RH_CUDA(cudaGraphLaunch(f->second, s));
        return RH_OK;
    };
    while (mask) {
        st = run(mask, 0);
        if (st) return st;
        RH_CUDA(cudaStreamSynchronize(s));          // the one host sync of the iteration
        uint32_t next = 0;
        for (int i = 0, k = 0; i < n_items; i++) {
            if (!(mask & (1u << i))) continue;
            double r = g0->bstat_h[2 * k];
            const bool singular = g0->bstat_h[2 * k + 1] != 0.0;
            k++;
            if (S.n_x == 0) r = 0.0;
            res[i] = r;
            if (singular) stat[i] = RH_ESINGULAR;
            else if (r <= tol) stat[i] = RH_OK;
            else if (it[i] >= max_iter || !std::isfinite(r)) stat[i] = RH_ENOCONV;
            else next |= 1u << i;
        }
        mask = next;
        if (!mask) break;
        st = run(mask, 1);
        if (st) return st;
        for (int i = 0; i < n_items; i++)
            if (mask & (1u << i)) it[i]++;
    }
    rh_status worst = RH_OK;
    for (int i = 0; i < n_items; i++) {
        rh_grid* g = grids[i];
        if (iters) iters[i] = it[i];
        if (resid) resid[i] = res[i];
        if (status) status[i] = stat[i];
        if (stat[i] == RH_ESINGULAR) worst = RH_ESINGULAR;
        else if (stat[i] == RH_ENOCONV && worst == RH_OK) worst = RH_ENOCONV;
        if (x_out && x_out[i]) {
            k_get_x<<<nblk(S.n_bus, 128), 128, 0, s>>>(S.n_bus, g->ix_th, g->ix_v, g->vm, g->va, g->xbuf);
            RH_CUDA(cudaGetLastError());
            RH_CUDA(cudaMemcpyAsync(x_out[i], g->xbuf, S.n_x * sizeof(double), cudaMemcpyDeviceToHost, s));
        }
    }
    RH_CUDA(cudaStreamSynchronize(s));
    if (worst == RH_ESINGULAR) return fail(worst, "a static pivot below 1e-14 max|J_x| (see status[])");
    if (worst == RH_ENOCONV) return fail(worst, "Newton did not reach the tolerance for every item (see status[])");
    return RH_OK;
}

rh_status rh_adjoint(rh_grid* g, double* F, double* lambda, double* grad) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    rh_status st = set_device(g);
    if (st) return st;
    const auto& S = g->S;
    cudaStream_t s = g->stream;
    g->adjoint_ready = false;
    if (!g->adj_exec) {
        st = capture_graph(g, [&] { return enqueue_adjoint(g); }, &g->adj_exec, &g->adj_kernels);
        if (st) return st;
    }
    RH_CUDA(cudaGraphLaunch(g->adj_exec, s));
    if (lambda) {
        rh::launch_gather_rows(S.n_x, 1, g->xmap, g->lam, 1, g->xbuf, S.n_x, 1.0, S.n_x, s);
        RH_CUDA(cudaMemcpyAsync(lambda, g->xbuf, S.n_x * sizeof(double), cudaMemcpyDeviceToHost, s));
    }
    if (grad) RH_CUDA(cudaMemcpyAsync(grad, g->grad, S.n_p * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (F) RH_CUDA(cudaMemcpyAsync(F, g->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
    st = check_err_flag(g);   // synchronises the stream
    if (st) return st;
    g->adjoint_ready = true;
    return RH_OK;
}

rh_status rh_reduced_hessian(rh_grid* g, double* H, int64_t ldh, double* F, double* grad, void* stream,
                             uint32_t flags) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    const auto& S = g->S;
    if (!H || ldh < S.n_p) return fail(RH_EINVAL, "bad H or leading dimension");
    rh_status st = set_device(g);
    if (st) return st;
    const int np = S.n_p;
    const bool host = !(flags & RH_DEVICE_PTRS);
    double* Hd = H;
    int64_t lh = ldh;
    if (host) {
        st = ensure_stage(g, (size_t)np * np);
        if (st) return st;
        Hd = g->stage_out;
        lh = np;
    }
    st = ensure_ws(g, (size_t)np);
    if (st) return st;
    g->adjoint_ready = false;
    g->hess_timed = false;
    if (g->hess_exec && (g->hess_H != Hd || g->hess_ld != lh || g->hess_V != g->V || g->hess_T != g->T)) {
        cudaGraphExecDestroy(g->hess_exec);
        g->hess_exec = nullptr;
    }
    if (!g->hess_exec) {
        // the first launch's reach schedule is built here: the capture cannot allocate
        rh::ReachSched* rs = nullptr;
        st = reach_schedule(g, first_launch_ctas(np), &rs);
        if (st) return st;
        if (!g->stream2) RH_CUDA(cudaStreamCreateWithFlags(&g->stream2, cudaStreamNonBlocking));
        if (!g->ev_fork) RH_CUDA(cudaEventCreateWithFlags(&g->ev_fork, cudaEventDisableTiming));
        if (!g->ev_join) RH_CUDA(cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming));
        if (!g->ev_d0) RH_CUDA(cudaEventCreate(&g->ev_d0));
        if (!g->ev_d1) RH_CUDA(cudaEventCreate(&g->ev_d1));
        if (!g->ev_v) RH_CUDA(cudaEventCreate(&g->ev_v));
        if (!g->ev_c) RH_CUDA(cudaEventCreate(&g->ev_c));
        st = capture_graph(g, [&] { return enqueue_reduced_hessian(g, Hd, lh); }, &g->hess_exec, &g->hess_kernels);
        if (st) return st;
        g->hess_H = Hd;
        g->hess_ld = lh;
        g->hess_V = g->V;
        g->hess_T = g->T;
    }
    if (stream) {   // order after the caller's earlier work on its stream
        if (!g->ev_user) RH_CUDA(cudaEventCreateWithFlags(&g->ev_user, cudaEventDisableTiming));
        RH_CUDA(cudaEventRecord(g->ev_user, (cudaStream_t)stream));
        RH_CUDA(cudaStreamWaitEvent(g->stream, g->ev_user, 0));
    }
    RH_CUDA(cudaGraphLaunch(g->hess_exec, g->stream));
    if (host)
        RH_CUDA(cudaMemcpy2DAsync(H, ldh * sizeof(double), Hd, lh * sizeof(double), np * sizeof(double), np,
                                  cudaMemcpyDeviceToHost, g->stream));
    if (grad) RH_CUDA(cudaMemcpyAsync(grad, g->grad, np * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    if (F) RH_CUDA(cudaMemcpyAsync(F, g->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    st = check_err_flag(g);   // synchronises the stream
    if (st) return st;
    g->adjoint_ready = true;
    g->hess_timed = true;
    return RH_OK;
}

rh_status rh_reduced_hessian_times(const rh_grid* g, float* ms) {
    if (!g || !ms) return fail(RH_EINVAL, "NULL grid or ms");
    if (!g->hess_timed) return fail(RH_ESTATE, "no completed rh_reduced_hessian call on this grid");
    RH_CUDA(cudaEventElapsedTime(ms, g->ev_d0, g->ev_d1));
    RH_CUDA(cudaEventElapsedTime(ms + 1, g->ev_d0, g->ev_v));
    RH_CUDA(cudaEventElapsedTime(ms + 2, g->ev_d0, g->ev_c));
    return RH_OK;
}

rh_status rh_reduced_hessian_flops(const rh_grid* g, int32_t n_sm, double* algorithmic, double* executed) {
    if (!g || !algorithmic || !executed) return fail(RH_EINVAL, "NULL argument");
    const auto& S = g->S;
    if (n_sm <= 0) {
        if (g->device < 0) return fail(RH_EINVAL, "n_sm must be given for a symbolic-only grid");
        RH_CUDA(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, g->device));
    }
    const int np = S.n_p, T = S.n_x - S.t0;
    // incidences (off-diagonal admittance entries) and the slack-gradient entries
    int64_t n_inc = 0;
    for (int i = 0; i < S.n_bus; i++) n_inc += S.yp[i + 1] - S.yp[i] - 1;
    const int deg_ref = S.yp[S.ref + 1] - S.yp[S.ref] - 1;
    const int n_gref = 1 + 2 * deg_ref;
    // the CTA counts of the two direction launches (as rh_reduced_hessian launches them)
    const int slots = rh::dirs_cta_slots_for(n_sm);
    const int per = (np + slots - 2) / std::max(1, slots - 1);
    const int n_cta2 = rh::dirs_ctas_for(np, slots);
    const int n_cta1 = std::min(n_cta2, std::max(1, (np + std::max(1, per) - 1) / std::max(1, per)));
    const bool tailed = rh::dirs_tail_fits(T, np, n_cta1) && rh::dirs_tail_fits(T, np, n_cta2);
    // FMAs of bus block k in a forward / backward sweep: both rows' parts outside the
    // bus, plus the (v, theta) entry of a PQ bus
    auto fwd_fma = [&](int k) {
        const int q = S.q0[k];
        return (int64_t)S.nv[k] * (S.diagpos[q] - S.rowptr[q]) + (S.nv[k] == 2 ? 1 : 0);
    };
    auto bwd_fma = [&](int k) {
        const int q = S.q0[k];
        return (int64_t)S.nv[k] * (S.rowptr[q + 1] - S.diagpos[q] - S.nv[k]) + (S.nv[k] == 2 ? 1 : 0);
    };
    const int sparse_end = tailed ? S.tail_bus0 : S.n_elim;
    int64_t ext = 0, tail = 0;   // the tail rows' part left of the tail (its external phase); one dense tail solve
    if (tailed) {
        for (int k = S.tail_bus0; k < S.n_elim; k++) {
            const int q = S.q0[k];
            int n = 0;
            for (int t = S.rowptr[q]; t < S.diagpos[q] && S.col[t] < S.t0; t++) n++;
            ext += (int64_t)S.nv[k] * n;
        }
        tail = (int64_t)T * (T - 1) / 2;
    }
    std::vector<char> need(S.n_elim, 0);     // buses whose psi rows SpMulAdd reads, and their ancestors
    for (int k = 0; k < S.n_elim; k++)
        for (int t = 0; t < S.nv[k]; t++)
            if (S.jp_ptr[S.q0[k] + t + 1] > S.jp_ptr[S.q0[k] + t]) need[k] = 1;
    for (int k = 0; k < S.n_elim; k++)
        if (need[k])
            for (int c : S.colpat[k]) need[c] = 1;
    int64_t l_all = 0, u_all = 0, ut = 0, lt = 0, fold = 0;
    const bool fold_ut = tailed && S.tail_bus0 > 0;
    for (int k = 0; k < sparse_end; k++) {
        l_all += fwd_fma(k);
        u_all += bwd_fma(k);
        if (fold_ut && S.flevel[k] == 0) fold += S.nv[k] == 2 ? 1 : 0;   // done by the projection
        else ut += fwd_fma(k);
        if (!tailed || need[k]) lt += bwd_fma(k);
    }
    // the projection, per direction: 3 + 3 flops per bus, 8 per incidence, 4 per bus next to the
    // slack, 2 n_gref + 1 for the slack term, 1 per Pg row, 2 per PQ bus of level 0 (the folded
    // first level of the U'^T sweep)
    const double proj = 6.0 * S.n_bus + 8.0 * n_inc + 4.0 * (1 + deg_ref) + 2.0 * n_gref + 1.0 + S.n_pv + 2.0 * fold;
    const double nnz_jp = (double)S.jp_col.size();
    const double l2 = proj + 2.0 * (ut + ext + 2 * tail + lt) + 2.0 * nnz_jp;
    // launch 1 (identity W): the L sweep over each CTA's reach, the buses of its J_p columns and
    // their ancestors in the sparse part (all buses without the dense tail), then the tail's
    // external phase, the two tail solves and the U sweep
    double l1 = 0.0;
    std::vector<int> bpos(S.n_x);
    for (int k = 0; k < S.n_elim; k++)
        for (int t = 0; t < S.nv[k]; t++) bpos[S.q0[k] + t] = k;
    std::vector<char> in(S.n_elim);
    for (int c = 0; c < n_cta1 && np > 0; c++) {
        const int c0 = (int)((int64_t)c * np / n_cta1), c1 = (int)((int64_t)(c + 1) * np / n_cta1);
        int64_t l = l_all;
        if (tailed) {
            std::fill(in.begin(), in.end(), 0);
            for (int j = c0; j < c1; j++) {    // the launch's columns, in the tree order
                const int col = g->colmap[j];
                for (int t = S.jpt_ptr[col]; t < S.jpt_ptr[col + 1]; t++) in[bpos[S.jpt_row[t]]] = 1;
            }
            l = 0;
            for (int k = 0; k < S.tail_bus0; k++) {
                if (!in[k]) continue;
                l += fwd_fma(k);
                if (!S.colpat[k].empty() && S.colpat[k][0] < S.tail_bus0) in[S.colpat[k][0]] = 1;
            }
        }
        l1 += (double)(c1 - c0) * 2.0 * (l + ext + 2 * tail + u_all);
    }
    *executed = l1 + np * l2;
    // Algorithm 2 for a dense W on the unit-diagonal factors, per direction: SpMul and
    // SpMulAdd (2 nnz(J_p) each), four sweeps (2 nnz(L) and 2 (nnz(U) - n_x) each), the
    // projection (8 per incidence and per bus, 4 per slack-gradient entry, 1 per Pg row)
    const double sweeps = 2.0 * (2.0 * S.nnz_l + 2.0 * (S.nnz_u - S.n_x));
    *algorithmic = (double)np * (4.0 * nnz_jp + sweeps + 8.0 * n_inc + 8.0 * S.n_bus + 4.0 * n_gref + S.n_pv);
    return RH_OK;
}

rh_status rh_hessvec(rh_grid* g, const double* W, int64_t ldw, int32_t N, double* HW, int64_t ldhw, void* stream,
                     uint32_t flags) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    if (N < 0) return fail(RH_EINVAL, "N must be >= 0");
    if (N == 0) return RH_OK;
    const auto& S = g->S;
    if (!W || !HW || ldw < S.n_p || ldhw < S.n_p) return fail(RH_EINVAL, "bad W / HW or leading dimension");
    if (!g->adjoint_ready) return fail(RH_ESTATE, "rh_hessvec needs rh_adjoint for the current state");
    rh_status st = set_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const double* Wd = W;
    double* HWd = HW;
    int64_t lw = ldw, lh = ldhw;
    bool host = !(flags & RH_DEVICE_PTRS);
    if (host) {
        st = ensure_stage(g, (size_t)S.n_p * N);
        if (st) return st;
        RH_CUDA(cudaMemcpy2DAsync(g->stage_in, S.n_p * sizeof(double), W, ldw * sizeof(double),
                                  S.n_p * sizeof(double), N, cudaMemcpyHostToDevice, s));
        Wd = g->stage_in;
        HWd = g->stage_out;
        lw = lh = S.n_p;
    }
    st = ensure_ws(g, (size_t)N);
    if (st) return st;
    st = dirs(g, N, N, g->V, g->T, Wd, lw, 0, HWd, lh,
              rh::PH_WLOAD | rh::PH_SPMUL | rh::PH_L | rh::PH_U | rh::PH_TPROJ | rh::PH_UT | rh::PH_LT |
                  rh::PH_MULADD,
              s);
    if (st) return st;
    if (host) {
        RH_CUDA(cudaMemcpy2DAsync(HW, ldhw * sizeof(double), g->stage_out, S.n_p * sizeof(double),
                                  S.n_p * sizeof(double), N, cudaMemcpyDeviceToHost, s));
        RH_CUDA(cudaStreamSynchronize(s));
    }
    return RH_OK;
}

int64_t rh_hv_work_doubles(const rh_grid* g, int32_t N) {
    if (!g || N < 0) return -1;
    return 2 * (int64_t)g->rows() * (int64_t)N;
}

rh_status rh_batch_hessvec(int32_t n_items, const rh_hv_item* items, int32_t width, void* stream) {
    const rh_hv_config cfg = {width, 0, 0};
    return rh_batch_hessvec_cfg(n_items, items, &cfg, stream);
}

rh_status rh_batch_hessvec_cfg(int32_t n_items, const rh_hv_item* items, const rh_hv_config* cfg, void* stream) {
    if (!cfg) return fail(RH_EINVAL, "config is NULL");
    const int width = cfg->width;
    const int threads = cfg->threads ? cfg->threads : 384;
    const int ks_cap = cfg->split_lanes ? cfg->split_lanes : 32;
    if (width < 0) return fail(RH_EINVAL, "width must be >= 0");
    if (!rh::dirs_batch_shape_ok(threads)) return fail(RH_EINVAL, "threads must be 0, 128, 192, 256 or 384");
    if (ks_cap < 1 || ks_cap > 32 || (ks_cap & (ks_cap - 1))) return fail(RH_EINVAL, "split_lanes must be 0 or a power of two <= 32");
    if (n_items < 0 || (n_items > 0 && !items)) return fail(RH_EINVAL, "bad item list");
    if (n_items == 0) return RH_OK;
    int device = -1;
    for (int i = 0; i < n_items; i++) {
        const rh_hv_item& it = items[i];
        if (!it.grid) return fail(RH_EINVAL, "item " + std::to_string(i) + ": NULL grid");
        const auto& S = it.grid->S;
        if (it.N < 0 || (it.N > 0 && (!it.W || !it.HW)) || it.ldw < S.n_p || it.ldhw < S.n_p)
            return fail(RH_EINVAL, "item " + std::to_string(i) + ": bad W / HW, leading dimension or N");
        if (!it.grid->adjoint_ready)
            return fail(RH_ESTATE, "item " + std::to_string(i) + ": rh_batch_hessvec needs rh_adjoint for the grid's state");
        if (device < 0) device = it.grid->device;
        if (it.grid->device != device) return fail(RH_EINVAL, "all items must be on the same device");
        if (!it.work)
            for (int j = 0; j < i; j++)
                if (!items[j].work && items[j].grid == it.grid)
                    return fail(RH_EINVAL, "a grid appears twice with work = NULL");
    }
    rh_status st = set_device(items[0].grid);
    if (st) return st;
    for (int i = 0; i < n_items; i++)
        if (!items[i].work && items[i].N > 0) {
            st = ensure_ws(items[i].grid, (size_t)items[i].N);
            if (st) return st;
        }
    const unsigned all = rh::PH_WLOAD | rh::PH_SPMUL | rh::PH_L | rh::PH_U | rh::PH_TPROJ | rh::PH_UT | rh::PH_LT |
                         rh::PH_MULADD;
    std::unique_ptr<rh::DirBatch> B(new rh::DirBatch());
    for (int first = 0; first < n_items; first += rh::kMaxBatch) {
        int n = std::min(rh::kMaxBatch, n_items - first);
        B->n_items = 0;
        B->cta_ptr[0] = 0;
        for (int k = 0; k < n; k++) {
            const rh_hv_item& it = items[first + k];
            if (it.N == 0) continue;
            rh_grid* g = it.grid;
            int G = width > 0 ? (it.N + width - 1) / width : rh::dirs_ctas_for(it.N, rh::dirs_batch_slots(threads));
            G = std::max(G, (it.N + 255) / 256);
            rh::DirLaunch& L = B->l[B->n_items];
            L.N = it.N;
            L.n_cta = G;
            L.ld = it.N;
            L.cta_stride = 0;
            L.V = it.work ? it.work : g->V;
            L.T = it.work ? it.work + (size_t)g->rows() * it.N : g->T;
            L.W = it.W;
            L.ldw = it.ldw;
            L.col0 = 0;
            L.HW = it.HW;
            L.ldhw = it.ldhw;
            L.phases = all;
            L.ws_elems = it.work ? (int64_t)g->rows() * it.N : (int64_t)g->ws_elems;
            L.colmap = nullptr;
            L.reach = nullptr;
            int Tt = g->S.n_x - g->S.t0;
            L.use_tail = rh::dirs_tail_fits(Tt, it.N, G) ? 1 : 0;
            L.use_reach = 0;
            B->g[B->n_items] = g->dir();
            B->g[B->n_items].ks_cap = ks_cap;
            B->cta_ptr[B->n_items + 1] = B->cta_ptr[B->n_items] + G;
            B->n_items++;
        }
        rh::launch_dirs_batch(*B, threads, (cudaStream_t)stream);
        RH_CUDA(cudaGetLastError());
    }
    return RH_OK;
}

rh_status rh_hessian(rh_grid* g, int32_t block_n, double* H, int64_t ldh, void* stream, uint32_t flags) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    const auto& S = g->S;
    if (!H || ldh < S.n_p) return fail(RH_EINVAL, "bad H or leading dimension");
    if (block_n <= 0) return fail(RH_EINVAL, "block_n must be positive");
    if (!g->adjoint_ready) return fail(RH_ESTATE, "rh_hessian needs rh_adjoint for the current state");
    rh_status st = set_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    int np = S.n_p;
    bool concurrent = (flags & RH_HESSIAN_CONCURRENT) != 0;
    bool host = !(flags & RH_DEVICE_PTRS);
    double* Hd = H;
    int64_t lh = ldh;
    if (host) {
        st = ensure_stage(g, (size_t)np * np);
        if (st) return st;
        Hd = g->stage_out;
        lh = np;
    }
    const unsigned all = rh::PH_WLOAD | rh::PH_SPMUL | rh::PH_L | rh::PH_U | rh::PH_TPROJ | rh::PH_UT | rh::PH_LT |
                         rh::PH_MULADD;
    int width = concurrent ? np : (block_n < np ? block_n : np);
    st = ensure_ws(g, (size_t)width);
    if (st) return st;
    if (concurrent) {
        st = dirs(g, np, np, g->V, g->T, nullptr, 0, 0, Hd, lh, all, s);
        if (st) return st;
    } else {
        for (int c0 = 0; c0 < np; c0 += block_n) {
            int n = np - c0 < block_n ? np - c0 : block_n;
            st = dirs(g, n, width, g->V, g->T, nullptr, 0, c0, Hd + (int64_t)c0 * lh, lh, all, s);
            if (st) return st;
        }
    }
    if (host) {
        RH_CUDA(cudaMemcpy2DAsync(H, ldh * sizeof(double), Hd, lh * sizeof(double), np * sizeof(double), np,
                                  cudaMemcpyDeviceToHost, s));
        RH_CUDA(cudaStreamSynchronize(s));
    }
    return RH_OK;
}

rh_status rh_hessian_columns(rh_grid* g, int32_t col0, int32_t ncols, double* H, int64_t ldh, void* stream,
                             uint32_t flags) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    const auto& S = g->S;
    if (col0 < 0 || ncols < 0 || (int64_t)col0 + ncols > S.n_p) return fail(RH_EINVAL, "column range outside [0, n_p)");
    if (ncols == 0) return RH_OK;
    if (!H || ldh < S.n_p) return fail(RH_EINVAL, "bad H or leading dimension");
    if (!g->adjoint_ready) return fail(RH_ESTATE, "rh_hessian_columns needs rh_adjoint for the current state");
    rh_status st = set_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int np = S.n_p;
    const bool host = !(flags & RH_DEVICE_PTRS);
    double* Hd = H;
    int64_t lh = ldh;
    if (host) {
        st = ensure_stage(g, (size_t)np * ncols);
        if (st) return st;
        Hd = g->stage_out;
        lh = np;
    }
    st = ensure_ws(g, (size_t)ncols);
    if (st) return st;
    st = dirs(g, ncols, ncols, g->V, g->T, nullptr, 0, col0, Hd, lh,
              rh::PH_WLOAD | rh::PH_SPMUL | rh::PH_L | rh::PH_U | rh::PH_TPROJ | rh::PH_UT | rh::PH_LT | rh::PH_MULADD,
              s);
    if (st) return st;
    if (host) {
        RH_CUDA(cudaMemcpy2DAsync(H, ldh * sizeof(double), Hd, lh * sizeof(double), np * sizeof(double), ncols,
                                  cudaMemcpyDeviceToHost, s));
        RH_CUDA(cudaStreamSynchronize(s));
    }
    return RH_OK;
}

rh_status rh_solve(rh_grid* g, double* R, int64_t ldr, int32_t nrhs, int32_t trans, void* stream, uint32_t flags) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    const auto& S = g->S;
    if (nrhs < 0 || !R || ldr < S.n_x) return fail(RH_EINVAL, "bad R, leading dimension or nrhs");
    if (nrhs == 0) return RH_OK;
    rh_status st = set_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure_ws(g, (size_t)nrhs);
    if (st) return st;
    double* Rd = R;
    int64_t lr = ldr;
    bool host = !(flags & RH_DEVICE_PTRS);
    if (host) {
        st = ensure_stage(g, (size_t)S.n_x * nrhs);
        if (st) return st;
        RH_CUDA(cudaMemcpy2DAsync(g->stage_in, S.n_x * sizeof(double), R, ldr * sizeof(double),
                                  S.n_x * sizeof(double), nrhs, cudaMemcpyHostToDevice, s));
        Rd = g->stage_in;
        lr = S.n_x;
    }
    rh::launch_scatter_rows(S.n_x, nrhs, g->xmap, Rd, lr, g->V, nrhs, 1.0, S.n_x, s);
    // unit-diagonal factors (J_x = D L'' U'): D^-1 R in, or D^-1 out for the transpose
    if (!trans) rh::launch_scale_rows(S.n_x, nrhs, g->invdiag, g->V, nrhs, s);
    st = dirs(g, nrhs, nrhs, g->V, g->V, nullptr, 0, 0, nullptr, 0,
              trans ? (rh::PH_UT | rh::PH_LT) : (rh::PH_L | rh::PH_U), s);
    if (st) return st;
    if (trans) rh::launch_scale_rows(S.n_x, nrhs, g->invdiag, g->V, nrhs, s);
    rh::launch_gather_rows(S.n_x, nrhs, g->xmap, g->V, nrhs, Rd, lr, 1.0, S.n_x, s);
    RH_CUDA(cudaGetLastError());
    if (host) {
        RH_CUDA(cudaMemcpy2DAsync(R, ldr * sizeof(double), g->stage_in, S.n_x * sizeof(double),
                                  S.n_x * sizeof(double), nrhs, cudaMemcpyDeviceToHost, s));
        RH_CUDA(cudaStreamSynchronize(s));
    }
    return RH_OK;
}

rh_status rh_lagrangian_hessvec(rh_grid* g, const double* V, int64_t ldv, int32_t N, double* Y, int64_t ldy,
                                void* stream, uint32_t flags) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    const auto& S = g->S;
    int nu = S.n_x + S.n_p;
    if (N < 0 || !V || !Y || ldv < nu || ldy < nu) return fail(RH_EINVAL, "bad V / Y, leading dimension or N");
    if (N == 0) return RH_OK;
    if (!g->adjoint_ready) return fail(RH_ESTATE, "needs rh_adjoint for the current state");
    rh_status st = set_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = ensure_ws(g, (size_t)N);
    if (st) return st;
    const double* Vd = V;
    double* Yd = Y;
    int64_t lv = ldv, ly = ldy;
    bool host = !(flags & RH_DEVICE_PTRS);
    if (host) {
        st = ensure_stage(g, (size_t)nu * N);
        if (st) return st;
        RH_CUDA(cudaMemcpy2DAsync(g->stage_in, nu * sizeof(double), V, ldv * sizeof(double), nu * sizeof(double), N,
                                  cudaMemcpyHostToDevice, s));
        Vd = g->stage_in;
        Yd = g->stage_out;
        lv = ly = nu;
    }
    rh::launch_scatter_rows(nu, N, g->xmap, Vd, lv, g->V, N, 1.0, S.n_x, s);
    RH_CUDA(cudaMemsetAsync(g->V + (size_t)(S.n_x + S.n_p) * N, 0, N * sizeof(double), s));
    st = dirs(g, N, N, g->V, g->T, nullptr, 0, 0, nullptr, 0, rh::PH_TPROJ, s);
    if (st) return st;
    rh::launch_gather_rows(nu, N, g->xmap, g->T, N, Yd, ly, -1.0, S.n_x, s);
    RH_CUDA(cudaGetLastError());
    if (host) {
        RH_CUDA(cudaMemcpy2DAsync(Y, ldy * sizeof(double), g->stage_out, nu * sizeof(double), nu * sizeof(double), N,
                                  cudaMemcpyDeviceToHost, s));
        RH_CUDA(cudaStreamSynchronize(s));
    }
    return RH_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free reduced-Hessian-vector products.
//
// Some callers cannot let the library call cudaMalloc: a host application that
// owns all device memory through its own pool, a real-time loop that forbids
// allocation after start-up, or code whose device memory is budgeted in
// advance.  rh_hessvec_noalloc serves them: it runs the same direction kernel
// as rh_hessvec, but its two direction buffers live in the fixed array below,
// which every GPU that loads librh holds (2 x 8 MiB) until the process exits.
// ---------------------------------------------------------------------------
#define RH_NOALLOC_DOUBLES (1u << 20)   // doubles per buffer: 8 MiB

static __device__ __align__(256) double rh_noalloc_scratch[2 * RH_NOALLOC_DOUBLES];

namespace {
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[64] = {nullptr};   // per device: device address of rh_noalloc_scratch

// The array's name in host code is only a host-side stand-in; the device
// address is looked up once per device, with that device current.
rh_status noalloc_scratch(int device, double** out) {
    if (device < 0 || device >= 64) return fail(RH_EINVAL, "device id out of range for the fixed scratch table");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, rh_noalloc_scratch);
        if (e != cudaSuccess) return fail(RH_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_ptr[device] = (double*)p;
    }
    *out = g_noalloc_ptr[device];
    return RH_OK;
}
}  // namespace

rh_status rh_hessvec_noalloc(rh_grid* g, const double* W, int64_t ldw, int32_t N, double* HW, int64_t ldhw,
                             void* stream) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    if (N < 0) return fail(RH_EINVAL, "N must be >= 0");
    if (N == 0) return RH_OK;
    const auto& S = g->S;
    if (!W || !HW || ldw < S.n_p || ldhw < S.n_p) return fail(RH_EINVAL, "bad W / HW or leading dimension");
    if ((uint64_t)g->rows() * (uint64_t)N > RH_NOALLOC_DOUBLES)
        return fail(RH_EINVAL, "rh_hessvec_noalloc: N * (n_x + n_p + 1) = " +
                                   std::to_string((uint64_t)g->rows() * (uint64_t)N) + " exceeds the fixed scratch of " +
                                   std::to_string(RH_NOALLOC_DOUBLES) + " doubles per buffer; use rh_hessvec or a smaller N");
    if (!g->adjoint_ready) return fail(RH_ESTATE, "rh_hessvec_noalloc needs rh_adjoint for the current state");
    rh_status st = set_device(g);
    if (st) return st;
    double* scratch = nullptr;
    st = noalloc_scratch(g->device, &scratch);
    if (st) return st;
    // Every row the kernel reads is written by an earlier phase of the same
    // call (W rows, the zero row, -B, the projection), so nothing is cleared.
    rh::DirLaunch L;
    L.N = N;
    L.n_cta = balanced_ctas(N);
    L.ld = N;
    L.cta_stride = 0;
    L.V = scratch;
    L.T = scratch + RH_NOALLOC_DOUBLES;
    L.W = W;
    L.ldw = ldw;
    L.col0 = 0;
    L.HW = HW;
    L.ldhw = ldhw;
    L.phases = rh::PH_WLOAD | rh::PH_SPMUL | rh::PH_L | rh::PH_U | rh::PH_TPROJ | rh::PH_UT | rh::PH_LT | rh::PH_MULADD;
    L.ws_elems = RH_NOALLOC_DOUBLES;
    L.colmap = nullptr;
    L.reach = nullptr;
    L.use_tail = rh::dirs_tail_fits(S.n_x - S.t0, N, L.n_cta) ? 1 : 0;
    L.use_reach = 0;
    rh::launch_dirs(g->dir(), L, (cudaStream_t)stream);
    RH_CUDA(cudaGetLastError());
    return RH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Real-time tracking step (section 6.3, eq. 18-19)
// ---------------------------------------------------------------------------
extern "C" {

rh_status rh_potrf(int32_t n, double* A, int64_t lda, int32_t* info, void* stream) {
    if (n < 0 || !info) return fail(RH_EINVAL, "n must be >= 0 and info non-NULL");
    if (n > 0 && (!A || lda < n)) return fail(RH_EINVAL, "bad A or leading dimension");
    RH_CUDA(rh::launch_potrf(n, A, lda, info, nullptr, (cudaStream_t)stream));
    return RH_OK;
}

rh_status rh_potrs(int32_t n, const double* L, int64_t ldl, double* B, int64_t ldb, int32_t nrhs, double* work,
                   void* stream) {
    if (n < 0 || nrhs < 0) return fail(RH_EINVAL, "n and nrhs must be >= 0");
    if (n == 0 || nrhs == 0) return RH_OK;
    if (!L || !B || !work || ldl < n || ldb < n) return fail(RH_EINVAL, "bad L, B, work or leading dimension");
    RH_CUDA(rh::launch_potrs(n, L, ldl, B, ldb, nrhs, work, true, (cudaStream_t)stream));
    return RH_OK;
}

rh_status rh_rto_step(rh_grid* g, double* H, int64_t ldh, double* d, double* p_next, int32_t* info, void* stream,
                      uint32_t flags) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    const auto& S = g->S;
    if (!H || ldh < S.n_p || !d || !info) return fail(RH_EINVAL, "bad H, leading dimension, d or info");
    if (!g->adjoint_ready) return fail(RH_ESTATE, "rh_rto_step needs rh_adjoint for the current state");
    rh_status st = set_device(g);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int np = S.n_p;
    // Step 1 (second half): the reduced Hessian, all n_p columns in one launch
    st = rh_hessian(g, np, H, ldh, stream, RH_HESSIAN_CONCURRENT | RH_DEVICE_PTRS);
    if (st) return st;
    // Step 2: H = L L^T with the forward solve L y = -g fused into the
    // factorisation (y in rto_y), then L^T d = y; p_next = p + d
    k_rto_rhs<<<nblk(np, 128), 128, 0, s>>>(np, g->grad, g->rto_y);
    RH_CUDA(cudaGetLastError());
    RH_CUDA(rh::launch_potrf(np, H, ldh, info, g->rto_y, s));
    RH_CUDA(rh::launch_potrs(np, H, ldh, d, np, 1, g->rto_y, false, s));
    double* pn = p_next ? p_next : g->rto_y;
    if (p_next || (flags & RH_RTO_APPLY)) {
        k_rto_next<<<nblk(np, 128), 128, 0, s>>>(np, g->pbuf, d, pn);
        RH_CUDA(cudaGetLastError());
    }
    if (flags & RH_RTO_APPLY) {
        int nt = std::max(np, S.n_bus);
        k_rto_apply<<<nblk(nt, 128), 128, 0, s>>>(np, S.n_bus, info, pn, g->pbuf, g->ip_v, g->ip_pg, g->vm, g->pg);
        RH_CUDA(cudaGetLastError());
        g->adjoint_ready = false;
        // the grid's own stream (power flow, adjoint) must see the new parameters
        if (!g->apply_done) RH_CUDA(cudaEventCreateWithFlags(&g->apply_done, cudaEventDisableTiming));
        RH_CUDA(cudaEventRecord(g->apply_done, s));
        RH_CUDA(cudaStreamWaitEvent(g->stream, g->apply_done, 0));
    }
    return RH_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Coloured forward-mode Jacobian (section 4.2.2, Fig. 2)
// ---------------------------------------------------------------------------
extern "C" {

rh_status rh_set_jacobian_method(rh_grid* g, int32_t method) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    if (method != RH_JAC_ANALYTIC && method != RH_JAC_COLORED_AD) return fail(RH_EINVAL, "unknown Jacobian method");
    if (method == g->jac_method) return RH_OK;
    g->jac_method = method;
    g->adjoint_ready = false;
    g->drop_graphs();   // the captured setups hold the previous assembly kernel
    return RH_OK;
}

rh_status rh_grid_coloring(const rh_grid* g, int32_t* colors_x, int32_t* colors_p, int32_t* n_colors_x,
                           int32_t* n_colors_p) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    const auto& S = g->S;
    if (colors_x) std::copy(S.colors_x.begin(), S.colors_x.end(), colors_x);
    if (colors_p) std::copy(S.colors_p.begin(), S.colors_p.end(), colors_p);
    if (n_colors_x) *n_colors_x = S.n_colors_x;
    if (n_colors_p) *n_colors_p = S.n_colors_p;
    return RH_OK;
}

rh_status rh_jacobian(rh_grid* g, int32_t method, int32_t* jx_row, int32_t* jx_col, double* jx_val, int32_t* jp_row,
                      int32_t* jp_col, double* jp_val) {
    if (!g) return fail(RH_EINVAL, "NULL grid");
    if (method != RH_JAC_ANALYTIC && method != RH_JAC_COLORED_AD) return fail(RH_EINVAL, "unknown Jacobian method");
    rh_status st = set_device(g);
    if (st) return st;
    const auto& S = g->S;
    cudaStream_t s = g->stream;
    g->adjoint_ready = false;          // the factors in A are overwritten
    st = assemble(g, method, nullptr, s);
    if (st) return st;
    std::vector<double> A(S.col.size()), jp(S.jp_col.size());
    if (!A.empty()) RH_CUDA(cudaMemcpyAsync(A.data(), g->A, A.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (!jp.empty()) RH_CUDA(cudaMemcpyAsync(jp.data(), g->jpv, jp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    RH_CUDA(cudaStreamSynchronize(s));
    for (size_t k = 0; k < S.jx_slot.size(); k++) {
        if (jx_row) jx_row[k] = S.jx_row[k];
        if (jx_col) jx_col[k] = S.jx_col[k];
        if (jx_val) jx_val[k] = A[S.jx_slot[k]];
    }
    for (int q = 0; q < S.n_x; q++)
        for (int t = S.jp_ptr[q]; t < S.jp_ptr[q + 1]; t++) {
            if (jp_row) jp_row[t] = S.jp_xrow[q];
            if (jp_col) jp_col[t] = S.jp_col[t];
            if (jp_val) jp_val[t] = jp[t];
        }
    return RH_OK;
}

}  // extern "C"
