// rh_kernels.h -- device data layout and kernel launchers of librh.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace rh {

// Phases of the direction kernel (one bit each, executed in this order).
enum : unsigned {
    PH_WLOAD = 1u << 0,    // W (or identity columns) -> rows n_x.. of V; zero row
    PH_SPMUL = 1u << 1,    // V[x rows] = -J_p W                          (Alg. 2 SpMul)
    PH_L = 1u << 2,        // V <- L^{-1} V                                (BatchSparseSolve 1)
    PH_U = 1u << 3,        // V <- U^{-1} V
    PH_TPROJ = 1u << 4,    // T[x rows] = -y_x, T[p rows] = y_p            (BatchTensorProjection)
    PH_UT = 1u << 5,       // T <- U^{-T} T                                (BatchSparseSolve 2)
    PH_LT = 1u << 6,       // T <- L^{-T} T
    PH_MULADD = 1u << 7,   // HW = y_p + J_p^T psi                         (SpMulAdd)
};

// A bus-level schedule: level l holds the bus blocks slots[ptr[l] .. ptr[l+1]),
// maxext[l] = their longest row part.  Slots are packed descriptors
//   forward  {q, n, rp, rpv}: theta row q, n columns left of the bus (or left of
//            the dense tail for the tail's external phase), row parts at rp / rpv
//            (rpv = -1 for a PV bus);
//   backward {q, n, ue0, ue1}: U parts right of the bus at ue0 / ue1 (-1: PV).
struct LevelSet {
    int n_lev;
    const int *ptr;
    const int4 *slots;
    const int *maxext;
};

// Read-only grid data used by the direction kernel, all device pointers.
struct DirGrid {
    int n_x, n_p;
    int nnz;                                   // positions of the pattern of A (index checks)
    int zero_row;                              // n_x + n_p: a row of zeros in V
    // filled matrix A = L + U (CSR), its transposed values and 1/diagonal
    const int *col;
    const double *A, *At, *invdiag;
    LevelSet lf, lb;                           // full forward / backward schedules
    LevelSet sf, sb, ef;                       // sparse part only, and the tail's external phase
    LevelSet sbr;                              // sb restricted to the rows of J_p and their ancestors
    // dense trailing block [t0, t0 + T): packed strictly-triangular columns
    //   triL  (L,  lower, unit)            triU  (U,  upper, column j scaled by 1/u_jj)
    //   triUt (U^T, lower, column j scaled) triLt (L^T, upper, unit)
    int t0, T;
    const double *triL, *triU, *triUt, *triLt;
    // Unit-diagonal factors used by k_dirs (J_x = D L'' U', D = diag(U)): values of
    // L'' and U' in A's pattern and transposed, the dense tail's triangles of L'',
    // U', U'^T, L''^T, and D^-1 J_p by p index (jptvd)
    const double *Ad, *Atd;
    const double *triLd, *triUd, *triUtd, *triLtd;
    const double *jptvd;
    // bus structure by theta row: theta row of the bus owning row q; the bus's
    // elimination-tree parent as 2 * (its theta row) + (1 if it has a v row), or -1
    // for a root or a parent in the dense tail
    const int *qtheta, *bparent;
    // J_p by internal rows and by p index; rows with and without entries
    const int *jp_ptr, *jp_col;
    const double *jpv;
    int n_jp_rows, n_jp_zero;
    const int *jp_rows, *jp_zero_rows;
    const int *jpt_ptr, *jpt_row;
    const double *jptv;
    // narrow-level k-split cap of the sweeps: lanes per row at most (1, 2, 4, ..., 32)
    int ks_cap;
    // projection data (per bus, original ids); rows are V/Y row indices
    int n_bus;
    const int *tp_bus;                         // bus processing order (internal order, slack last)
    const int *uth, *uv;                       // rows of theta_b (zero row at the slack) and v_b
    const int *tp_l0;                          // position of (v, theta) in At for a PQ bus of forward level 0, else -1
    const int *inc_ptr, *inc_uth, *inc_uv;     // incident branches: rows of the other end
    const double4_32a *inc_coef;               // (K, -a, b, -c) per incidence (state dependent)
    const double *d2, *asum, *csum;            // per-bus coefficients (state dependent)
    const uint8_t *has_gref;
    const double *gref_th, *gref_v;            // grad P_slack at the rows of bus b
    int n_gref;
    const int *gref_row;
    const double *gref_val;
    const double *c2ref;                       // device scalar c''_slack
    const int *pg_row;                         // per bus: row of Pg (or -1)
    const double *pg_curv;                     // per bus: c''_k
};

struct DirLaunch {
    int N;                     // directions in this launch
    int n_cta;                 // CTAs; CTA c owns directions [c*N/n_cta, (c+1)*N/n_cta)
    // Layout of V and T: element (row r, direction c0 + d) of CTA c is at
    //   cta_stride > 0 (panel-major): c * cta_stride + r * ld + d   (each CTA's panel contiguous)
    //   cta_stride = 0 (interleaved):  r * ld + c0 + d              (ld >= N)
    int64_t ld;
    int64_t cta_stride;
    double *V, *T;             // tangent buffer; buffer of the transposed sweeps / projection
    const double *W;           // n_p x N column-major (ldw), or NULL for identity columns
    int64_t ldw;
    int col0;                  // identity columns start at col0
    double *HW;                // n_p x N column-major (ldhw)
    int64_t ldhw;
    unsigned phases;
    int64_t ws_elems;          // doubles of V and of T each (0: not stated; index checks of the bounds build)
    int use_tail;              // dense tail in shared memory (needs T * ceil(N / n_cta) <= 4096)
    int use_reach;             // identity W: forward L sweep only over the reach of B's nonzeros (needs use_tail,
                               // and phases L and U in the same launch)
    // identity W: direction j is column colmap[col0 + j] of the identity and writes that
    // column of HW (relative to HW: colmap[col0 + j] - col0); NULL: column col0 + j
    const int* colmap;
    // identity W with use_reach: each CTA's reach precomputed on the host (NULL: found at
    // run time, a bit mask grown level by level)
    const struct ReachSched* reach;
};

// The reach of every CTA of one identity-W launch (N directions on n_cta CTAs, columns
// through colmap): for CTA c, the sparse buses its J_p columns can make nonzero in the
// forward L sweep (those columns' buses and their ancestors), as forward-sweep slots
// grouped by level (only the CTA's nonempty levels), and the bit mask of their rows.
struct ReachSched {
    int n_cta, words;          // CTAs; 32-bit words of a row mask ((n_x + 31) / 32)
    const int* nlev;           // [n_cta] levels of CTA c
    const int* lev0;           // [n_cta] CTA c's first entry in ptr / maxext
    const int* ptr;            // per CTA nlev + 1 offsets into slots
    const int* maxext;         // per CTA and level: longest row part
    const int4* slots;         // forward slots {q, n, rp, rpv} of the reach buses
    const unsigned* masks;     // [n_cta * words] rows of the reach
};

// Up to kMaxBatch (grid, W block) items of one batched launch, passed by value as
// the kernel parameter (about 16 KB).
constexpr int kMaxBatch = 32;
struct DirBatch {
    int n_items;
    int cta_ptr[kMaxBatch + 1];
    DirGrid g[kMaxBatch];
    DirLaunch l[kMaxBatch];
};
// threads: one of the compiled CTA shapes (dirs_batch_shape_ok)
void launch_dirs_batch(const DirBatch& B, int threads, cudaStream_t st);
bool dirs_batch_shape_ok(int threads);
int dirs_batch_ctas_per_sm(int threads);   // resident CTAs per SM of a shape (0: not compiled)
int dirs_batch_slots(int threads);         // resident CTAs of a shape on the current device

// Grid-wide power-flow evaluation data (per bus, original ids).
struct PfGrid {
    int n_bus, n_x, ref;
    int nnz_a, nnz_jp;                 // slots of A and of J_p (index checks)
    const int *yp, *yj, *ydiag;
    const double *G, *B;
    const int *qth, *qv, *ip_v, *ip_pg;
    const int *jac_dst;
    const int *pg_slot;
    double base_mva;
    const double *c2, *c1;
    // the warp-per-entry evaluation: bus of every admittance entry, and the buses
    // [pf_wb[w], pf_wb[w + 1]) of warp w (n_pfw = 0: one thread per bus instead)
    const int *yrow, *pf_wb;
    int n_pfw;
};

struct PfState {
    double *vm, *va, *pg, *pd, *qd;  // per bus
    double *P, *Q;                   // injections (output)
    double *sc;                      // per bus: sin, cos of the angle (launch_pf_prep; NULL: not kept)
};

// ---- programmatic dependent launch --------------------------------------------
// The long chains of dependent launches (refactorisation levels, dense-tail and
// Cholesky tile columns, the triangular solves) use programmatic stream
// serialisation: the next launch is scheduled as the current one's CTAs exit
// instead of after its completion is signalled, hiding part of the launch
// latency.  Every kernel launched this way calls pdl_wait() before it touches
// memory, which returns once the previous kernel in the stream has completed
// and its writes are visible; without a previous kernel it returns at once.
// The first kernel of a chain is launched without the attribute (pdl = false),
// so it is fully ordered after whatever precedes it (copies, event waits).
#ifdef __CUDACC__
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ---- division-free elimination of dense tiles -----------------------------------
// The diagonal tiles of the dense factorisations (the refactorisation's dense
// tail LU, the tracking step's Cholesky) are eliminated by cross-multiplied steps
// a_rc <- 2^-e (d a_rc - a_rj a_jc), d the current pivot and 2^-e the power of two
// that brings it into [1, 2), instead of a reciprocal of every pivot on the
// critical path.
// e with 2^-e d in [1, 2) for a positive normal pivot d (e <= 1022, so 2^-e is
// normal too); 0 for any other value, where the factorisation has failed.
__device__ __forceinline__ int pivot_shift(double d) {
    const int f = (int)((__double_as_longlong(d) >> 52) & 0x7ff);
    return (d > 0.0 && f != 0 && f != 0x7ff) ? min(f - 1023, 1022) : 0;
}

// v * 2^-sh for |sh| <= 1022 by an integer update of the exponent field, with
// the bits of the IEEE multiplication whenever v and the result are normal
// numbers; zero, subnormal, infinite and NaN v are returned as they are, a
// result below the normal range is flushed to a signed zero and one above it
// becomes a signed infinity.  Selects only, no branch: the update sits on the
// critical path of every elimination step.
__device__ __forceinline__ double scale_pow2(double v, int sh) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned long long sign = b & 0x8000000000000000ull;
    const int f = (int)((b >> 52) & 0x7ffu);
    const int nf = f - sh;
    unsigned long long r = b - ((unsigned long long)(long long)sh << 52);
    r = nf < 1 ? sign : r;
    r = nf > 0x7fe ? (sign | 0x7ff0000000000000ull) : r;
    r = (f == 0 || f == 0x7ff) ? b : r;
    return __longlong_as_double((long long)r);
}
#endif
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, args...);
}

// ---- launchers (all asynchronous on `st`) ----------------------------------
void launch_injections(const PfGrid& g, const PfState& s, cudaStream_t st);
// residual (internal order) and/or Jacobian values; gmax / jmax receive
// max |g| and max |J_x| as ordered bit patterns (zeroed by the caller).
// Before launch_pf_eval: sin and cos of every bus angle into s.sc and, with zero,
// A (nnz_a slots), the two maxima and *err (if given) cleared.
void launch_pf_prep(const PfGrid& g, const PfState& s, double* A, unsigned long long* umax, int* err, bool zero,
                    cudaStream_t st);
void launch_pf_eval(const PfGrid& g, const PfState& s, double* gres, double* A, double* jpv,
                    unsigned long long* gmax, unsigned long long* jmax, bool want_jac, cudaStream_t st);
void launch_newton_update(const PfGrid& g, const PfState& s, const double* dx, cudaStream_t st);
// Coloured forward-mode Jacobian (section 4.2.2): the injections evaluated on
// dual numbers whose tangents are the seed colours (col_th, col_v, col_pg per
// bus), in chunks of tangents; writes the J_x slots of A (and max |J_x| into
// jmax) and the J_p values.  The residual comes from launch_pf_eval.
cudaError_t launch_jac_ad(const PfGrid& g, const PfState& s, const int* col_th, const int* col_v, const int* col_pg,
                          int n_colors, double* A, double* jpv, unsigned long long* jmax, cudaStream_t st);
// Fixed-pattern LU refactorisation data (device pointers).
struct RfGrid {
    int n_x, t0, T;                    // dense trailing block [t0, n_x), T = n_x - t0
    int nnz;                           // positions of A (index checks)
    double* tailD;                     // T x T row-major scratch of the tiled dense LU
    const int* tail_pos;               // (i, j) of the trailing block -> position in A, -1 if structurally zero
    const int *rf_lev_bus, *q0;
    const uint8_t *nv;
    const int *rowptr, *col, *diagpos, *tpos;
    const int *tgt_pos;                // update targets (positions in A; -1: empty lane), grouped by level
    // 3 int2 per group: {dt (first level) or bus k (later levels), dv}, {a_it, a_tj},
    // {a_iv, a_vj} positions; grp: each target's first group (all -1: none), xgrp:
    // its further groups [xptr[t], xptr[t + 1])
    const int2 *grp, *xgrp;
    const int64_t *xptr;
    // pivot quantities per sparse bus (1/u_tt, l_vt, 1/u_vv, u_tv), written by the
    // pivot jobs (bus piv_bus[q], block positions piv_pos[4 q ..]; see launch_refactor)
    double4_32a *piv;
    int n_piv;
    const int *piv_bus, *piv_pos;
    // pivot steps by entry (k_rf_pivot): bus and positions {a_tj, a_vj, a_jt, a_jv}
    int64_t n_pe;
    const int *pe_bus;
    const int4 *pe_pos;
    double *A, *invdiag;
    const unsigned long long *jmax;
    int *err;
};
// L2 prefetch of up to 8 read-only device arrays (16-byte aligned; the bytes of
// each are rounded down to a multiple of 16); `first` is filled by the launcher.
struct PrefetchList {
    int n;
    const char* p[8];
    unsigned long long bytes[8];
    unsigned long long first[9];
};
void launch_prefetch_l2(const PrefetchList& L, cudaStream_t st);
// One update launch per level (its pivot jobs [piv_lev_ptr[l], piv_lev_ptr[l + 1])
// at the front), the pivot steps of every sparse bus, then the dense tail's LU.
cudaError_t launch_refactor(const RfGrid& g, const int* lev_ptr_host, const int64_t* tgt_lev_ptr_host,
                            const int* piv_lev_ptr_host, int n_lev, cudaStream_t st);
// At (transposed values), Ad / Atd (the unit-diagonal factors L'', U' of J_x = D L'' U'
// and their transpose), jptv (J_p by p index) and jptvd (D^-1 J_p by p index)
void launch_transpose_values(int nnz, const int* tpos, const int* arow, const int* col, const int* diagpos,
                             const double* A, const double* invdiag, double* At, double* Ad, double* Atd, int nnz_jp,
                             const int* jpt_src, const int* jpt_row, const double* jpv, double* jptv, double* jptvd,
                             cudaStream_t st);
void launch_dirs(const DirGrid& g, const DirLaunch& L, cudaStream_t st);
// raise the dynamic shared-memory limits of the kernels that need it (once per grid)
cudaError_t prepare_kernels();
bool dirs_tail_fits(int T, int N, int n_cta);
// dense tail triangles of the current factors (pos: T*T map to A, -1 where structurally zero)
// x[r][c] *= s[r] for r < n, c < N
void launch_scale_rows(int n, int N, const double* s, double* x, int64_t ld, cudaStream_t st);
// triangles of the single solves (triL .. triLt) and of the unit-diagonal factors (triLd .. triLtd)
void launch_build_tail(int T, int t0, const int* pos, const double* A, const double* invdiag, double* triL,
                       double* triU, double* triUt, double* triLt, double* triLd, double* triUd, double* triUtd,
                       double* triLtd, cudaStream_t st);
// One right-hand side in one CTA with x in shared memory: mode 2 also keeps the
// dense tail triangle there (needs the tail triangles built), 1 without it,
// 0 when x does not fit (use the direction kernel instead).
int solve1_mode(int n_x, int T);
cudaError_t launch_solve1(const DirGrid& g, double* x, unsigned phases, bool use_tail, cudaStream_t st);

// Dense Cholesky of the tracking step (dense.cu).  A, L, B, work, y and info
// are device pointers; column-major.  info receives 0 or the 1-based column of
// the first pivot that is not positive.  launch_potrf with y != NULL also runs
// the forward solve L y = b in place on the vector y (b on entry).
// launch_potrs: work holds n * nrhs doubles; with forward = false it only runs
// the backward sweep L^T X = work, writing X into B.
// ---- Newton power flow over several grids of one topology (load scenarios) ----
// Every batched launch takes item i from blockIdx.y (blockIdx.x for the solve):
// the grids share their symbolic data, so every level range is the same for all.
constexpr int kMaxPfBatch = 32;
struct PfBatchItem {
    PfGrid g;
    PfState s;
    double *A, *jpv;            // J_x values (in A's slots), J_p values
    double* x;                  // residual in, Newton step out (internal order)
    unsigned long long* umax;   // max |g|, max |J_x| as ordered bits
    int* err;                   // pivot flag of the refactorisation
};
struct PfBatch {
    int n, max_bus;
    PfBatchItem it[kMaxPfBatch];
};
struct RfBatch {
    int n;
    RfGrid g[kMaxPfBatch];
};
struct TriBatch {
    int n, T, t0;
    const int* pos[kMaxPfBatch];
    const double *A[kMaxPfBatch], *invdiag[kMaxPfBatch];
    double *triL[kMaxPfBatch], *triU[kMaxPfBatch];
};
struct Solve1Batch {
    int n;
    DirGrid g[kMaxPfBatch];
    double* x[kMaxPfBatch];
};
// residual and Jacobian of every item (after launch_pf_prep_batch)
void launch_pf_eval_batch(const PfBatch& B, cudaStream_t st);
// every item's sin/cos per bus, A and the maxima cleared (not the pivot flag)
void launch_pf_prep_batch(const PfBatch& B, cudaStream_t st);
// out[2 i] = max |g| of item i, out[2 i + 1] = its pivot flag
void launch_batch_status(const PfBatch& B, double* out, cudaStream_t st);
cudaError_t launch_refactor_batch(const RfBatch& B, const int* lev_ptr_host, const int64_t* tgt_lev_ptr_host,
                                  const int* piv_lev_ptr_host, int n_lev, cudaStream_t st);
// the dense tail's triangles of the single solves (L, and U with columns scaled by 1/u_jj)
void launch_tail_tri_batch(const TriBatch& B, cudaStream_t st);
cudaError_t launch_solve1_batch(const Solve1Batch& B, unsigned phases, bool use_tail, int n_x, int T, cudaStream_t st);
void launch_newton_update_batch(const PfBatch& B, cudaStream_t st);

int dense_tile(int n);
cudaError_t launch_potrf(int n, double* A, int64_t lda, int* info, double* y, cudaStream_t s);
cudaError_t launch_potrs(int n, const double* L, int64_t ldl, double* B, int64_t ldb, int nrhs, double* work,
                         bool forward, cudaStream_t s);
int dirs_default_ctas(int N);
// CTA slots of the direction kernel on a device of n_sm SMs, and the CTAs a launch of
// N directions takes there
int dirs_cta_slots_for(int n_sm);
int dirs_ctas_for(int N, int slots);
// CTAs of k_dirs the device holds at once (CTAs per SM x SMs)
int dirs_cta_slots();

// adjoint helpers
struct AdjData {
    double *rhs;          // n_x, internal order (output: -grad_x f)
    double *cref, *c2ref; // device scalars c'_slack, c''_slack
    double *F;            // device scalar
    double *gref_th, *gref_v;   // per bus
    int *gref_row;        // up to n_gref_max entries
    double *gref_val;
    int n_gref;           // number of entries (static: slack + its neighbours)
    const int *uth, *uv;  // combined rows per bus
};
void launch_adjoint_rhs(const PfGrid& g, const PfState& s, const AdjData& a, cudaStream_t st);
void launch_adjoint_coef(const PfGrid& g, const PfState& s, const double* lambda_int, const double* cref,
                         const int* inc_ptr, const int* inc_nb, double4_32a* inc_coef, double* d2, double* asum,
                         double* csum, double* pg_curv, cudaStream_t st);
void launch_gradient(const PfGrid& g, const PfState& s, int n_p, const int* jpt_ptr, const int* jpt_row,
                     const double* jptv, const double* lambda_int, const double* cref, const double* gref_v,
                     double* grad, cudaStream_t st);

// permutation helpers between external (x, p) order and the internal rows
void launch_gather_rows(int n_rows, int N, const int* map, const double* src, int64_t lds, double* dst,
                        int64_t ldd, double scale_x, int n_x, cudaStream_t st);
void launch_scatter_rows(int n_rows, int N, const int* map, const double* src, int64_t lds, double* dst,
                         int64_t ldd, double scale_x, int n_x, cudaStream_t st);

}  // namespace rh
