/*
 * rh.h -- C ABI of librh: batched reduced-Hessian-vector products of the polar
 * power-flow equations on one GB300 GPU (FP64 throughout).
 *
 * Method: "Batched Second-Order Adjoint Sensitivity for Reduced Space
 * Methods" (arXiv 2201.00241).  Notation follows the paper:
 *   g(x, p) = 0        balance equations, eq. (3), x = (theta_pv, theta_pq, v_pq)
 *   p                  parameters (v at every generator bus, Pg at PV buses)
 *   f(x, p)            generation cost; F(p) = f(x(p), p), eq. (5)
 *   lambda             first-order adjoint, eq. (7)
 *   HW                 reduced Hessian applied to W = (w_1..w_N), eq. (9)-(10),
 *                      computed by the parallel reduction of Algorithm 2.
 *
 * Index conventions (all arrays are 0-based):
 *   x  = [theta at PV buses (ascending bus id), theta at PQ buses, v at PQ buses]
 *   p  = [v at generator buses incl. the slack (ascending id), Pg at PV buses]
 *   rows of g and of lambda are ordered like x (P_i <-> theta_i, Q_i <-> v_i).
 *   Bus types: 0 slack (exactly one), 1 PV, 2 PQ.  Powers are per unit on
 *   base_mva; the cost is sum_k c2_k (S Pg_k)^2 + c1_k S Pg_k with S = base_mva,
 *   the slack generation being P_inj + Pd at the slack.
 *
 * Errors: every call returns an rh_status and never aborts; on error the
 * outputs are unspecified and rh_last_error() (thread-local) says why.
 *
 * Ownership: rh_grid_create copies every descriptor array; W, HW, H and all
 * other caller buffers stay owned by the caller and are only used during the
 * call (stream-ordered for device pointers, see RH_DEVICE_PTRS).
 *
 * Streams: entry points taking a `stream` (a cudaStream_t, NULL = legacy
 * default) enqueue their GPU work on it.  One grid must not be used from two
 * host threads at once.
 */
#ifndef RH_H
#define RH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rh_grid rh_grid;

typedef enum {
    RH_OK = 0,
    RH_EINVAL = 1,      /* bad argument or inconsistent grid                      */
    RH_ENOMEM = 2,      /* device or host allocation failed                       */
    RH_ESINGULAR = 3,   /* a static pivot |u_kk| <= 1e-14 max|J_x|                */
    RH_ENOCONV = 4,     /* Newton did not reach the tolerance                     */
    RH_ETIMEOUT = 5,    /* a bounded device wait gave up                          */
    RH_ECUDA = 6,       /* a CUDA runtime call failed                             */
    RH_ESTATE = 7       /* call order: e.g. rh_hessvec before rh_adjoint          */
} rh_status;

/* Pointer-kind flag for W / HW / H / R arguments. */
#define RH_HOST_PTRS 0u     /* caller buffers are in host memory (copied by the call; the call synchronises) */
#define RH_DEVICE_PTRS 1u   /* caller buffers are device pointers on the grid's device (stream-ordered)      */

typedef struct {
    int32_t n_bus, n_branch;
    const int32_t *from, *to;       /* branch end buses, 0 <= from, to < n_bus, from != to   */
    const double *r, *x, *b;        /* series resistance, reactance, total line charging (p.u.) */
    const int8_t *bus_type;         /* 0 slack, 1 PV, 2 PQ                                   */
    const double *c2, *c1;          /* cost coefficients per bus (used at generator buses)    */
    double base_mva;                /* S                                                     */
    /* Weight of one forward level in the choice between the two fill-reducing
     * orders (rh_grid_create), in factor-entry x direction units: an order costs
     * (entries off the bus blocks) x n_p + order_level_cost x (forward levels).
     * 0 picks the order with fewer entries; must be >= 0.  Python callers take
     * the value from the grid record (1.7e6 measured for GB300's direction
     * sweeps: one level of the four sweeps costs about as much as 1.7 M
     * entry-direction FMAs). */
    int64_t order_level_cost;
    /* Dense-tail bound of the sparse LU of J_x (section 5.2 factors J_x once
     * and refactors it with a fixed pattern; here the longest suffix of the
     * elimination order with at most max_tail variables, where fill has made
     * the factors nearly dense, is stored and swept as dense triangles).
     * 0 takes 16 * max(1, round(sqrt(n_x) / 16)) (the top separator of a
     * near-planar grid has about sqrt(n_x) variables; 16, 48, 80 and 128 for
     * the 118-, 1354-, 2869- and 9241-bus grids of the tests); otherwise
     * 2 <= max_tail <= 512.  Results do not depend on
     * it beyond rounding; it trades sparse levels at the top of the
     * elimination tree for dense work (the Python autotuner picks it per grid
     * and batch). */
    int32_t max_tail;
} rh_grid_desc;

typedef struct {
    int32_t n_bus, n_branch, n_gen, n_pv, n_pq;
    int32_t n_x, n_p;
    int32_t n_levels_fwd, n_levels_bwd;   /* bus-level schedule depths               */
    int64_t nnz_jx, nnz_jp;               /* structural nonzeros of J_x and J_p      */
    int64_t nnz_l, nnz_u;                 /* strictly-lower L, upper U incl. diagonal */
    int64_t refactor_updates;             /* multiply-subtract count of a refactor   */
    int32_t setup_kernels;                /* kernels one rh_adjoint launches (counted in its
                                             captured graph; 0 before the first call)    */
    int32_t hessian_kernels;              /* kernels one rh_reduced_hessian launches (its
                                             captured graph; 0 before the first call)    */
    int32_t max_tail;                     /* dense-tail bound in use (rh_grid_desc.max_tail,
                                             or its default)                             */
    int32_t tail_vars;                    /* variables of the dense tail (<= max_tail)     */
} rh_dims;

/*
 * Load a grid (paper section 3.1).  Builds the pi-model admittance matrix
 * (series y = 1/(r + jx), b/2 at each end), and runs the host symbolic phase:
 * fill-reducing ordering of the bus graph (exact minimum degree or minimum
 * weighted fill, whichever costs less for a full reduced Hessian by the
 * cost of desc->order_level_cost; each bus contributes theta then v),
 * symbolic LU of J_x, bus-level schedules, and
 * uploads the fixed patterns to `device`.  The paper factors J_x on the host
 * once and refactors on the device with the same pattern (section 5.2); here
 * only the symbolic part runs on the host.
 * device < 0 runs the symbolic phase only (no CUDA call at all): such a grid
 * answers rh_grid_dims and rh_grid_symbolic, every other call returns
 * RH_ESTATE.
 * Returns RH_EINVAL for a grid without exactly one slack bus, an out-of-range
 * or self-loop branch, a non-positive |r + jx|, a negative order_level_cost or a
 * max_tail outside {0} and [2, 512].
 */
rh_status rh_grid_create(const rh_grid_desc *desc, int32_t device, rh_grid **out);
void rh_grid_destroy(rh_grid *grid);
rh_status rh_grid_dims(const rh_grid *grid, rh_dims *out);

/*
 * Symbolic data for bit-exact comparison (host buffers sized from rh_dims):
 *   perm[n_x]        internal variable q -> x index
 *   bus_order[n_bus-1], level[n_bus-1]   elimination order (bus ids) and the
 *                    forward level of each eliminated bus (longest chain of
 *                    bus-level dependencies through the rows of L)
 *   Lp[n_x+1], Lj[nnz_l]   CSR of the strictly lower part of L (internal indices)
 *   Up[n_x+1], Uj[nnz_u]   CSR of U including the diagonal
 * Any pointer may be NULL to skip that array.
 */
rh_status rh_grid_symbolic(const rh_grid *grid, int32_t *perm, int32_t *bus_order, int32_t *level,
                           int32_t *Lp, int32_t *Lj, int32_t *Up, int32_t *Uj);

/*
 * Power injections of eq. (2) (diagonal admittance term included) at bus
 * voltages vm, va (host arrays of n_bus); P, Q host outputs of n_bus.
 * Evaluated on the device.
 */
rh_status rh_injections(rh_grid *grid, const double *vm, const double *va, double *P, double *Q);

/*
 * Set the parameters p (host, n_p; NULL keeps the current parameters, e.g.
 * those a tracking step applied on the device) and, optionally, the loads
 * pd, qd (host, n_bus each; NULL keeps the previous loads, initially zero).
 * Invalidates the factors, lambda and the projection coefficients.
 */
rh_status rh_set_state(rh_grid *grid, const double *p, const double *pd, const double *qd);

/*
 * Newton-Raphson power flow (section 3.2): x_{k+1} = x_k - J_x^{-1} g(x_k, p),
 * entirely on the device (residual and Jacobian kernel, fixed-pattern LU
 * refactorisation, triangular solves).  x0 (host, n_x) is the initial guess,
 * or NULL to continue from the current state (initially flat: theta = 0,
 * v = 1).  Stops when ||g||_inf <= tol or after max_iter steps.  x_out (host,
 * n_x), iters and resid (final ||g||_inf) may be NULL.
 * Returns RH_ENOCONV if the tolerance is not met, RH_ESINGULAR on a zero pivot.
 */
rh_status rh_powerflow(rh_grid *grid, const double *x0, double tol, int32_t max_iter,
                       double *x_out, int32_t *iters, double *resid);

/*
 * Newton power flow (section 3.2) for up to 32 grids of one topology at once,
 * for instance the load scenarios of one network (each its own rh_grid, with its
 * own loads and parameters): every Newton iteration evaluates the residuals and
 * Jacobians of all items in one launch, refactors them together (one launch per
 * level for all items: their patterns and schedules are the same), solves each
 * item's Newton step in its own CTA, and reads all residuals and pivot flags in
 * one copy: one host synchronisation per iteration for the whole batch.  The
 * work of an iteration is replayed from CUDA graphs captured per set of items
 * still iterating.  An item stops when ||g||_inf <= tol (status RH_OK), after
 * max_iter steps or on a non-finite residual (RH_ENOCONV), or when a static pivot
 * is below 1e-14 max|J_x| (RH_ESINGULAR); the others go on.
 *   grids   n_items distinct grids with the same structure (created from the
 *           same branch list and bus types) on one device; RH_EINVAL otherwise
 *   x0      NULL, or n_items host pointers (each n_x, or NULL: continue from the
 *           item's current state)
 *   x_out   NULL, or n_items host pointers (each n_x, or NULL) for the final x
 *   iters, resid, status   NULL or n_items entries each: Newton steps taken, final
 *           ||g||_inf, and the item's status
 * Synchronous.  Returns RH_OK if every item converged, else RH_ESINGULAR if any
 * item met a bad pivot, else RH_ENOCONV.  Invalidates the items' adjoints.
 */
rh_status rh_batch_powerflow(int32_t n_items, rh_grid *const *grids, const double *const *x0, double tol,
                             int32_t max_iter, double *const *x_out, int32_t *iters, double *resid,
                             int32_t *status);

/*
 * Per-state setup of the hot path at the current (x, p): Jacobian assembly
 * into the fixed LU pattern, LU refactorisation, first-order adjoint
 * lambda = -J_x^{-T} grad_x f (eq. 7), reduced gradient
 * grad F = grad_p f + J_p^T lambda, F = f(x, p), and the per-branch second-order
 * coefficients of lambda^T Hess g + Hess f used by every later rh_hessvec.
 * Outputs (host, nullable): F, lambda[n_x], grad[n_p].
 * Returns RH_ESINGULAR when a static pivot is below 1e-14 max|J_x| (for
 * instance a PQ bus without any branch); the grid then stays without an
 * adjoint (rh_hessvec returns RH_ESTATE).
 */
rh_status rh_adjoint(rh_grid *grid, double *F, double *lambda, double *grad);

/*
 * Reduced Hessian-vector products HW = (Hess F) W for N directions
 * (Algorithm 2, eq. 9-10): B = J_p W; Z = -J_x^{-1} B; (Y_x, Y_p) = the
 * projection of lambda^T Hess g + Hess f on (Z, W) (eq. 13); Psi = -J_x^{-T} Y_x;
 * HW = Y_p + J_p^T Psi.  Requires a prior rh_adjoint for the current state
 * (RH_ESTATE otherwise).
 *   W   n_p x N, column-major, leading dimension ldw >= n_p (column j = w_j)
 *   HW  n_p x N, column-major, leading dimension ldhw >= n_p
 * flags: RH_HOST_PTRS or RH_DEVICE_PTRS.  With device pointers the call is
 * asynchronous on `stream`; with host pointers it copies and synchronises.
 * N = 0 is a no-op.  Every direction is computed independently, so column j of
 * HW does not depend on the other columns of W: a NaN or an infinity in column
 * j of W makes column j of HW non-finite and leaves every other column as it
 * would be without it.
 */
rh_status rh_hessvec(rh_grid *grid, const double *W, int64_t ldw, int32_t N,
                     double *HW, int64_t ldhw, void *stream, uint32_t flags);

/*
 * Cross-instance batching: several (grid, W block) items, for instance the load
 * scenarios of one topology (each its own rh_grid with its own state) or
 * requests on grids of different sizes, computed by ONE kernel launch on
 * `stream` (asynchronous).  Items are independent; item i gets
 * ceil(N_i / width) CTAs (width = target directions per CTA, the right-hand-
 * side interleave width; 0 picks the rh_hessvec default per item).  Up to 32
 * items per launch; larger batches take several launches.
 *   grid    adjoint-ready grid (rh_adjoint for its current state); all items
 *           must be on the same device
 *   W, HW   DEVICE pointers, n_p x N column-major (ldw, ldhw >= n_p of the grid)
 *   work    DEVICE workspace of at least rh_hv_work_doubles(grid, N) doubles
 *           owned by the caller, or NULL to use (and grow) the grid's own
 *           workspace; a grid may appear at most once with work = NULL.
 * Items must not share workspaces or outputs.  Each item's result equals
 * rh_hessvec on the same grid and W up to rounding.
 */
typedef struct {
    rh_grid *grid;
    const double *W;
    int64_t ldw;
    int32_t N;
    double *HW;
    int64_t ldhw;
    double *work;
} rh_hv_item;

int64_t rh_hv_work_doubles(const rh_grid *grid, int32_t N);
rh_status rh_batch_hessvec(int32_t n_items, const rh_hv_item *items, int32_t width, void *stream);

/*
 * Launch configuration of a batched launch (Algorithm 2's level tiles):
 *   width        target directions per CTA (the right-hand-side interleave
 *                width); 0 spreads each item over the SMs' CTA slots
 *   threads      CTA size, one of the compiled shapes 128, 192, 256, 384,
 *                resident at 6, 4, 3, 2 CTAs per SM (768 threads an SM each);
 *                0 takes 384.  A CTA's level of a sweep is one barrier: small
 *                CTAs mean more independent level chains per SM, large ones
 *                more (bus, direction) items per barrier.
 *   split_lanes  narrow-level k-split cap: a level with fewer (bus, direction)
 *                items than threads / 2 splits each row's dot product over up
 *                to split_lanes adjacent lanes (a power of two, 1 = no split, at
 *                most 32); 0 takes 32.
 * RH_EINVAL for any other value (checked before anything else, also when
 * n_items is 0).  Every configuration computes each item's HW up to rounding.
 * rh_batch_hessvec(n, items, width, stream) is this call with {width, 0, 0}.
 */
typedef struct {
    int32_t width;
    int32_t threads;
    int32_t split_lanes;
} rh_hv_config;

rh_status rh_batch_hessvec_cfg(int32_t n_items, const rh_hv_item *items, const rh_hv_config *config,
                               void *stream);

/*
 * Full reduced Hessian H = Hess F (n_p x n_p, column-major, leading dimension
 * ldh >= n_p), computed as HW for W = I by blocks of block_n columns
 * (section 5.3; block count ceil(n_p / block_n)).  All blocks are issued in
 * one launch when `flags` has RH_HESSIAN_CONCURRENT, otherwise one launch per
 * block.  Requires rh_adjoint for the current state.
 */
#define RH_HESSIAN_CONCURRENT 2u
rh_status rh_hessian(rh_grid *grid, int32_t block_n, double *H, int64_t ldh, void *stream, uint32_t flags);

/*
 * Columns col0 .. col0 + ncols - 1 of the reduced Hessian: HW for W the columns
 * col0.. of the identity (Algorithm 2; section 5.3 computes H by such column
 * blocks, which are independent), all in one launch.  This is the unit of a
 * column-block partition of H over several GPUs, each computing its own block.
 *   H   n_p x ncols, column-major, ldh >= n_p; column j of H receives H[:, col0 + j]
 * flags: RH_HOST_PTRS or RH_DEVICE_PTRS, as for rh_hessvec.  Requires rh_adjoint
 * for the current state (RH_ESTATE otherwise); RH_EINVAL for a range outside
 * [0, n_p).  ncols = 0 is a no-op.
 */
rh_status rh_hessian_columns(rh_grid *grid, int32_t col0, int32_t ncols, double *H, int64_t ldh, void *stream,
                             uint32_t flags);

/*
 * The reduced Hessian at the current state in one call (sections 4 and 5:
 * Jacobians, refactorisation, the adjoint of eq. 7, then Algorithm 2 with
 * W = I, all n_p directions in flight): J_x and J_p, the LU refactorisation,
 * lambda, grad F and F, and H = Hess F (n_p x n_p, column-major, ldh >= n_p).
 * The adjoint's transposed solve runs on a second stream beside the first half
 * of the direction sweeps (SpMul, L and U), which do not need lambda; the
 * projection and the transposed sweeps follow once both are done.  The device
 * work is one captured CUDA graph, rebuilt when H, ldh or the workspace change.
 *
 * H: host (default) or, with RH_DEVICE_PTRS, device memory; F (1) and grad
 * (n_p) are optional host outputs (NULL skips them).  `stream` (may be NULL):
 * the call first waits for the work already queued there.  Synchronous: on
 * return the results are in place, and the grid is ready for rh_hessvec as after
 * rh_adjoint.  Returns RH_ESINGULAR when a static pivot is below 1e-14 max|J_x|
 * (H is then not meaningful), RH_EINVAL for a NULL H or ldh < n_p.
 */
rh_status rh_reduced_hessian(rh_grid *grid, double *H, int64_t ldh, double *F, double *grad, void *stream,
                             uint32_t flags);

/*
 * Device times in milliseconds of the last completed rh_reduced_hessian call,
 * from CUDA events recorded inside its graph, all measured from the fork that
 * follows the factorisation:
 *   ms[0]  end of the second direction launch (both launches, and any wait for
 *          the adjoint branch between them),
 *   ms[1]  end of the first direction launch (SpMul, L and U sweeps),
 *   ms[2]  end of the adjoint branch (transposed solve, coefficients, grad F).
 * RH_ESTATE before the first completed call.
 */
rh_status rh_reduced_hessian_times(const rh_grid *grid, float *ms);

/*
 * FP64 work of the two direction launches of one rh_reduced_hessian call (all
 * n_p directions of Algorithm 2 with W = I), counted on the host from the
 * symbolic data; flops, an FMA counting 2.
 *   algorithmic  what Algorithm 2 needs for n_p dense directions on the
 *                unit-diagonal factors: SpMul and SpMulAdd (2 nnz(J_p) each),
 *                the four sweeps (2 nnz(L), 2 (nnz(U) - n_x) each) and the
 *                projection (eq. 13: 8 per incidence and per bus, 4 per
 *                slack-gradient entry, 1 per Pg row)
 *   executed     what the kernels issue for those launches: the forward L
 *                sweep over each CTA's reach only (the rows W = I can make
 *                nonzero for that CTA's directions), the last L^T sweep over
 *                the rows SpMulAdd reads, no multiplications in SpMul (it
 *                scatters columns of J_p), the dense tail as a full triangle
 *   n_sm         SMs of the device (it fixes the CTA split); 0 takes the grid's
 *                device, required > 0 on a symbolic-only grid.
 * Host only, no device work.
 */
rh_status rh_reduced_hessian_flops(const rh_grid *grid, int32_t n_sm, double *algorithmic, double *executed);

/*
 * Measurement utility (not part of the paper's method): the FP64 FMA rate of
 * `device`, the roofline the direction kernel is bound by.  Runs
 * ctas_per_sm x (SM count) CTAs of threads_per_cta threads (a multiple of 32,
 * at most 1024), each thread 8 independent FMA chains of `iters` steps, and
 * returns the rate in GFLOP/s (an FMA counting 2) and the time in ms (ms may be
 * NULL).  Synchronous; allocates and frees a small device buffer.  Returns
 * RH_EINVAL for bad arguments (rh_last_error is not set by this call).
 */
rh_status rh_fp64_fma_rate(int32_t device, int32_t ctas_per_sm, int32_t threads_per_cta, int64_t iters,
                           double *gflops, float *ms);

/*
 * Solve J_x X = R (trans = 0) or J_x^T X = R (trans = 1) with the current
 * device factors (after rh_adjoint or rh_refactor), in place.  R is n_x x nrhs,
 * column-major, leading dimension ldr >= n_x, indexed like x.  These are the
 * batched sparse solves of Algorithm 2 on their own.
 */
rh_status rh_solve(rh_grid *grid, double *R, int64_t ldr, int32_t nrhs, int32_t trans,
                   void *stream, uint32_t flags);

/*
 * Assemble J_x, J_p at the current state and refactor (the first two steps of
 * rh_adjoint).  A_out (host, nullable, nnz_l + nnz_u doubles) receives the
 * factors in the CSR pattern of rh_grid_symbolic, row by row: the strictly
 * lower entries of L then the entries of U.
 */
rh_status rh_refactor(rh_grid *grid, double *A_out);

/*
 * The projection step of Algorithm 2 on its own (eq. 11/13): Y = [Hess l] V
 * with l = f + lambda^T g at the current state and lambda of the last
 * rh_adjoint.  V, Y are (n_x + n_p) x N column-major with leading dimensions
 * ldv, ldy; rows 0..n_x-1 are indexed like x, rows n_x.. like p.
 */
rh_status rh_lagrangian_hessvec(rh_grid *grid, const double *V, int64_t ldv, int32_t N,
                                double *Y, int64_t ldy, void *stream, uint32_t flags);

/*
 * Allocation-free form of rh_hessvec (the paper has no counterpart).  For
 * callers that must not have the library allocate device memory after
 * start-up, such as an application that
 * owns all device memory through its own pool, or a real-time control loop
 * that forbids allocation once running.  The two direction buffers of the
 * computation live in a fixed device array of 2 x 8 MiB that every GPU holding
 * librh keeps until the process exits, so this call makes no cudaMalloc,
 * cudaFree or allocating library call.
 *   W, HW   DEVICE pointers, n_p x N column-major (ldw, ldhw >= n_p)
 *   limit   N * (n_x + n_p + 1) <= 1048576 (e.g. N <= 52 on a 9241-bus grid,
 *           N <= 353 on a 1354-bus grid); larger N returns RH_EINVAL.
 * Asynchronous on `stream`.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress, once per device); make that first call
 * before any stream capture.  All calls on a device share the one array, which
 * keeps the previous call's contents (the kernel initialises everything it
 * reads), so calls that overlap on the GPU, for instance on two streams or for
 * two grids at once, race and give wrong results: serialise them.
 * Requires rh_adjoint for the current state (RH_ESTATE otherwise).
 */
rh_status rh_hessvec_noalloc(rh_grid *grid, const double *W, int64_t ldw, int32_t N,
                             double *HW, int64_t ldhw, void *stream);

/*
 * Dense FP64 Cholesky factorisation A = L L^T of a symmetric positive definite
 * n x n matrix: the factorisation of the real-time tracking step (section 6.3,
 * eq. 19), where the paper calls a vendor library.
 *   A     DEVICE pointer, column-major, leading dimension lda >= n.  The lower
 *         triangle is read and overwritten with L; the strictly upper triangle
 *         is neither read nor written.
 *   info  DEVICE pointer to one int32: 0, or j + 1 for the first column j whose
 *         pivot (the diagonal of the Schur complement) is not positive, i.e. A
 *         is not positive definite; L is then unspecified from column j on.
 * Asynchronous on `stream` (the status only reports argument and launch
 * errors; read info after the stream).  n = 0 only sets info to 0.
 */
rh_status rh_potrf(int32_t n, double *A, int64_t lda, int32_t *info, void *stream);

/*
 * Solve L L^T X = B in place with the factor written by rh_potrf (its lower
 * triangle is read).  L, B, work are DEVICE pointers: B is n x nrhs
 * column-major (ldb >= n); work holds n * nrhs doubles owned by the caller
 * (the intermediate L^{-1} B).  Asynchronous on `stream`.
 */
rh_status rh_potrs(int32_t n, const double *L, int64_t ldl, double *B, int64_t ldb, int32_t nrhs, double *work,
                   void *stream);

/*
 * One update of the real-time tracking algorithm (section 6.3, eq. 18-19) at
 * the grid's current loads and state, after rh_adjoint (RH_ESTATE otherwise),
 * which supplies the reduced gradient g:
 *   Step 1, second half: H = Hess F, every column in one launch (rh_hessian
 *           with RH_HESSIAN_CONCURRENT);
 *   Step 2: H = L L^T (rh_potrf), d = -H^{-1} g (rh_potrs), p_next = p + d.
 *   H       DEVICE, n_p x n_p column-major, ldh >= n_p; holds H with its lower
 *           triangle replaced by L on return
 *   d       DEVICE, n_p: the step
 *   p_next  DEVICE, n_p, or NULL
 *   info    DEVICE int32, as for rh_potrf; d and p_next are unspecified when
 *           it is not 0
 * flags: RH_RTO_APPLY also makes p_next the grid's parameters, as rh_set_state
 * with unchanged loads would, but only if info is 0 (decided on the device);
 * it invalidates the adjoint, and later calls on the grid are ordered after it.
 * Asynchronous on `stream`.
 */
#define RH_RTO_APPLY 4u
rh_status rh_rto_step(rh_grid *grid, double *H, int64_t ldh, double *d, double *p_next, int32_t *info,
                      void *stream, uint32_t flags);

/*
 * Coloured forward-mode Jacobian (section 4.2.2, Fig. 2): the paper assembles
 * J_x and J_p by forward-mode AD on dual numbers, with the columns compressed
 * by a colouring.  Here the colouring is greedy: columns in index order (x
 * order for J_x, p order for J_p), each taking the smallest colour that no
 * earlier column sharing a row with it holds.  The injections are evaluated on
 * dual numbers seeded with the unit tangent of each variable's colour, 8
 * colours per pass, and every structural entry is read from the tangent of
 * its column's colour.
 *
 * rh_set_jacobian_method: the assembly used by every later rh_powerflow,
 * rh_adjoint and rh_refactor on the grid (RH_JAC_ANALYTIC, the default, or
 * RH_JAC_COLORED_AD).  Invalidates the adjoint.
 *
 * rh_grid_coloring (host outputs, any pointer may be NULL; works on a
 * symbolic-only grid): colors_x[n_x], colors_p[n_p] and the colour counts.
 *
 * rh_jacobian: J_x and J_p at the current state by `method`, as host triplets
 * in x / p indices: nnz_jx entries of J_x sorted by (row, column) and nnz_jp
 * entries of J_p (rh_dims); any pointer may be NULL.  Overwrites the factors,
 * so rh_adjoint is needed again before rh_hessvec.  Synchronous.
 */
#define RH_JAC_ANALYTIC 0
#define RH_JAC_COLORED_AD 1
rh_status rh_set_jacobian_method(rh_grid *grid, int32_t method);
rh_status rh_grid_coloring(const rh_grid *grid, int32_t *colors_x, int32_t *colors_p, int32_t *n_colors_x,
                           int32_t *n_colors_p);
rh_status rh_jacobian(rh_grid *grid, int32_t method, int32_t *jx_row, int32_t *jx_col, double *jx_val,
                      int32_t *jp_row, int32_t *jp_col, double *jp_val);

/*
 * Index checks (a development aid, no counterpart in the paper).  librh built
 * with -DRH_BOUNDS (librh_bounds.so) checks, in its kernels, every row, slot and
 * position index it reads or writes against the size of its array; a failed
 * check sets a bit of an error word on the device and skips that access (no
 * trap, no early exit that a barrier would wait for).  rh_bounds_check sets
 * *enabled to 1 in that build (0 in the normal one, *errors then 0), and reads
 * and clears the error word of `device` into *errors (0: no index outside its
 * array since the last call).
 */
rh_status rh_bounds_check(int32_t device, int32_t *enabled, uint32_t *errors);

/* Message of the last error on this thread ("" if none). */
const char *rh_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
