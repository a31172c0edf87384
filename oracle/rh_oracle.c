/*
 * rh_oracle.c -- plain, slow, CPU reference for the reduced-Hessian-vector
 * product of the polar power-flow equations (arXiv 2201.00241).
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU
 * baseline leg of the benchmark call it; the CUDA library never does, and the
 * two share no code.  Everything here is IEEE fp64, compiled with
 * -ffp-contract=off, written for readability over speed; single-threaded,
 * except that orc_hessvec_threads may share the independent columns of W out
 * among threads (each column's arithmetic is the same either way).
 *
 * What it computes (paper sections and equations):
 *   - power injections, eq. (2), including the diagonal admittance term;
 *   - the balance equations g(x, p), eq. (3), state x = (theta_pv, theta_pq, v_pq);
 *   - parameters p = (v at every generator bus incl. the slack, Pg at PV buses),
 *     the reading that reproduces the n_x / n_p counts of Table 1;
 *   - cost f = sum over generators of c2 (S Pg)^2 + c1 S Pg, the slack Pg being
 *     P_inj + Pd at the slack (a function of x and p);
 *   - textbook analytic Jacobians J_x = dg/dx and J_p = dg/dp;
 *   - Newton-Raphson power flow (section 3.2) with its own left-looking sparse LU
 *     under a static fill-reducing ordering of the bus graph;
 *   - first-order adjoint lambda and reduced gradient, eq. (6)-(7);
 *   - the explicit Hessian of the Lagrangian l = f + lambda^T g over (x, p),
 *     assembled bus by bus from the second derivatives of every P_i and Q_i
 *     (no automatic differentiation);
 *   - the adjoint-adjoint reduced Hessian-vector product, eq. (9)-(10):
 *       z   = -J_x^{-1} J_p w
 *       y   = [Hess l] (z, w)                     (eq. 11 / 13)
 *       psi = -J_x^{-T} y_x
 *       Hw  = y_p + J_p^T psi
 *     one direction at a time (Algorithm 1), no batching, no fusion.
 *   - the symbolic data of the factorization (ordering, patterns, levels),
 *     derived independently for bit-exact comparison with the library;
 *   - the dense Cholesky factorisation and the two triangular solves of the
 *     real-time tracking step (section 6.3, eq. 18-19).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define REF 0
#define PV 1
#define PQ 2

/* ------------------------------------------------------------------------ */
/* grid                                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n_bus, n_branch, n_x, n_p, n_gen, ref;
    int8_t *type;
    double *c2, *c1;
    double S;                 /* base MVA */
    long long level_cost;     /* weight of one forward level in the order cost */
    /* admittance matrix, one row per bus, diagonal included (CSR) */
    int *yp, *yj;
    double *G, *B;
    int *ydiag;               /* position of (i,i) in row i */
    /* index maps; -1 where the bus variable is not of that kind */
    int *ix_th;               /* theta_i -> x index (non-slack buses)       */
    int *ix_v;                /* v_i     -> x index (PQ buses)              */
    int *ip_v;                /* v_i     -> p index (generator buses)       */
    int *ip_pg;               /* Pg_i    -> p index (PV buses)              */
} orc_grid;

/* bus voltages and generation recovered from (x, p) */
typedef struct {
    double *vm, *va, *pg;     /* pg valid at PV buses */
} orc_state;

static void *xcalloc(size_t n, size_t s) {
    void *p = calloc(n ? n : 1, s);
    if (!p) abort();
    return p;
}

void orc_grid_free(orc_grid *g) {
    if (!g) return;
    free(g->type); free(g->c2); free(g->c1);
    free(g->yp); free(g->yj); free(g->G); free(g->B); free(g->ydiag);
    free(g->ix_th); free(g->ix_v); free(g->ip_v); free(g->ip_pg);
    free(g);
}

/*
 * Admittance matrix of the pi branch model: series y = 1/(r + j x) between the
 * end buses, half of the total line charging b at each end (no taps, no bus
 * shunts).  Y_ij = Y_ji -= y, Y_ii += y + j b/2, Y_jj += y + j b/2.
 * Parallel branches add up.  G = Re Y, B = Im Y.
 */
orc_grid *orc_grid_new(int n_bus, int n_branch, const int32_t *fr, const int32_t *to,
                       const double *r, const double *x, const double *b,
                       const int8_t *type, const double *c2, const double *c1,
                       double base_mva, long long level_cost) {
    orc_grid *g = xcalloc(1, sizeof *g);
    g->n_bus = n_bus;
    g->n_branch = n_branch;
    g->S = base_mva;
    g->level_cost = level_cost;
    g->type = xcalloc(n_bus, 1);
    g->c2 = xcalloc(n_bus, sizeof(double));
    g->c1 = xcalloc(n_bus, sizeof(double));
    memcpy(g->type, type, n_bus);
    memcpy(g->c2, c2, n_bus * sizeof(double));
    memcpy(g->c1, c1, n_bus * sizeof(double));

    /* dense neighbour marks are fine for an oracle: build the row lists */
    int *deg = xcalloc(n_bus, sizeof(int));
    for (int e = 0; e < n_branch; e++) { deg[fr[e]]++; deg[to[e]]++; }
    /* candidate rows (with duplicates), then merge */
    int *cp = xcalloc(n_bus + 1, sizeof(int));
    for (int i = 0; i < n_bus; i++) cp[i + 1] = cp[i] + deg[i] + 1;
    int *cj = xcalloc(cp[n_bus], sizeof(int));
    double *cg = xcalloc(cp[n_bus], sizeof(double));
    double *cb = xcalloc(cp[n_bus], sizeof(double));
    int *fill = xcalloc(n_bus, sizeof(int));
    for (int i = 0; i < n_bus; i++) { cj[cp[i]] = i; fill[i] = 1; }
    for (int e = 0; e < n_branch; e++) {
        int i = fr[e], j = to[e];
        double den = r[e] * r[e] + x[e] * x[e];
        double ys_re = r[e] / den, ys_im = -x[e] / den;
        /* diagonal */
        cg[cp[i]] += ys_re; cb[cp[i]] += ys_im + 0.5 * b[e];
        cg[cp[j]] += ys_re; cb[cp[j]] += ys_im + 0.5 * b[e];
        /* off-diagonal */
        int k = cp[i] + fill[i]++;
        cj[k] = j; cg[k] = -ys_re; cb[k] = -ys_im;
        k = cp[j] + fill[j]++;
        cj[k] = i; cg[k] = -ys_re; cb[k] = -ys_im;
    }
    /* merge duplicates (parallel branches): sort each row by column */
    g->yp = xcalloc(n_bus + 1, sizeof(int));
    g->yj = xcalloc(cp[n_bus], sizeof(int));
    g->G = xcalloc(cp[n_bus], sizeof(double));
    g->B = xcalloc(cp[n_bus], sizeof(double));
    g->ydiag = xcalloc(n_bus, sizeof(int));
    int nz = 0;
    for (int i = 0; i < n_bus; i++) {
        g->yp[i] = nz;
        int a = cp[i], e = cp[i] + fill[i];
        /* insertion sort by column (rows are short) */
        for (int k = a + 1; k < e; k++) {
            int kj = cj[k]; double kg = cg[k], kb = cb[k];
            int m = k - 1;
            while (m >= a && cj[m] > kj) { cj[m + 1] = cj[m]; cg[m + 1] = cg[m]; cb[m + 1] = cb[m]; m--; }
            cj[m + 1] = kj; cg[m + 1] = kg; cb[m + 1] = kb;
        }
        for (int k = a; k < e; k++) {
            if (nz > g->yp[i] && g->yj[nz - 1] == cj[k]) {
                g->G[nz - 1] += cg[k]; g->B[nz - 1] += cb[k];
            } else {
                g->yj[nz] = cj[k]; g->G[nz] = cg[k]; g->B[nz] = cb[k]; nz++;
            }
        }
        for (int k = g->yp[i]; k < nz; k++) if (g->yj[k] == i) g->ydiag[i] = k;
    }
    g->yp[n_bus] = nz;
    free(deg); free(cp); free(cj); free(cg); free(cb); free(fill);

    /* index maps: x = [theta at PV (asc), theta at PQ (asc), v at PQ (asc)]
                   p = [v at generators incl. slack (asc), Pg at PV (asc)] */
    g->ix_th = xcalloc(n_bus, sizeof(int));
    g->ix_v = xcalloc(n_bus, sizeof(int));
    g->ip_v = xcalloc(n_bus, sizeof(int));
    g->ip_pg = xcalloc(n_bus, sizeof(int));
    int n_pv = 0, n_pq = 0, n_gen = 0;
    g->ref = -1;
    for (int i = 0; i < n_bus; i++) {
        if (type[i] == PV) n_pv++;
        else if (type[i] == PQ) n_pq++;
        else g->ref = i;
        if (type[i] != PQ) n_gen++;
    }
    g->n_gen = n_gen;
    g->n_x = n_pv + 2 * n_pq;
    g->n_p = 2 * n_gen - 1;
    int kpv = 0, kpq = 0, kg = 0;
    for (int i = 0; i < n_bus; i++) {
        g->ix_th[i] = g->ix_v[i] = g->ip_v[i] = g->ip_pg[i] = -1;
        if (type[i] == PV) { g->ix_th[i] = kpv; g->ip_pg[i] = n_gen + kpv; kpv++; }
        if (type[i] == PQ) { g->ix_th[i] = n_pv + kpq; g->ix_v[i] = n_pv + n_pq + kpq; kpq++; }
        if (type[i] != PQ) { g->ip_v[i] = kg++; }
    }
    return g;
}

int orc_n_x(const orc_grid *g) { return g->n_x; }
int orc_n_p(const orc_grid *g) { return g->n_p; }
int orc_ref(const orc_grid *g) { return g->ref; }

void orc_index_maps(const orc_grid *g, int32_t *ix_th, int32_t *ix_v, int32_t *ip_v, int32_t *ip_pg) {
    for (int i = 0; i < g->n_bus; i++) {
        ix_th[i] = g->ix_th[i]; ix_v[i] = g->ix_v[i];
        ip_v[i] = g->ip_v[i]; ip_pg[i] = g->ip_pg[i];
    }
}

static void state_alloc(const orc_grid *g, orc_state *s) {
    s->vm = xcalloc(g->n_bus, sizeof(double));
    s->va = xcalloc(g->n_bus, sizeof(double));
    s->pg = xcalloc(g->n_bus, sizeof(double));
}
static void state_free(orc_state *s) { free(s->vm); free(s->va); free(s->pg); }

static void state_from(const orc_grid *g, const double *x, const double *p, orc_state *s) {
    for (int i = 0; i < g->n_bus; i++) {
        s->va[i] = g->ix_th[i] >= 0 ? x[g->ix_th[i]] : 0.0;   /* theta_slack = 0 */
        s->vm[i] = g->ix_v[i] >= 0 ? x[g->ix_v[i]] : p[g->ip_v[i]];
        s->pg[i] = g->ip_pg[i] >= 0 ? p[g->ip_pg[i]] : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* eq. (2): injections                                                       */
/* ------------------------------------------------------------------------ */

/* P_i = v_i sum_j v_j (G_ij cos(t_i - t_j) + B_ij sin(t_i - t_j)),
   Q_i = v_i sum_j v_j (G_ij sin(t_i - t_j) - B_ij cos(t_i - t_j)), j over i and its neighbours. */
void orc_injections(const orc_grid *g, const double *vm, const double *va, double *P, double *Q) {
    for (int i = 0; i < g->n_bus; i++) {
        double p = 0.0, q = 0.0;
        for (int k = g->yp[i]; k < g->yp[i + 1]; k++) {
            int j = g->yj[k];
            double t = va[i] - va[j];
            double c = cos(t), s = sin(t);
            p += vm[j] * (g->G[k] * c + g->B[k] * s);
            q += vm[j] * (g->G[k] * s - g->B[k] * c);
        }
        P[i] = vm[i] * p;
        Q[i] = vm[i] * q;
    }
}

/* ------------------------------------------------------------------------ */
/* eq. (3): balance equations; rows ordered like x (P_i <-> theta_i, Q_i <-> v_i) */
/* ------------------------------------------------------------------------ */

void orc_residual(const orc_grid *g, const double *x, const double *p,
                  const double *pd, const double *qd, double *out) {
    orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
    double *P = xcalloc(g->n_bus, sizeof(double)), *Q = xcalloc(g->n_bus, sizeof(double));
    orc_injections(g, s.vm, s.va, P, Q);
    for (int i = 0; i < g->n_bus; i++) {
        if (g->ix_th[i] >= 0) out[g->ix_th[i]] = P[i] - s.pg[i] + pd[i];  /* pg = 0 at PQ */
        if (g->ix_v[i] >= 0) out[g->ix_v[i]] = Q[i] + qd[i];
    }
    free(P); free(Q); state_free(&s);
}

/* slack generation Pg_ref = P_ref + Pd_ref, and the cost f */
static double slack_pg(const orc_grid *g, const orc_state *s, const double *pd) {
    int r = g->ref;
    double p = 0.0;
    for (int k = g->yp[r]; k < g->yp[r + 1]; k++) {
        int j = g->yj[k];
        double t = s->va[r] - s->va[j];
        p += s->vm[j] * (g->G[k] * cos(t) + g->B[k] * sin(t));
    }
    return s->vm[r] * p + pd[r];
}

static double gen_pg(const orc_grid *g, const orc_state *s, const double *pd, int i) {
    return i == g->ref ? slack_pg(g, s, pd) : s->pg[i];
}

double orc_objective(const orc_grid *g, const double *x, const double *p, const double *pd) {
    orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
    double f = 0.0;
    for (int i = 0; i < g->n_bus; i++) {
        if (g->type[i] == PQ) continue;
        double P = g->S * gen_pg(g, &s, pd, i);
        f += g->c2[i] * P * P + g->c1[i] * P;
    }
    state_free(&s);
    return f;
}

/* ------------------------------------------------------------------------ */
/* sparse matrices (triplets -> CSC), just enough for the oracle            */
/* ------------------------------------------------------------------------ */

typedef struct { int nr, nc; int *p, *i; double *x; } csc;

typedef struct { int n, cap; int *r, *c; double *v; } trip;

static void trip_add(trip *t, int r, int c, double v) {
    if (t->n == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->r = realloc(t->r, t->cap * sizeof(int));
        t->c = realloc(t->c, t->cap * sizeof(int));
        t->v = realloc(t->v, t->cap * sizeof(double));
        if (!t->r || !t->c || !t->v) abort();
    }
    t->r[t->n] = r; t->c[t->n] = c; t->v[t->n] = v; t->n++;
}
static void trip_free(trip *t) { free(t->r); free(t->c); free(t->v); memset(t, 0, sizeof *t); }

/* duplicates are summed; rows sorted within each column */
static csc trip_to_csc(const trip *t, int nr, int nc) {
    csc A; A.nr = nr; A.nc = nc;
    int *cnt = xcalloc(nc + 1, sizeof(int));
    for (int k = 0; k < t->n; k++) cnt[t->c[k] + 1]++;
    for (int j = 0; j < nc; j++) cnt[j + 1] += cnt[j];
    int *ti = xcalloc(t->n, sizeof(int));
    double *tx = xcalloc(t->n, sizeof(double));
    int *pos = xcalloc(nc, sizeof(int));
    for (int j = 0; j < nc; j++) pos[j] = cnt[j];
    for (int k = 0; k < t->n; k++) { int d = pos[t->c[k]]++; ti[d] = t->r[k]; tx[d] = t->v[k]; }
    A.p = xcalloc(nc + 1, sizeof(int));
    A.i = xcalloc(t->n, sizeof(int));
    A.x = xcalloc(t->n, sizeof(double));
    int nz = 0;
    for (int j = 0; j < nc; j++) {
        A.p[j] = nz;
        int a = cnt[j], e = cnt[j + 1];
        for (int k = a + 1; k < e; k++) {       /* insertion sort by row */
            int ki = ti[k]; double kx = tx[k]; int m = k - 1;
            while (m >= a && ti[m] > ki) { ti[m + 1] = ti[m]; tx[m + 1] = tx[m]; m--; }
            ti[m + 1] = ki; tx[m + 1] = kx;
        }
        for (int k = a; k < e; k++) {
            if (nz > A.p[j] && A.i[nz - 1] == ti[k]) A.x[nz - 1] += tx[k];
            else { A.i[nz] = ti[k]; A.x[nz] = tx[k]; nz++; }
        }
    }
    A.p[nc] = nz;
    free(cnt); free(ti); free(tx); free(pos);
    return A;
}
static void csc_free(csc *A) { free(A->p); free(A->i); free(A->x); memset(A, 0, sizeof *A); }

/* y += A x  (A is nr x nc) */
static void csc_gemv(const csc *A, const double *x, double *y) {
    for (int j = 0; j < A->nc; j++)
        for (int k = A->p[j]; k < A->p[j + 1]; k++) y[A->i[k]] += A->x[k] * x[j];
}
/* y += A^T x */
static void csc_gemv_t(const csc *A, const double *x, double *y) {
    for (int j = 0; j < A->nc; j++) {
        double s = 0.0;
        for (int k = A->p[j]; k < A->p[j + 1]; k++) s += A->x[k] * x[A->i[k]];
        y[j] += s;
    }
}

/* ------------------------------------------------------------------------ */
/* Jacobians (textbook polar form)                                           */
/* ------------------------------------------------------------------------ */

/*
 * For j != i, with t = theta_i - theta_j, c = cos t, s = sin t:
 *   dP_i/dtheta_j =  v_i v_j (G_ij s - B_ij c)     dP_i/dv_j = v_i (G_ij c + B_ij s)
 *   dQ_i/dtheta_j = -v_i v_j (G_ij c + B_ij s)     dQ_i/dv_j = v_i (G_ij s - B_ij c)
 * and on the diagonal
 *   dP_i/dtheta_i = -Q_i - B_ii v_i^2               dP_i/dv_i = P_i / v_i + G_ii v_i
 *   dQ_i/dtheta_i =  P_i - G_ii v_i^2               dQ_i/dv_i = Q_i / v_i - B_ii v_i
 * Each derivative goes to J_x when its variable is in x and to J_p when it is in p;
 * the Pg columns of J_p are -1 on the P row of their bus.
 */
static void jacobians(const orc_grid *g, const orc_state *s, csc *Jx, csc *Jp) {
    int n = g->n_bus;
    double *P = xcalloc(n, sizeof(double)), *Q = xcalloc(n, sizeof(double));
    orc_injections(g, s->vm, s->va, P, Q);
    trip tx = {0}, tp = {0};
    for (int i = 0; i < n; i++) {
        int rP = g->ix_th[i], rQ = g->ix_v[i];
        if (rP < 0 && rQ < 0) continue;                 /* slack: no row */
        double vi = s->vm[i];
        for (int k = g->yp[i]; k < g->yp[i + 1]; k++) {
            int j = g->yj[k];
            double dPdt, dPdv, dQdt, dQdv;
            if (j == i) {
                double Gii = g->G[k], Bii = g->B[k];
                dPdt = -Q[i] - Bii * vi * vi;
                dPdv = P[i] / vi + Gii * vi;
                dQdt = P[i] - Gii * vi * vi;
                dQdv = Q[i] / vi - Bii * vi;
            } else {
                double t = s->va[i] - s->va[j], c = cos(t), sn = sin(t);
                double vj = s->vm[j], G = g->G[k], B = g->B[k];
                dPdt = vi * vj * (G * sn - B * c);
                dPdv = vi * (G * c + B * sn);
                dQdt = -vi * vj * (G * c + B * sn);
                dQdv = vi * (G * sn - B * c);
            }
            int cth = g->ix_th[j];
            if (cth >= 0) {
                if (rP >= 0) trip_add(&tx, rP, cth, dPdt);
                if (rQ >= 0) trip_add(&tx, rQ, cth, dQdt);
            }
            if (g->ix_v[j] >= 0) {
                if (rP >= 0) trip_add(&tx, rP, g->ix_v[j], dPdv);
                if (rQ >= 0) trip_add(&tx, rQ, g->ix_v[j], dQdv);
            } else {
                if (rP >= 0) trip_add(&tp, rP, g->ip_v[j], dPdv);
                if (rQ >= 0) trip_add(&tp, rQ, g->ip_v[j], dQdv);
            }
        }
        if (g->ip_pg[i] >= 0) trip_add(&tp, rP, g->ip_pg[i], -1.0);
    }
    *Jx = trip_to_csc(&tx, g->n_x, g->n_x);
    *Jp = trip_to_csc(&tp, g->n_x, g->n_p);
    trip_free(&tx); trip_free(&tp);
    free(P); free(Q);
}

/* dense copies for small test cases: column-major n_x*n_x and n_x*n_p */
void orc_jacobians_dense(const orc_grid *g, const double *x, const double *p, double *jx, double *jp) {
    orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
    csc Jx, Jp; jacobians(g, &s, &Jx, &Jp);
    memset(jx, 0, sizeof(double) * g->n_x * g->n_x);
    memset(jp, 0, sizeof(double) * g->n_x * g->n_p);
    for (int j = 0; j < Jx.nc; j++)
        for (int k = Jx.p[j]; k < Jx.p[j + 1]; k++) jx[(size_t)j * g->n_x + Jx.i[k]] = Jx.x[k];
    for (int j = 0; j < Jp.nc; j++)
        for (int k = Jp.p[j]; k < Jp.p[j + 1]; k++) jp[(size_t)j * g->n_x + Jp.i[k]] = Jp.x[k];
    csc_free(&Jx); csc_free(&Jp); state_free(&s);
}

/* ------------------------------------------------------------------------ */
/* static ordering: minimum weighted fill on the bus graph                   */
/* ------------------------------------------------------------------------ */

/*
 * Graph: the non-slack buses, an edge wherever a branch joins two of them.
 * Eliminating bus e joins its remaining neighbours into a clique; each pair
 * (a, b) of them that is not yet adjacent adds w_a * w_b entries to L, with
 * w = 1 for a PV bus and 2 for a PQ bus (its x variables).  Repeatedly
 * eliminate the remaining bus that adds the fewest (ties: the smallest sum of
 * w over its remaining neighbours, then the smallest bus id).  The elimination
 * graph is a dense bit matrix; after each elimination the scores of all buses
 * within two steps of it are recomputed from the matrix (no other score can
 * change), which is slow but plainly correct.
 * Each bus contributes its x variables in the order theta, then v.
 * perm[q] = x index of the variable eliminated q-th; bus_order[k] = bus id.
 */
/*
 * Exact minimum degree: repeatedly eliminate the remaining bus of smallest
 * current degree (ties: smallest bus id); its remaining neighbours become a
 * clique.  Same graph and output as mf_order below.
 */
static void md_order(const orc_grid *g, int *perm, int *bus_order, int *n_elim) {
    int n = g->n_bus;
    size_t words = (size_t)(n + 63) / 64;
    uint64_t *adj = xcalloc((size_t)n * words, sizeof(uint64_t));
    int *deg = xcalloc(n, sizeof(int));
    char *alive = xcalloc(n, 1);
#define HAS(a, b) ((adj[(size_t)(a) * words + (b) / 64] >> ((b) % 64)) & 1u)
#define SET(a, b) (adj[(size_t)(a) * words + (b) / 64] |= (uint64_t)1 << ((b) % 64))
#define CLR(a, b) (adj[(size_t)(a) * words + (b) / 64] &= ~((uint64_t)1 << ((b) % 64)))
    for (int i = 0; i < n; i++) alive[i] = g->type[i] != REF;
    for (int i = 0; i < n; i++) {
        if (!alive[i]) continue;
        for (int k = g->yp[i]; k < g->yp[i + 1]; k++) {
            int j = g->yj[k];
            if (j != i && alive[j] && !HAS(i, j)) { SET(i, j); deg[i]++; }
        }
    }
    int *nb = xcalloc(n, sizeof(int));
    int cnt = 0, q = 0;
    for (;;) {
        int best = -1;
        for (int i = 0; i < n; i++)
            if (alive[i] && (best < 0 || deg[i] < deg[best])) best = i;
        if (best < 0) break;
        int m = 0;
        for (int j = 0; j < n; j++) if (alive[j] && j != best && HAS(best, j)) nb[m++] = j;
        alive[best] = 0;
        for (int a = 0; a < m; a++) { CLR(nb[a], best); deg[nb[a]]--; }
        for (int a = 0; a < m; a++)
            for (int c = a + 1; c < m; c++)
                if (!HAS(nb[a], nb[c])) { SET(nb[a], nb[c]); SET(nb[c], nb[a]); deg[nb[a]]++; deg[nb[c]]++; }
        bus_order[cnt++] = best;
        perm[q++] = g->ix_th[best];
        if (g->ix_v[best] >= 0) perm[q++] = g->ix_v[best];
    }
#undef HAS
#undef SET
#undef CLR
    *n_elim = cnt;
    free(adj); free(deg); free(alive); free(nb);
}

/*
 * Cost of an elimination order, replayed on a fresh elimination graph: the
 * factor entries outside the bus blocks (sum over buses of w_k times the
 * weight of the neighbours it has when eliminated, w as in mf_order) times
 * n_dirs, plus the grid's level_cost per forward level (a bus's level is one
 * more than the highest level of the buses whose elimination reached it).
 * level_cost is a parameter of the ordering rule (the paper gives none, it
 * relies on a host LU), passed in with the grid.
 */
static long long order_cost(const orc_grid *g, const int *bus_order, int n_elim, long long n_dirs) {
    int n = g->n_bus;
    size_t words = (size_t)(n + 63) / 64;
    uint64_t *adj = xcalloc((size_t)n * words, sizeof(uint64_t));
    char *alive = xcalloc(n, 1);
    int *lev = xcalloc(n, sizeof(int));
#define HAS(a, b) ((adj[(size_t)(a) * words + (b) / 64] >> ((b) % 64)) & 1u)
#define SET(a, b) (adj[(size_t)(a) * words + (b) / 64] |= (uint64_t)1 << ((b) % 64))
    for (int i = 0; i < n; i++) alive[i] = g->type[i] != REF;
    for (int i = 0; i < n; i++) {
        if (!alive[i]) continue;
        for (int k = g->yp[i]; k < g->yp[i + 1]; k++) {
            int j = g->yj[k];
            if (j != i && alive[j]) SET(i, j);
        }
    }
    int *nb = xcalloc(n, sizeof(int));
    long long entries = 0;
    int n_lev = 0;
    for (int k = 0; k < n_elim; k++) {
        int e = bus_order[k];
        alive[e] = 0;
        int m = 0;                                  /* remaining neighbours of e, from its row of bits */
        for (size_t wd = 0; wd < words; wd++) {
            uint64_t bits = adj[(size_t)e * words + wd];
            while (bits) {
                int j = (int)(wd * 64) + __builtin_ctzll(bits);
                bits &= bits - 1;
                if (alive[j]) nb[m++] = j;
            }
        }
        long long s = 0;
        for (int a = 0; a < m; a++) {
            int j = nb[a];
            s += g->type[j] == PQ ? 2 : 1;
            if (lev[j] < lev[e] + 1) lev[j] = lev[e] + 1;
            for (int c = 0; c < m; c++)
                if (c != a) SET(j, nb[c]);
        }
        entries += (g->type[e] == PQ ? 2 : 1) * s;
        if (lev[e] + 1 > n_lev) n_lev = lev[e] + 1;
    }
#undef HAS
#undef SET
    free(adj); free(alive); free(lev); free(nb);
    return entries * n_dirs + g->level_cost * n_lev;
}

/* the remaining neighbours of bus v in the elimination graph, read from its row of bits */
static int mf_row(const uint64_t *adj, size_t words, int v, const char *alive, int *out) {
    int m = 0;
    const uint64_t *row = adj + (size_t)v * words;
    for (size_t k = 0; k < words; k++) {
        uint64_t bits = row[k];
        while (bits) {
            int j = (int)(k * 64) + __builtin_ctzll(bits);
            bits &= bits - 1;
            if (alive[j] && j != v) out[m++] = j;
        }
    }
    return m;
}

static void mf_order(const orc_grid *g, int *perm, int *bus_order, int *n_elim) {
    int n = g->n_bus;
    size_t words = (size_t)(n + 63) / 64;
    uint64_t *adj = xcalloc((size_t)n * words, sizeof(uint64_t));
    char *alive = xcalloc(n, 1);
    int *w = xcalloc(n, sizeof(int));
    long long *fill = xcalloc(n, sizeof(long long)), *wdeg = xcalloc(n, sizeof(long long));
    int *nb = xcalloc(n, sizeof(int)), *nb2 = xcalloc(n, sizeof(int)), *hit = xcalloc(n, sizeof(int));
#define HAS(a, b) ((adj[(size_t)(a) * words + (b) / 64] >> ((b) % 64)) & 1u)
#define SET(a, b) (adj[(size_t)(a) * words + (b) / 64] |= (uint64_t)1 << ((b) % 64))
#define CLR(a, b) (adj[(size_t)(a) * words + (b) / 64] &= ~((uint64_t)1 << ((b) % 64)))
    for (int i = 0; i < n; i++) {
        alive[i] = g->type[i] != REF;
        w[i] = g->type[i] == PQ ? 2 : 1;
        hit[i] = -1;
    }
    for (int i = 0; i < n; i++) {
        if (!alive[i]) continue;
        for (int k = g->yp[i]; k < g->yp[i + 1]; k++) {
            int j = g->yj[k];
            if (j != i && alive[j]) SET(i, j);
        }
    }
    /* score of bus v: the weight of its non-adjacent neighbour pairs, and its weighted degree */
#define SCORE(v)                                                                   \
    do {                                                                           \
        int m_ = mf_row(adj, words, (v), alive, nb2);                              \
        long long f_ = 0, s_ = 0;                                                  \
        for (int a_ = 0; a_ < m_; a_++) {                                          \
            s_ += w[nb2[a_]];                                                      \
            for (int c_ = a_ + 1; c_ < m_; c_++)                                   \
                if (!HAS(nb2[a_], nb2[c_])) f_ += (long long)w[nb2[a_]] * w[nb2[c_]]; \
        }                                                                          \
        fill[v] = f_;                                                              \
        wdeg[v] = s_;                                                              \
    } while (0)
    for (int i = 0; i < n; i++) if (alive[i]) SCORE(i);
    int cnt = 0, q = 0;
    for (;;) {
        int best = -1;
        for (int i = 0; i < n; i++) {
            if (!alive[i]) continue;
            if (best < 0 || fill[i] < fill[best] || (fill[i] == fill[best] && wdeg[i] < wdeg[best])) best = i;
        }
        if (best < 0) break;
        int m = mf_row(adj, words, best, alive, nb);
        alive[best] = 0;
        for (int a = 0; a < m; a++) CLR(nb[a], best);
        for (int a = 0; a < m; a++)
            for (int c = a + 1; c < m; c++)
                if (!HAS(nb[a], nb[c])) { SET(nb[a], nb[c]); SET(nb[c], nb[a]); }
        /* rescore every bus within two steps of the eliminated one: its former
           neighbours and their neighbours (no other score can change) */
        for (int a = 0; a < m; a++) {
            hit[nb[a]] = cnt;
            int m2 = mf_row(adj, words, nb[a], alive, nb2);
            for (int c = 0; c < m2; c++) hit[nb2[c]] = cnt;
        }
        for (int j = 0; j < n; j++) if (alive[j] && hit[j] == cnt) SCORE(j);
        bus_order[cnt++] = best;
        perm[q++] = g->ix_th[best];
        if (g->ix_v[best] >= 0) perm[q++] = g->ix_v[best];
    }
#undef SCORE
#undef HAS
#undef SET
#undef CLR
    *n_elim = cnt;
    free(adj); free(alive); free(w); free(fill); free(wdeg); free(nb); free(nb2); free(hit);
}

/*
 * The static order: whichever of minimum degree and minimum weighted fill has
 * the smaller order_cost for the directions of a full reduced Hessian (n_p);
 * ties go to minimum degree.
 */
static void static_order(const orc_grid *g, int *perm, int *bus_order, int *n_elim) {
    int nx = g->n_x, nb = g->n_bus;
    int *perm2 = xcalloc(nx > 0 ? nx : 1, sizeof(int)), *bo2 = xcalloc(nb, sizeof(int));
    int n1 = 0, n2 = 0;
    md_order(g, perm, bus_order, &n1);
    mf_order(g, perm2, bo2, &n2);
    if (order_cost(g, bo2, n2, g->n_p) < order_cost(g, bus_order, n1, g->n_p)) {
        memcpy(perm, perm2, (size_t)nx * sizeof(int));
        memcpy(bus_order, bo2, (size_t)n2 * sizeof(int));
        n1 = n2;
    }
    *n_elim = n1;
    free(perm2); free(bo2);
}

/* One candidate order on its own (which = 0: minimum degree, 1: minimum weighted
 * fill, 2: the static choice); bus_order has n_bus entries.  Returns n_elim. */
int orc_order(const orc_grid *g, int which, int32_t *bus_order) {
    int *perm = xcalloc(g->n_x > 0 ? g->n_x : 1, sizeof(int)), *bo = xcalloc(g->n_bus, sizeof(int));
    int n = 0;
    if (which == 0) md_order(g, perm, bo, &n);
    else if (which == 1) mf_order(g, perm, bo, &n);
    else static_order(g, perm, bo, &n);
    for (int k = 0; k < n; k++) bus_order[k] = bo[k];
    free(perm); free(bo);
    return n;
}

/* ------------------------------------------------------------------------ */
/* left-looking sparse LU of B = A(perm, perm), no numerical pivoting       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n;
    int *perm;        /* internal q -> x index */
    int *iperm;       /* x index -> q          */
    csc L;            /* unit lower, diagonal not stored */
    csc U;            /* upper, diagonal stored last in each column */
} orc_lu;

static void lu_free(orc_lu *F) { free(F->perm); free(F->iperm); csc_free(&F->L); csc_free(&F->U); }

/*
 * Column k of B: scatter it into a dense work vector w; for j = 0..k-1 in
 * increasing order, w[j] is final (it is U_jk) and column j of L is applied:
 * w[i] -= L_ij w[j].  Then U(0:k, k) = w(0:k), L(k+1:n, k) = w(k+1:n) / w[k].
 * Exact zeros are skipped, which changes no value.
 * Returns 0, or -1 if a pivot is not above tau * max|A|.
 */
static int lu_factor(const csc *A, const int *perm, orc_lu *F) {
    int n = A->nc;
    F->n = n;
    F->perm = xcalloc(n, sizeof(int));
    F->iperm = xcalloc(n, sizeof(int));
    for (int q = 0; q < n; q++) { F->perm[q] = perm[q]; F->iperm[perm[q]] = q; }
    double amax = 0.0;
    for (int k = 0; k < A->p[n]; k++) if (fabs(A->x[k]) > amax) amax = fabs(A->x[k]);
    double *w = xcalloc(n, sizeof(double));
    char *nzw = xcalloc(n, 1);
    trip tu = {0};
    /* L columns are needed while factoring: keep them as growing CSC */
    int *Lp = xcalloc(n + 1, sizeof(int));
    int lcap = 1024, lnz = 0;
    int *Li = xcalloc(lcap, sizeof(int));
    double *Lx = xcalloc(lcap, sizeof(double));
    int status = 0;
    for (int k = 0; k < n; k++) {
        int col = perm[k];
        for (int t = A->p[col]; t < A->p[col + 1]; t++) {
            int i = F->iperm[A->i[t]];
            w[i] = A->x[t]; nzw[i] = 1;
        }
        for (int j = 0; j < k; j++) {
            if (!nzw[j] || w[j] == 0.0) continue;
            double ujk = w[j];
            for (int t = Lp[j]; t < Lp[j + 1]; t++) { w[Li[t]] -= Lx[t] * ujk; nzw[Li[t]] = 1; }
        }
        double piv = w[k];
        if (!(fabs(piv) > 1e-14 * amax)) status = -1;
        for (int j = 0; j < k; j++) if (nzw[j] && w[j] != 0.0) trip_add(&tu, j, k, w[j]);
        trip_add(&tu, k, k, piv);
        Lp[k] = lnz;
        for (int i = k + 1; i < n; i++) {
            if (!nzw[i] || w[i] == 0.0) continue;
            if (lnz == lcap) {
                lcap *= 2;
                Li = realloc(Li, lcap * sizeof(int)); Lx = realloc(Lx, lcap * sizeof(double));
                if (!Li || !Lx) abort();
            }
            Li[lnz] = i; Lx[lnz] = w[i] / piv; lnz++;
        }
        Lp[k + 1] = lnz;
        for (int i = 0; i < n; i++) { w[i] = 0.0; nzw[i] = 0; }
    }
    F->L.nr = F->L.nc = n; F->L.p = Lp; F->L.i = Li; F->L.x = Lx;
    F->U = trip_to_csc(&tu, n, n);
    trip_free(&tu);
    free(w); free(nzw);
    return status;
}

/* solve J v = b in place (b, v indexed like x) */
static void lu_solve(const orc_lu *F, double *b) {
    int n = F->n;
    double *y = xcalloc(n, sizeof(double));
    for (int q = 0; q < n; q++) y[q] = b[F->perm[q]];
    for (int j = 0; j < n; j++)                                   /* L y = Pb */
        for (int t = F->L.p[j]; t < F->L.p[j + 1]; t++) y[F->L.i[t]] -= F->L.x[t] * y[j];
    for (int j = n - 1; j >= 0; j--) {                            /* U v = y  */
        int last = F->U.p[j + 1] - 1;                             /* diagonal */
        y[j] /= F->U.x[last];
        for (int t = F->U.p[j]; t < last; t++) y[F->U.i[t]] -= F->U.x[t] * y[j];
    }
    for (int q = 0; q < n; q++) b[F->perm[q]] = y[q];
    free(y);
}

/* solve J^T v = b in place: U^T w = Pb, then L^T v' = w */
static void lu_solve_t(const orc_lu *F, double *b) {
    int n = F->n;
    double *y = xcalloc(n, sizeof(double));
    for (int q = 0; q < n; q++) y[q] = b[F->perm[q]];
    for (int j = 0; j < n; j++) {                                 /* U^T, forward */
        int last = F->U.p[j + 1] - 1;
        double s = y[j];
        for (int t = F->U.p[j]; t < last; t++) s -= F->U.x[t] * y[F->U.i[t]];
        y[j] = s / F->U.x[last];
    }
    for (int j = n - 1; j >= 0; j--) {                            /* L^T, backward */
        double s = y[j];
        for (int t = F->L.p[j]; t < F->L.p[j + 1]; t++) s -= F->L.x[t] * y[F->L.i[t]];
        y[j] = s;
    }
    for (int q = 0; q < n; q++) b[F->perm[q]] = y[q];
    free(y);
}

static int factor_at(const orc_grid *g, const orc_state *s, orc_lu *F, csc *Jp_out) {
    csc Jx, Jp;
    jacobians(g, s, &Jx, &Jp);
    int *perm = xcalloc(g->n_x, sizeof(int)), *bo = xcalloc(g->n_bus, sizeof(int)), nb;
    static_order(g, perm, bo, &nb);
    int st = lu_factor(&Jx, perm, F);
    free(perm); free(bo);
    csc_free(&Jx);
    if (Jp_out) *Jp_out = Jp; else csc_free(&Jp);
    return st;
}

/* solve J_x X = R (trans = 0) or J_x^T X = R (trans = 1), R column-major n_x * nrhs, in place */
int orc_solve(const orc_grid *g, const double *x, const double *p, double *R, int nrhs, int trans) {
    orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
    orc_lu F; int st = factor_at(g, &s, &F, NULL);
    for (int c = 0; c < nrhs; c++) {
        if (trans) lu_solve_t(&F, R + (size_t)c * g->n_x);
        else lu_solve(&F, R + (size_t)c * g->n_x);
    }
    lu_free(&F); state_free(&s);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Newton-Raphson power flow (section 3.2)                                   */
/* ------------------------------------------------------------------------ */

/* x holds the initial guess on entry and the solution on exit.
   Returns 0 on convergence (||g||_inf <= tol), 1 if not converged, -1 singular. */
int orc_newton(const orc_grid *g, const double *p, const double *pd, const double *qd,
               double *x, double tol, int max_iter, int *iters, double *resid) {
    double *r = xcalloc(g->n_x, sizeof(double));
    int it = 0, status = 1;
    for (;;) {
        orc_residual(g, x, p, pd, qd, r);
        double nr = 0.0;
        for (int k = 0; k < g->n_x; k++) if (fabs(r[k]) > nr || isnan(r[k])) nr = isnan(r[k]) ? INFINITY : fabs(r[k]);
        *resid = nr;
        if (nr <= tol) { status = 0; break; }
        if (it >= max_iter || !isfinite(nr)) break;
        orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
        orc_lu F; int st = factor_at(g, &s, &F, NULL);
        state_free(&s);
        if (st) { lu_free(&F); status = -1; break; }
        lu_solve(&F, r);                                /* r <- J_x^{-1} g */
        for (int k = 0; k < g->n_x; k++) x[k] -= r[k];
        lu_free(&F);
        it++;
    }
    *iters = it;
    free(r);
    return status;
}

/* ------------------------------------------------------------------------ */
/* first-order adjoint, eq. (6)-(7)                                          */
/* ------------------------------------------------------------------------ */

/* c'_k and c''_k of the quadratic cost as a function of Pg in p.u. */
static double dcost(const orc_grid *g, int i, double pg) { return 2.0 * g->c2[i] * g->S * g->S * pg + g->c1[i] * g->S; }
static double d2cost(const orc_grid *g, int i) { return 2.0 * g->c2[i] * g->S * g->S; }

/*
 * Gradient of P_ref (slack injection) with respect to (x, p), as a dense
 * vector over the combined index u = (x, p) of length n_x + n_p.
 */
static void grad_pref(const orc_grid *g, const orc_state *s, double *gu) {
    int r = g->ref, nx = g->n_x;
    memset(gu, 0, sizeof(double) * (g->n_x + g->n_p));
    double vr = s->vm[r], Pr = 0.0;
    for (int k = g->yp[r]; k < g->yp[r + 1]; k++) {
        int j = g->yj[k];
        double t = s->va[r] - s->va[j];
        Pr += vr * s->vm[j] * (g->G[k] * cos(t) + g->B[k] * sin(t));
    }
    for (int k = g->yp[r]; k < g->yp[r + 1]; k++) {
        int j = g->yj[k];
        double G = g->G[k], B = g->B[k];
        if (j == r) {
            gu[nx + g->ip_v[r]] += Pr / vr + G * vr;
            continue;
        }
        double t = s->va[r] - s->va[j], c = cos(t), sn = sin(t), vj = s->vm[j];
        if (g->ix_th[j] >= 0) gu[g->ix_th[j]] += vr * vj * (G * sn - B * c);
        double dv = vr * (G * c + B * sn);
        if (g->ix_v[j] >= 0) gu[g->ix_v[j]] += dv; else gu[nx + g->ip_v[j]] += dv;
    }
}

/* lambda (indexed like g rows = like x), grad F (n_p), F.  Returns LU status. */
int orc_adjoint(const orc_grid *g, const double *x, const double *p, const double *pd, const double *qd,
                double *lambda, double *grad, double *F) {
    (void)qd;
    orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
    int nx = g->n_x, np = g->n_p;
    double *gu = xcalloc(nx + np, sizeof(double));
    grad_pref(g, &s, gu);
    double cref = dcost(g, g->ref, slack_pg(g, &s, pd));
    /* grad_x f = c'_ref grad_x P_ref ;  lambda = -J_x^{-T} grad_x f */
    for (int k = 0; k < nx; k++) lambda[k] = -cref * gu[k];
    orc_lu LU; csc Jp;
    int st = factor_at(g, &s, &LU, &Jp);
    lu_solve_t(&LU, lambda);
    /* grad_p F = grad_p f + J_p^T lambda */
    for (int k = 0; k < np; k++) grad[k] = cref * gu[nx + k];
    for (int i = 0; i < g->n_bus; i++) if (g->ip_pg[i] >= 0) grad[g->ip_pg[i]] += dcost(g, i, s.pg[i]);
    csc_gemv_t(&Jp, lambda, grad);
    *F = orc_objective(g, x, p, pd);
    lu_free(&LU); csc_free(&Jp); free(gu); state_free(&s);
    return st;
}

/* ------------------------------------------------------------------------ */
/* explicit Hessian of the Lagrangian over u = (x, p)                        */
/* ------------------------------------------------------------------------ */

/*
 * l = f + lambda^T g.  With mu_i = lambda of the P row of bus i (and, for the
 * slack, mu = c'_ref since f depends on P_ref) and nu_i = lambda of the Q row
 * (0 where there is none):
 *   Hess l = sum_i mu_i Hess P_i + nu_i Hess Q_i
 *            + c''_ref grad P_ref grad P_ref^T + sum_{PV k} c''_k e_Pg_k e_Pg_k^T.
 * Each P_i (Q_i) is v_i^2 G_ii (-v_i^2 B_ii) plus one term h = v_i v_j C(t),
 * t = theta_i - theta_j, per neighbour j, with C = G cos t + B sin t
 * (C = G sin t - B cos t for Q).  Hess h in (v_i, v_j, t):
 *   d2h/dv_i dv_j = C,  d2h/dv_i dt = v_j C',  d2h/dv_j dt = v_i C',
 *   d2h/dt^2 = v_i v_j C'',  d2h/dv_i^2 = d2h/dv_j^2 = 0,
 * and t maps to (theta_i, theta_j) with signs (+1, -1).  theta_slack is not a
 * variable, so its rows and columns are dropped.
 */
static int uidx_th(const orc_grid *g, int i) { return g->ix_th[i]; }
static int uidx_v(const orc_grid *g, int i) { return g->ix_v[i] >= 0 ? g->ix_v[i] : g->n_x + g->ip_v[i]; }

static void hadd(trip *t, int a, int b, double v) {
    if (a < 0 || b < 0 || v == 0.0) return;
    trip_add(t, a, b, v);
}

static csc lagrangian_hessian(const orc_grid *g, const orc_state *s, const double *pd, const double *lambda) {
    int n = g->n_bus, nu = g->n_x + g->n_p;
    double *mu = xcalloc(n, sizeof(double)), *nuw = xcalloc(n, sizeof(double));
    double cref = dcost(g, g->ref, slack_pg(g, s, pd));
    for (int i = 0; i < n; i++) {
        mu[i] = g->ix_th[i] >= 0 ? lambda[g->ix_th[i]] : cref;
        nuw[i] = g->ix_v[i] >= 0 ? lambda[g->ix_v[i]] : 0.0;
    }
    trip t = {0};
    for (int i = 0; i < n; i++) {
        double vi = s->vm[i];
        int ui_v = uidx_v(g, i), ui_t = uidx_th(g, i);
        for (int k = g->yp[i]; k < g->yp[i + 1]; k++) {
            int j = g->yj[k];
            double G = g->G[k], B = g->B[k];
            if (j == i) {
                /* mu_i G_ii v_i^2 - nu_i B_ii v_i^2 */
                hadd(&t, ui_v, ui_v, 2.0 * (mu[i] * G - nuw[i] * B));
                continue;
            }
            double vj = s->vm[j], tt = s->va[i] - s->va[j], c = cos(tt), sn = sin(tt);
            /* weighted C, C', C'' of the P and Q terms */
            double C = mu[i] * (G * c + B * sn) + nuw[i] * (G * sn - B * c);
            double C1 = mu[i] * (-G * sn + B * c) + nuw[i] * (G * c + B * sn);
            double C2 = -C;
            int uj_v = uidx_v(g, j), uj_t = uidx_th(g, j);
            /* (v_i, v_j) */
            hadd(&t, ui_v, uj_v, C); hadd(&t, uj_v, ui_v, C);
            /* (v_i, t) and (v_j, t), t -> +theta_i, -theta_j */
            hadd(&t, ui_v, ui_t, vj * C1); hadd(&t, ui_t, ui_v, vj * C1);
            hadd(&t, ui_v, uj_t, -vj * C1); hadd(&t, uj_t, ui_v, -vj * C1);
            hadd(&t, uj_v, ui_t, vi * C1); hadd(&t, ui_t, uj_v, vi * C1);
            hadd(&t, uj_v, uj_t, -vi * C1); hadd(&t, uj_t, uj_v, -vi * C1);
            /* (t, t) */
            double tt2 = vi * vj * C2;
            hadd(&t, ui_t, ui_t, tt2); hadd(&t, uj_t, uj_t, tt2);
            hadd(&t, ui_t, uj_t, -tt2); hadd(&t, uj_t, ui_t, -tt2);
        }
    }
    /* c''_ref grad P_ref grad P_ref^T */
    double *gu = xcalloc(nu, sizeof(double));
    grad_pref(g, s, gu);
    double c2r = d2cost(g, g->ref);
    for (int a = 0; a < nu; a++) {
        if (gu[a] == 0.0) continue;
        for (int b = 0; b < nu; b++) if (gu[b] != 0.0) hadd(&t, a, b, c2r * gu[a] * gu[b]);
    }
    for (int i = 0; i < n; i++) if (g->ip_pg[i] >= 0) hadd(&t, g->n_x + g->ip_pg[i], g->n_x + g->ip_pg[i], d2cost(g, i));
    csc H = trip_to_csc(&t, nu, nu);
    trip_free(&t); free(gu); free(mu); free(nuw);
    return H;
}

/* dense Hessian of the Lagrangian (column-major (n_x+n_p)^2), small cases */
void orc_lagrangian_hessian_dense(const orc_grid *g, const double *x, const double *p, const double *pd,
                                  const double *lambda, double *out) {
    orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
    csc H = lagrangian_hessian(g, &s, pd, lambda);
    int nu = g->n_x + g->n_p;
    memset(out, 0, sizeof(double) * nu * nu);
    for (int j = 0; j < nu; j++)
        for (int k = H.p[j]; k < H.p[j + 1]; k++) out[(size_t)j * nu + H.i[k]] = H.x[k];
    csc_free(&H); state_free(&s);
}

/* ------------------------------------------------------------------------ */
/* reduced Hessian-vector products, eq. (9)-(10), one direction at a time   */
/* ------------------------------------------------------------------------ */

/*
 * W: n_p x N column-major (ldw >= n_p), HW: n_p x N column-major (ldh >= n_p).
 * For each column w:  b = J_p w;  z = -J_x^{-1} b;  y = [Hess l](z, w);
 * psi = -J_x^{-T} y_x;  Hw = y_p + J_p^T psi.
 * The per-state data (adjoint, LU, J_p, the Lagrangian Hessian) is formed once;
 * every column then runs the same steps on its own work vectors, so the
 * columns may be shared out among threads without changing any result.
 * Returns the LU status (0 ok, -1 singular pivot).
 */
typedef struct {
    const orc_grid *g;
    const orc_lu *LU;
    const csc *Jp, *H;
    const double *W;
    int ldw, N, ldh, n_threads, t;
    double *HW;
} hv_job;

static void hessvec_column(const hv_job *j, int c, double *v, double *y) {
    int nx = j->g->n_x, np = j->g->n_p, nu = nx + np;
    const double *w = j->W + (size_t)c * j->ldw;
    memset(v, 0, sizeof(double) * nu);
    csc_gemv(j->Jp, w, v);                     /* b = J_p w       */
    lu_solve(j->LU, v);                        /* J_x^{-1} b      */
    for (int k = 0; k < nx; k++) v[k] = -v[k]; /* z               */
    memcpy(v + nx, w, sizeof(double) * np);    /* v = (z, w)      */
    memset(y, 0, sizeof(double) * nu);
    csc_gemv(j->H, v, y);                      /* y = [Hess l] v  */
    for (int k = 0; k < nx; k++) y[k] = -y[k];
    lu_solve_t(j->LU, y);                      /* psi = -J^{-T} y_x */
    double *out = j->HW + (size_t)c * j->ldh;
    memcpy(out, y + nx, sizeof(double) * np);  /* y_p             */
    csc_gemv_t(j->Jp, y, out);                 /* + J_p^T psi     */
}

static void *hessvec_worker(void *arg) {
    const hv_job *j = arg;
    int nu = j->g->n_x + j->g->n_p;
    double *v = xcalloc(nu, sizeof(double)), *y = xcalloc(nu, sizeof(double));
    for (int c = j->t; c < j->N; c += j->n_threads) hessvec_column(j, c, v, y);
    free(v); free(y);
    return NULL;
}

/* n_threads <= 1: one thread, columns in order; else thread t takes the columns
 * t, t + n_threads, ...  */
int orc_hessvec_threads(const orc_grid *g, const double *x, const double *p, const double *pd, const double *qd,
                        const double *W, int ldw, int N, double *HW, int ldh, int n_threads) {
    int nx = g->n_x, np = g->n_p;
    orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
    double *lambda = xcalloc(nx, sizeof(double)), *grad = xcalloc(np, sizeof(double)), F;
    int st = orc_adjoint(g, x, p, pd, qd, lambda, grad, &F);
    orc_lu LU; csc Jp;
    st |= factor_at(g, &s, &LU, &Jp);
    csc H = lagrangian_hessian(g, &s, pd, lambda);
    if (n_threads > N) n_threads = N;
    if (n_threads < 1) n_threads = 1;
    hv_job *jobs = xcalloc(n_threads, sizeof(hv_job));
    pthread_t *tid = xcalloc(n_threads, sizeof(pthread_t));
    for (int t = 0; t < n_threads; t++) {
        hv_job j = {g, &LU, &Jp, &H, W, ldw, N, ldh, n_threads, t, HW};
        jobs[t] = j;
    }
    int started = 1;
    for (int t = 1; t < n_threads; t++) {
        if (pthread_create(&tid[t], NULL, hessvec_worker, &jobs[t]) != 0) break;
        started++;
    }
    for (int t = started; t < n_threads; t++) hessvec_worker(&jobs[t]);   /* threads that did not start */
    hessvec_worker(&jobs[0]);
    for (int t = 1; t < started; t++) pthread_join(tid[t], NULL);
    free(jobs); free(tid);
    csc_free(&H); csc_free(&Jp); lu_free(&LU);
    free(lambda); free(grad); state_free(&s);
    return st;
}

int orc_hessvec(const orc_grid *g, const double *x, const double *p, const double *pd, const double *qd,
                const double *W, int ldw, int N, double *HW, int ldh) {
    return orc_hessvec_threads(g, x, p, pd, qd, W, ldw, N, HW, ldh, 1);
}

/* ------------------------------------------------------------------------ */
/* symbolic data, derived from scratch for bit-exact comparison             */
/* ------------------------------------------------------------------------ */

/*
 * Ordering from static_order.  Patterns from a structural (boolean) left-looking
 * factorization of the permuted J_x pattern at the variable level: column k
 * gathers the rows of column k of B and, for every j < k already reached, the
 * rows of L(:, j).  J_x entries are taken as structurally nonzero wherever the
 * textbook Jacobian has a term (bus i coupled to itself or a neighbour j).
 * Levels: bus e (in elimination order) depends on every earlier bus owning a
 * column of the L rows of e; level(e) = 1 + max level of those (0 if none).
 *
 * Outputs (CSR by rows of the permuted matrix):
 *   perm[n_x]; bus_order[n_elim]; level[n_elim];
 *   Lp[n_x+1], Lj[nnzL]  strictly lower part of L;
 *   Up[n_x+1], Uj[nnzU]  upper part of U including the diagonal.
 * Call with NULL arrays to get nnzL, nnzU and n_elim only.
 */
int orc_symbolic(const orc_grid *g, int32_t *perm_out, int32_t *bus_order_out, int32_t *level_out,
                 int32_t *Lp_out, int32_t *Lj_out, int32_t *Up_out, int32_t *Uj_out,
                 int64_t *nnzL, int64_t *nnzU, int32_t *n_elim) {
    int nx = g->n_x, n = g->n_bus;
    int *perm = xcalloc(nx, sizeof(int)), *bo = xcalloc(n, sizeof(int)), nb = 0;
    static_order(g, perm, bo, &nb);
    int *iperm = xcalloc(nx, sizeof(int));
    for (int q = 0; q < nx; q++) iperm[perm[q]] = q;
    /* structural J_x pattern by columns, in permuted indices */
    trip t = {0};
    for (int i = 0; i < n; i++) {
        int rows[2] = {g->ix_th[i], g->ix_v[i]};
        for (int k = g->yp[i]; k < g->yp[i + 1]; k++) {
            int j = g->yj[k];
            int cols[2] = {g->ix_th[j], g->ix_v[j]};
            for (int a = 0; a < 2; a++) for (int b = 0; b < 2; b++)
                if (rows[a] >= 0 && cols[b] >= 0) trip_add(&t, iperm[rows[a]], iperm[cols[b]], 1.0);
        }
    }
    csc A = trip_to_csc(&t, nx, nx);
    trip_free(&t);
    /* boolean left-looking factorization */
    char *mark = xcalloc(nx, 1);
    int **Lcol = xcalloc(nx, sizeof(int *)); int *Lcnt = xcalloc(nx, sizeof(int));
    trip tu = {0}, tl = {0};
    for (int k = 0; k < nx; k++) {
        for (int s2 = A.p[k]; s2 < A.p[k + 1]; s2++) mark[A.i[s2]] = 1;
        for (int j = 0; j < k; j++) {
            if (!mark[j]) continue;
            for (int s2 = 0; s2 < Lcnt[j]; s2++) mark[Lcol[j][s2]] = 1;
        }
        int c = 0;
        for (int i = k + 1; i < nx; i++) if (mark[i]) c++;
        Lcol[k] = xcalloc(c, sizeof(int)); Lcnt[k] = c; c = 0;
        for (int i = 0; i < nx; i++) {
            if (!mark[i]) continue;
            if (i <= k) trip_add(&tu, i, k, 1.0);           /* U(i,k), row i col k */
            else { Lcol[k][c++] = i; trip_add(&tl, i, k, 1.0); }
            mark[i] = 0;
        }
    }
    /* CSR = CSC of the transpose: swap roles */
    trip tlr = {0}, tur = {0};
    for (int k = 0; k < tl.n; k++) trip_add(&tlr, tl.c[k], tl.r[k], 1.0);
    for (int k = 0; k < tu.n; k++) trip_add(&tur, tu.c[k], tu.r[k], 1.0);
    csc Lr = trip_to_csc(&tlr, nx, nx);   /* column index = row of L */
    csc Ur = trip_to_csc(&tur, nx, nx);
    *nnzL = Lr.p[nx]; *nnzU = Ur.p[nx]; *n_elim = nb;
    if (perm_out) {
        for (int q = 0; q < nx; q++) perm_out[q] = perm[q];
        for (int k = 0; k < nb; k++) bus_order_out[k] = bo[k];
        for (int q = 0; q <= nx; q++) { Lp_out[q] = Lr.p[q]; Up_out[q] = Ur.p[q]; }
        for (int k = 0; k < Lr.p[nx]; k++) Lj_out[k] = Lr.i[k];
        for (int k = 0; k < Ur.p[nx]; k++) Uj_out[k] = Ur.i[k];
        /* bus of every permuted variable */
        int *qbus = xcalloc(nx, sizeof(int)), q = 0;
        for (int k = 0; k < nb; k++) { qbus[q++] = k; if (g->ix_v[bo[k]] >= 0) qbus[q++] = k; }
        for (int k = 0; k < nb; k++) level_out[k] = 0;
        for (int r = 0; r < nx; r++) {
            int e = qbus[r];
            for (int s2 = Lr.p[r]; s2 < Lr.p[r + 1]; s2++) {
                int cb = qbus[Lr.i[s2]];
                if (cb != e && level_out[cb] + 1 > level_out[e]) level_out[e] = level_out[cb] + 1;
            }
        }
        free(qbus);
    }
    for (int k = 0; k < nx; k++) free(Lcol[k]);
    free(Lcol); free(Lcnt); free(mark);
    trip_free(&tl); trip_free(&tu); trip_free(&tlr); trip_free(&tur);
    csc_free(&A); csc_free(&Lr); csc_free(&Ur);
    free(perm); free(bo); free(iperm);
    return 0;
}

/* numeric L and U of the oracle's own factorization, as dense matrices (small cases) */
int orc_lu_dense(const orc_grid *g, const double *x, const double *p, int32_t *perm, double *Ld, double *Ud) {
    orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
    orc_lu F; int st = factor_at(g, &s, &F, NULL);
    int n = g->n_x;
    memset(Ld, 0, sizeof(double) * n * n); memset(Ud, 0, sizeof(double) * n * n);
    for (int q = 0; q < n; q++) { perm[q] = F.perm[q]; Ld[(size_t)q * n + q] = 1.0; }
    for (int j = 0; j < n; j++) {
        for (int t = F.L.p[j]; t < F.L.p[j + 1]; t++) Ld[(size_t)j * n + F.L.i[t]] = F.L.x[t];
        for (int t = F.U.p[j]; t < F.U.p[j + 1]; t++) Ud[(size_t)j * n + F.U.i[t]] = F.U.x[t];
    }
    lu_free(&F); state_free(&s);
    return st;
}

/* ------------------------------------------------------------------------ */
/* real-time tracking step, section 6.3 eq. (18)-(19)                       */
/* ------------------------------------------------------------------------ */
/* The paper's Step 2 solves H d = -g with a dense Cholesky factorisation.
 * The oracle writes that factorisation out from its definition, row by row
 * (the Cholesky-Banachiewicz order): for j = 0..n-1
 *     L_jj = sqrt(H_jj - sum_{k<j} L_jk^2)
 *     L_ij = (H_ij - sum_{k<j} L_ik L_jk) / L_jj        for i > j
 * with sums in ascending k.  Only the lower triangle of H is read; L is
 * written whole (zero above the diagonal).  Column-major, leading dimensions
 * ldh, ldl.  Returns 0, or j + 1 for the first pivot H_jj - sum L_jk^2 that is
 * not positive (L is then unspecified from column j on). */
int orc_cholesky(int n, const double *H, int ldh, double *L, int ldl) {
    for (int j = 0; j < n; j++)
        for (int i = 0; i < j; i++) L[i + (size_t)j * ldl] = 0.0;
    for (int j = 0; j < n; j++) {
        double s = H[j + (size_t)j * ldh];
        for (int k = 0; k < j; k++) s -= L[j + (size_t)k * ldl] * L[j + (size_t)k * ldl];
        if (!(s > 0.0)) return j + 1;
        double ljj = sqrt(s);
        L[j + (size_t)j * ldl] = ljj;
        for (int i = j + 1; i < n; i++) {
            double t = H[i + (size_t)j * ldh];
            for (int k = 0; k < j; k++) t -= L[i + (size_t)k * ldl] * L[j + (size_t)k * ldl];
            L[i + (size_t)j * ldl] = t / ljj;
        }
    }
    return 0;
}

/* Solve L L^T X = B in place for nrhs columns of B (leading dimension ldb):
 * forward substitution L y = b (ascending rows), then back substitution
 * L^T x = y (descending rows), each sum in ascending index order. */
void orc_cholesky_solve(int n, const double *L, int ldl, double *B, int nrhs, int ldb) {
    for (int c = 0; c < nrhs; c++) {
        double *b = B + (size_t)c * ldb;
        for (int i = 0; i < n; i++) {
            double s = b[i];
            for (int k = 0; k < i; k++) s -= L[i + (size_t)k * ldl] * b[k];
            b[i] = s / L[i + (size_t)i * ldl];
        }
        for (int i = n - 1; i >= 0; i--) {
            double s = b[i];
            for (int k = i + 1; k < n; k++) s -= L[k + (size_t)i * ldl] * b[k];
            b[i] = s / L[i + (size_t)i * ldl];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* sparse Jacobians and their column colouring (section 4.2.2, Fig. 2)       */
/* ------------------------------------------------------------------------ */
/* J_x and J_p at (x, p) in CSC (rows sorted, explicit zeros kept: the pattern
 * is structural).  Two calls: with NULL arrays only the counts are returned. */
void orc_jacobians_csc(const orc_grid *g, const double *x, const double *p,
                       int32_t *jx_p, int32_t *jx_i, double *jx_x,
                       int32_t *jp_p, int32_t *jp_i, double *jp_x, int64_t *nnz_x, int64_t *nnz_p) {
    orc_state s; state_alloc(g, &s); state_from(g, x, p, &s);
    csc Jx, Jp; jacobians(g, &s, &Jx, &Jp);
    *nnz_x = Jx.p[Jx.nc];
    *nnz_p = Jp.p[Jp.nc];
    if (jx_p) {
        for (int j = 0; j <= Jx.nc; j++) jx_p[j] = Jx.p[j];
        for (int k = 0; k < Jx.p[Jx.nc]; k++) { jx_i[k] = Jx.i[k]; jx_x[k] = Jx.x[k]; }
        for (int j = 0; j <= Jp.nc; j++) jp_p[j] = Jp.p[j];
        for (int k = 0; k < Jp.p[Jp.nc]; k++) { jp_i[k] = Jp.i[k]; jp_x[k] = Jp.x[k]; }
    }
    csc_free(&Jx); csc_free(&Jp); state_free(&s);
}

/* Greedy column colouring of a CSC pattern: columns in ascending order, each
 * takes the smallest colour that no earlier column sharing a row with it has.
 * Columns of one colour then have disjoint row sets, so the product of the
 * matrix with the 0/1 seed matrix of a colour recovers each of those columns
 * exactly (the compression of Fig. 2).  Returns the number of colours. */
static int greedy_colouring(const csc *A, int *colour) {
    /* row -> columns (CSR of the pattern) */
    int nr = A->nr, nc = A->nc, nz = A->p[nc];
    int *rp = xcalloc(nr + 1, sizeof(int)), *rc = xcalloc(nz > 0 ? nz : 1, sizeof(int));
    for (int k = 0; k < nz; k++) rp[A->i[k] + 1]++;
    for (int r = 0; r < nr; r++) rp[r + 1] += rp[r];
    int *fill = xcalloc(nr > 0 ? nr : 1, sizeof(int));
    for (int r = 0; r < nr; r++) fill[r] = rp[r];
    for (int j = 0; j < nc; j++)
        for (int k = A->p[j]; k < A->p[j + 1]; k++) rc[fill[A->i[k]]++] = j;
    int *used = xcalloc(nc + 1, sizeof(int));      /* used[c] == j + 1: colour c is taken for column j */
    int ncol = 0;
    for (int j = 0; j < nc; j++) {
        for (int k = A->p[j]; k < A->p[j + 1]; k++) {
            int r = A->i[k];
            for (int t = rp[r]; t < rp[r + 1]; t++)
                if (rc[t] < j) used[colour[rc[t]]] = j + 1;
        }
        int c = 0;
        while (used[c] == j + 1) c++;
        colour[j] = c;
        if (c + 1 > ncol) ncol = c + 1;
    }
    free(rp); free(rc); free(fill); free(used);
    return ncol;
}

/* Colourings of the J_x columns (x order) and of the J_p columns (p order).
 * The patterns are structural, so the state is irrelevant: a flat start. */
void orc_coloring(const orc_grid *g, int32_t *colors_x, int32_t *colors_p, int32_t *n_colors_x, int32_t *n_colors_p) {
    orc_state s; state_alloc(g, &s);
    for (int i = 0; i < g->n_bus; i++) { s.vm[i] = 1.0; s.va[i] = 0.0; s.pg[i] = 0.0; }
    csc Jx, Jp; jacobians(g, &s, &Jx, &Jp);
    int *cx = xcalloc(g->n_x + 1, sizeof(int)), *cp = xcalloc(g->n_p + 1, sizeof(int));
    *n_colors_x = greedy_colouring(&Jx, cx);
    *n_colors_p = greedy_colouring(&Jp, cp);
    for (int j = 0; j < g->n_x; j++) colors_x[j] = cx[j];
    for (int j = 0; j < g->n_p; j++) colors_p[j] = cp[j];
    free(cx); free(cp);
    csc_free(&Jx); csc_free(&Jp); state_free(&s);
}
