/*
 * eik_oracle.c -- plain, slow, obviously-correct FP64 CPU solvers for the
 * first-order upwind discretisation of |grad u| F = 1 (Chacon & Vladimirsky,
 * "Fast two-scale methods for Eikonal equations", Sec. 3, eq. Eik_discr).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, constant or helper with the
 * CUDA solver.
 *
 * Conventions (readings of points the paper leaves open):
 *   - grid: nx*ny nodes, node (i,j) stored at j*nx + i (x fastest);
 *     every node is an unknown; a neighbour outside the array counts as +inf
 *     (the state constraint "q = +inf on the boundary outside Q", Sec. 3);
 *   - f = h/F per node; F == 0 is an obstacle (f = +inf) whose value stays
 *     +inf unless it is itself a source;
 *   - sources are grid nodes with fixed value q; duplicates keep the min q;
 *   - +inf is IEEE infinity (the paper coded it as a large constant).
 *
 * Built with -O2 -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ENOTCONVERGED (-6)

/* ------------------------------------------------------------------ */
/* Local update, Sec. 3, eqs. one_sided_update and two_sided_update.    */
/* ------------------------------------------------------------------ */

/*
 * Update "from one quadrant" whose x-neighbour value is ux and y-neighbour
 * value is uy (eq. two_sided_update): the root U >= max(ux,uy) of
 *     (U-ux)^2 + (U-uy)^2 = f^2
 * when it exists, i.e. when |ux-uy| < f (at |ux-uy| == f both branches give
 * the same value); otherwise the smaller one-sided update f + min(ux,uy)
 * (eq. one_sided_update).
 */
static double quadrant_update(double ux, double uy, double f)
{
    double lo = ux < uy ? ux : uy;
    if (isinf(f) || isinf(lo))
        return INFINITY; /* nothing finite to build on */
    if (isinf(ux) || isinf(uy))
        return lo + f; /* only one finite neighbour: one-sided */
    double d = ux - uy;
    if (fabs(d) < f) {
        /* the larger root of 2U^2 - 2U(ux+uy) + ux^2 + uy^2 - f^2 = 0 */
        return (ux + uy + sqrt(2.0 * f * f - d * d)) / 2.0;
    }
    return lo + f;
}

/*
 * The full local update at one node: the minimum of the four quadrant
 * updates NE, NW, SW, SE (Sec. 3, text after eq. two_sided_update).  This is
 * written out over all four quadrants on purpose; the GPU solver uses the
 * one-quadrant shortcut of Remark regular_FSM_update instead.
 */
double orc_node_update(double ue, double uw, double un, double us, double f)
{
    double ne = quadrant_update(ue, un, f);
    double nw = quadrant_update(uw, un, f);
    double sw = quadrant_update(uw, us, f);
    double se = quadrant_update(ue, us, f);
    double m = ne;
    if (nw < m) m = nw;
    if (sw < m) m = sw;
    if (se < m) m = se;
    return m;
}

/* ------------------------------------------------------------------ */
/* Problem set-up shared by the three solvers of this file.            */
/* ------------------------------------------------------------------ */

typedef struct {
    int nx, ny;
    double *f;          /* h/F per node, +inf on obstacles */
    unsigned char *src; /* 1 on source nodes (the set Q) */
    double *q;          /* source values (valid where src) */
} problem;

static void problem_free(problem *p)
{
    free(p->f);
    free(p->src);
    free(p->q);
}

static int problem_init(problem *p, int nx, int ny, double h, const double *F,
                        int nsrc, const int32_t *si, const int32_t *sj,
                        const double *sq)
{
    memset(p, 0, sizeof(*p));
    if (nx < 1 || ny < 1 || !(h > 0.0) || !F || nsrc < 0)
        return ORC_EINVAL;
    if (nsrc > 0 && (!si || !sj || !sq))
        return ORC_EINVAL;
    size_t m = (size_t)nx * (size_t)ny;
    p->nx = nx;
    p->ny = ny;
    p->f = (double *)malloc(m * sizeof(double));
    p->src = (unsigned char *)calloc(m, 1);
    p->q = (double *)malloc(m * sizeof(double));
    if (!p->f || !p->src || !p->q) {
        problem_free(p);
        return ORC_ENOMEM;
    }
    for (size_t k = 0; k < m; ++k) {
        double Fk = F[k];
        if (!(Fk >= 0.0) || isinf(Fk)) { /* negative, NaN or +inf speed */
            problem_free(p);
            return ORC_EINVAL;
        }
        p->f[k] = (Fk == 0.0) ? INFINITY : h / Fk;
    }
    for (int s = 0; s < nsrc; ++s) {
        if (si[s] < 0 || si[s] >= nx || sj[s] < 0 || sj[s] >= ny || !isfinite(sq[s])) {
            problem_free(p);
            return ORC_EINVAL;
        }
        size_t k = (size_t)sj[s] * nx + si[s];
        if (!p->src[k] || sq[s] < p->q[k])
            p->q[k] = sq[s];
        p->src[k] = 1;
    }
    return ORC_OK;
}

/* value of the neighbour (i+di, j+dj); +inf outside the grid */
static inline double nb(const double *V, int nx, int ny, int i, int j)
{
    if (i < 0 || j < 0 || i >= nx || j >= ny)
        return INFINITY;
    return V[(size_t)j * nx + i];
}

static inline double T_at(const problem *p, const double *V, int i, int j)
{
    int nx = p->nx, ny = p->ny;
    return orc_node_update(nb(V, nx, ny, i + 1, j), nb(V, nx, ny, i - 1, j),
                           nb(V, nx, ny, i, j + 1), nb(V, nx, ny, i, j - 1),
                           p->f[(size_t)j * nx + i]);
}

static void init_values(const problem *p, double *V)
{
    size_t m = (size_t)p->nx * p->ny;
    for (size_t k = 0; k < m; ++k)
        V[k] = p->src[k] ? p->q[k] : INFINITY;
}

/* ------------------------------------------------------------------ */
/* Fast Marching, Sec. 3.1, Alg. FMM, with a binary heap.              */
/* ------------------------------------------------------------------ */

enum { FAR = 0, CONSIDERED = 1, ACCEPTED = 2 };

typedef struct {
    int32_t *node; /* heap array of node ids */
    int32_t *pos;  /* pos[node] = index in heap, -1 if absent */
    int32_t size;
    const double *V;
    int by_index;  /* equal values: smaller node id first (else any order) */
} heap;

static inline int heap_less(const heap *H, int a, int b)
{
    const double va = H->V[H->node[a]], vb = H->V[H->node[b]];
    if (H->by_index && va == vb)
        return H->node[a] < H->node[b];
    return va < vb;
}

static inline void heap_swap(heap *H, int a, int b)
{
    int32_t na = H->node[a], nb_ = H->node[b];
    H->node[a] = nb_;
    H->node[b] = na;
    H->pos[nb_] = a;
    H->pos[na] = b;
}

static void heap_up(heap *H, int k)
{
    while (k > 0) {
        int parent = (k - 1) / 2;
        if (!heap_less(H, k, parent))
            break;
        heap_swap(H, k, parent);
        k = parent;
    }
}

static void heap_down(heap *H, int k)
{
    for (;;) {
        int l = 2 * k + 1, r = l + 1, s = k;
        if (l < H->size && heap_less(H, l, s)) s = l;
        if (r < H->size && heap_less(H, r, s)) s = r;
        if (s == k)
            break;
        heap_swap(H, k, s);
        k = s;
    }
}

static void heap_push(heap *H, int32_t n)
{
    H->node[H->size] = n;
    H->pos[n] = H->size;
    H->size++;
    heap_up(H, H->size - 1);
}

static int32_t heap_pop(heap *H)
{
    int32_t top = H->node[0];
    H->size--;
    if (H->size > 0) {
        H->node[0] = H->node[H->size];
        H->pos[H->node[0]] = 0;
        heap_down(H, 0);
    }
    H->pos[top] = -1;
    return top;
}

/*
 * Recompute a non-Accepted, non-source node from its current neighbours and
 * keep the smaller value (Alg. FMM, "compute a temporary value ... if smaller,
 * replace").  Far nodes become Considered.
 */
static void fmm_touch(const problem *p, double *V, unsigned char *label, heap *H,
                      int i, int j)
{
    if (i < 0 || j < 0 || i >= p->nx || j >= p->ny)
        return;
    size_t k = (size_t)j * p->nx + i;
    if (label[k] == ACCEPTED || p->src[k])
        return;
    double t = T_at(p, V, i, j);
    if (t < V[k]) {
        V[k] = t;
        if (label[k] == CONSIDERED)
            heap_up(H, H->pos[k]); /* decrease-key */
    }
    if (label[k] == FAR && !isinf(V[k])) {
        label[k] = CONSIDERED;
        heap_push(H, (int32_t)k);
    }
}

/* Source order of the acceptance record: smaller q first, then node id. */
static const problem *g_src_problem;
static int src_cmp(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    const double qx = g_src_problem->q[x], qy = g_src_problem->q[y];
    if (qx != qy)
        return qx < qy ? -1 : 1;
    return x < y ? -1 : x > y;
}

/*
 * Alg. FMM on problem p.  order (may be null): the nodes in the order they
 * become Accepted -- the exit set first (it is Accepted in the
 * initialisation; listed by q, then id), then each node as the main loop
 * removes it from the heap.  by_index: equal values leave the heap in node
 * order.  Returns the number of Accepted nodes, or a negative error code.
 */
static int64_t fmm_run(const problem *p, double *U, int32_t *order, int by_index)
{
    const int nx = p->nx, ny = p->ny;
    size_t m = (size_t)nx * ny;
    unsigned char *label = (unsigned char *)calloc(m, 1);
    heap H;
    H.node = (int32_t *)malloc(m * sizeof(int32_t));
    H.pos = (int32_t *)malloc(m * sizeof(int32_t));
    H.size = 0;
    H.V = U;
    H.by_index = by_index;
    if (!label || !H.node || !H.pos) {
        free(label); free(H.node); free(H.pos);
        return ORC_ENOMEM;
    }
    for (size_t k = 0; k < m; ++k)
        H.pos[k] = -1;
    /* Initialisation: Q is Accepted with V = q, everything else Far, +inf. */
    init_values(p, U);
    int64_t acc = 0;
    for (size_t k = 0; k < m; ++k)
        if (p->src[k]) {
            label[k] = ACCEPTED;
            if (order)
                order[acc] = (int32_t)k;
            ++acc;
        }
    if (order && acc > 1) {
        g_src_problem = p;
        qsort(order, (size_t)acc, sizeof(int32_t), src_cmp);
    }
    /* Far neighbours of Accepted nodes become Considered. */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            if (p->src[(size_t)j * nx + i]) {
                fmm_touch(p, U, label, &H, i + 1, j);
                fmm_touch(p, U, label, &H, i - 1, j);
                fmm_touch(p, U, label, &H, i, j + 1);
                fmm_touch(p, U, label, &H, i, j - 1);
            }
    /* Main loop: accept the smallest Considered node, update its neighbours. */
    while (H.size > 0) {
        int32_t k = heap_pop(&H);
        label[k] = ACCEPTED;
        if (order)
            order[acc] = k;
        ++acc;
        int i = k % nx, j = k / nx;
        fmm_touch(p, U, label, &H, i + 1, j);
        fmm_touch(p, U, label, &H, i - 1, j);
        fmm_touch(p, U, label, &H, i, j + 1);
        fmm_touch(p, U, label, &H, i, j - 1);
    }
    free(label);
    free(H.node);
    free(H.pos);
    return acc;
}

int orc_fmm(int nx, int ny, double h, const double *F, int nsrc, const int32_t *si,
            const int32_t *sj, const double *sq, double *U, int64_t *n_accepted)
{
    problem p;
    int rc = problem_init(&p, nx, ny, h, F, nsrc, si, sj, sq);
    if (rc)
        return rc;
    int64_t acc = fmm_run(&p, U, NULL, 0);
    int64_t nq = 0; /* the exit set, Accepted before the main loop */
    for (size_t k = 0; k < (size_t)nx * ny; ++k)
        nq += p.src[k];
    problem_free(&p);
    if (acc < 0)
        return (int)acc;
    if (n_accepted)
        *n_accepted = acc - nq; /* removals from the heap */
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Fast Sweeping, Sec. 3.2, Algs. FSM_order and FSM.                   */
/* ------------------------------------------------------------------ */

int orc_fsm(int nx, int ny, double h, const double *F, int nsrc, const int32_t *si,
            const int32_t *sj, const double *sq, double *U, int32_t max_sweeps,
            int32_t *n_sweeps)
{
    problem p;
    int rc = problem_init(&p, nx, ny, h, F, nsrc, si, sj, sq);
    if (rc)
        return rc;
    init_values(&p, U);
    int32_t sweep = 0;
    int changed;
    do {
        changed = 0;
        /* Alg. FSM_order: direction = sweepNumber mod 4 chooses iOrder, jOrder */
        int dir = sweep % 4;
        int i_up = (dir == 0 || dir == 1);
        int j_up = (dir == 0 || dir == 3);
        for (int ii = 0; ii < nx; ++ii) {
            int i = i_up ? ii : nx - 1 - ii;
            for (int jj = 0; jj < ny; ++jj) {
                int j = j_up ? jj : ny - 1 - jj;
                size_t k = (size_t)j * nx + i;
                if (p.src[k])
                    continue;
                double t = T_at(&p, U, i, j);
                if (t < U[k]) {
                    U[k] = t;
                    changed = 1;
                }
            }
        }
        ++sweep;
    } while (changed && sweep < max_sweeps);
    if (n_sweeps)
        *n_sweeps = sweep;
    problem_free(&p);
    return changed ? ORC_ENOTCONVERGED : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Locking Sweeping, Sec. 3.2, Remark locking_FSM: Alg. FSM with a     */
/* locking flag per node.                                              */
/* ------------------------------------------------------------------ */

/*
 * One sweep in direction dir (Alg. FSM_order's numbering) over the nodes of
 * the box [i0,i1) x [j0,j1) that are unlocked (unl[k] != 0).  Every node the
 * sweep processes is locked; if its value decreases, each neighbour inside
 * the box whose value is larger (the only ones whose update can use it) is
 * unlocked.  Sources are never unlocked.  Returns 1 if a value changed; adds
 * the local updates computed to *evals and keeps *n_unl, the number of
 * unlocked nodes, current.
 */
static int sweep_locked(const problem *p, double *V, unsigned char *unl, int i0, int i1, int j0, int j1,
                        int dir, int64_t *evals, int64_t *n_unl)
{
    const int i_up = dir <= 1, j_up = dir == 0 || dir == 3;
    int changed = 0;
    for (int ii = i0; ii < i1; ++ii) {
        int i = i_up ? ii : i1 - 1 - (ii - i0);
        for (int jj = j0; jj < j1; ++jj) {
            int j = j_up ? jj : j1 - 1 - (jj - j0);
            size_t k = (size_t)j * p->nx + i;
            if (!unl[k]) continue;
            unl[k] = 0;
            --*n_unl;
            double t = T_at(p, V, i, j);
            ++*evals;
            if (!(t < V[k])) continue;
            V[k] = t;
            changed = 1;
            const int ni[4] = {i - 1, i + 1, i, i}, nj[4] = {j, j, j - 1, j + 1};
            for (int e = 0; e < 4; ++e) {
                if (ni[e] < i0 || ni[e] >= i1 || nj[e] < j0 || nj[e] >= j1) continue;
                size_t kn = (size_t)nj[e] * p->nx + ni[e];
                if (V[kn] > V[k] && !unl[kn] && !p->src[kn]) {
                    unl[kn] = 1;
                    ++*n_unl;
                }
            }
        }
    }
    return changed;
}

/*
 * LSM on the whole grid: every node starts locked except the non-source
 * neighbours of sources; sweeps in the directions of Alg. FSM_order run
 * while some node is unlocked.  The count of unlocked nodes stands in for
 * the final sweep that would find them all locked, so *n_sweeps is one less
 * than Alg. FSM's count or equal to it.  *n_evals: local updates computed.
 */
int orc_lsm(int nx, int ny, double h, const double *F, int nsrc, const int32_t *si,
            const int32_t *sj, const double *sq, double *U, int32_t max_sweeps,
            int32_t *n_sweeps, int64_t *n_evals)
{
    problem p;
    int rc = problem_init(&p, nx, ny, h, F, nsrc, si, sj, sq);
    if (rc)
        return rc;
    unsigned char *unl = (unsigned char *)calloc((size_t)nx * ny, 1);
    if (!unl) {
        problem_free(&p);
        return ORC_ENOMEM;
    }
    init_values(&p, U);
    int64_t n_unl = 0, evals = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            if (!p.src[(size_t)j * nx + i]) continue;
            const int ni[4] = {i - 1, i + 1, i, i}, nj[4] = {j, j, j - 1, j + 1};
            for (int e = 0; e < 4; ++e) {
                if (ni[e] < 0 || ni[e] >= nx || nj[e] < 0 || nj[e] >= ny) continue;
                size_t kn = (size_t)nj[e] * nx + ni[e];
                if (!p.src[kn] && !unl[kn]) {
                    unl[kn] = 1;
                    ++n_unl;
                }
            }
        }
    int32_t sweep = 0;
    while (n_unl > 0 && sweep < max_sweeps) {
        sweep_locked(&p, U, unl, 0, nx, 0, ny, sweep % 4, &evals, &n_unl);
        ++sweep;
    }
    if (n_sweeps)
        *n_sweeps = sweep;
    if (n_evals)
        *n_evals = evals;
    free(unl);
    problem_free(&p);
    return n_unl ? ORC_ENOTCONVERGED : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Jacobi "value iteration" from +inf (Sec. 2, eq. generic_value_it,   */
/* applied to the system of eq. Eik_discr): every node is updated from */
/* the previous iterate simultaneously, until nothing changes.         */
/* ------------------------------------------------------------------ */

int orc_jacobi(int nx, int ny, double h, const double *F, int nsrc, const int32_t *si,
               const int32_t *sj, const double *sq, double *U, int32_t max_iters,
               int32_t *n_iters)
{
    problem p;
    int rc = problem_init(&p, nx, ny, h, F, nsrc, si, sj, sq);
    if (rc)
        return rc;
    size_t m = (size_t)nx * ny;
    double *W = (double *)malloc(m * sizeof(double));
    if (!W) {
        problem_free(&p);
        return ORC_ENOMEM;
    }
    init_values(&p, U);
    int32_t it = 0;
    int changed;
    do {
        changed = 0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                size_t k = (size_t)j * nx + i;
                double t = p.src[k] ? U[k] : T_at(&p, U, i, j);
                W[k] = t < U[k] ? t : U[k];
                if (W[k] != U[k])
                    changed = 1;
            }
        memcpy(U, W, m * sizeof(double));
        ++it;
    } while (changed && it < max_iters);
    if (n_iters)
        *n_iters = it;
    free(W);
    problem_free(&p);
    return changed ? ORC_ENOTCONVERGED : ORC_OK;
}

/* ------------------------------------------------------------------ */
/* The operator T of eq. Eik_discr applied once to a given V: TV = V on  */
/* sources, the local update elsewhere.  Used to measure residuals.    */
/* ------------------------------------------------------------------ */

int orc_apply_T(int nx, int ny, double h, const double *F, int nsrc, const int32_t *si,
                const int32_t *sj, const double *sq, const double *V, double *TV)
{
    problem p;
    int rc = problem_init(&p, nx, ny, h, F, nsrc, si, sj, sq);
    if (rc)
        return rc;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t k = (size_t)j * nx + i;
            TV[k] = p.src[k] ? p.q[k] : T_at(&p, V, i, j);
        }
    problem_free(&p);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Heap-Cell Methods, Sec. 4.2 (HCM) and Sec. 4.3 (FHCM), serially:    */
/* Alg. generic_LC_cells over k x k cells kept in a binary heap by     */
/* cell value, with four directional flags per cell.                   */
/*   HCM:  a removed cell is swept until a sweep changes nothing; its  */
/*         flagged directions come first, then the other two of the    */
/*         first four, then the cycle of Alg. FSM_order (Remark        */
/*         HCM_preferred_sweeps and the list before it).  An           */
/*         activation across a side raises both flags that point away  */
/*         from that side.                                             */
/*   FHCM: a removed cell is swept once in each flagged direction and  */
/*         no more (Alg. FHCM); an activation raises one of the two    */
/*         flags when the boundary values on that side are monotone    */
/*         (the Monotonicity Check), both otherwise.                   */
/*   HCM with locking (Sec. 4.2, the Locking Sweeping version inside   */
/*         cells): the sweeps of HCM, each processing only the cell's  */
/*         unlocked nodes (Remark locking_FSM, as in orc_lsm), until   */
/*         none is left.  At a removal the nodes next to another cell  */
/*         start unlocked (their boundary data may have changed since  */
/*         the cell's last removal; the rest of the cell was left at    */
/*         its fixed point), and on the first removal also the nodes    */
/*         next to a source of the cell.  The values, and hence the     */
/*         removals, are those of HCM bit for bit.                      */
/* The activation test and the cell values follow Alg. generic_LC_cells */
/* and eq. cell_value: a node x_i on the border that changed during the */
/* removal (or a source, on the cell's first removal) with V_i < V_j    */
/* across the border, x_j not a source, adds the neighbour cell; the    */
/* neighbour's cell value becomes min(itself, max finite V on the       */
/* border + (k+1)/2 * h / F(y)), F read at the node across the border   */
/* from the largest value (the smallest h/F of the grid where that node */
/* is an obstacle).  Sweep directions are numbered as in Alg. FSM_order: */
/* 0 (i up, j up), 1 (i up, j down), 2 (i down, j down), 3 (i down, j up). */
/* ------------------------------------------------------------------ */

typedef struct {
    int32_t *cell;
    int32_t *pos;
    int32_t size;
    const double *key;
} cell_heap;

static int ch_less(const cell_heap *H, int a, int b) { return H->key[H->cell[a]] < H->key[H->cell[b]]; }
static void ch_swap(cell_heap *H, int a, int b)
{
    int32_t ca = H->cell[a], cb = H->cell[b];
    H->cell[a] = cb;
    H->cell[b] = ca;
    H->pos[cb] = a;
    H->pos[ca] = b;
}
static void ch_up(cell_heap *H, int k)
{
    while (k > 0) {
        int parent = (k - 1) / 2;
        if (!ch_less(H, k, parent)) break;
        ch_swap(H, k, parent);
        k = parent;
    }
}
static void ch_down(cell_heap *H, int k)
{
    for (;;) {
        int l = 2 * k + 1, r = l + 1, s = k;
        if (l < H->size && ch_less(H, l, s)) s = l;
        if (r < H->size && ch_less(H, r, s)) s = r;
        if (s == k) break;
        ch_swap(H, k, s);
        k = s;
    }
}

/* one Gauss-Seidel sweep of the cell's nodes in direction dir; 1 if a value changed */
static int sweep_cell(const problem *p, double *V, int i0, int i1, int j0, int j1, int dir)
{
    int i_up = (dir == 0 || dir == 1), j_up = (dir == 0 || dir == 3);
    int changed = 0;
    for (int ii = i0; ii < i1; ++ii) {
        int i = i_up ? ii : i1 - 1 - (ii - i0);
        for (int jj = j0; jj < j1; ++jj) {
            int j = j_up ? jj : j1 - 1 - (jj - j0);
            size_t k = (size_t)j * p->nx + i;
            if (p->src[k]) continue;
            double t = T_at(p, V, i, j);
            if (t < V[k]) {
                V[k] = t;
                changed = 1;
            }
        }
    }
    return changed;
}

/* stats: [0] cell removals, [1] sweeps, [2] monotone checks passed, [3] checks,
 * [4] local updates computed (every non-source node of a cell per sweep, or
 * the unlocked ones with locking) */
int orc_cells(int nx, int ny, double h, const double *F, int nsrc, const int32_t *si, const int32_t *sj,
              const double *sq, int k, int method, double *U, int64_t *stats)
{
    /* method: 0 HCM, 1 FHCM, 2 HCM with locking */
    if (k < 1 || method < 0 || method > 2) return ORC_EINVAL;
    const int fast = method == 1, lsm = method == 2;
    problem p;
    int rc = problem_init(&p, nx, ny, h, F, nsrc, si, sj, sq);
    if (rc) return rc;
    init_values(&p, U);
    const int cxn = (nx + k - 1) / k, cyn = (ny + k - 1) / k, J = cxn * cyn;
    double *cval = (double *)malloc((size_t)J * sizeof(double));
    unsigned char *flags = (unsigned char *)calloc((size_t)J, 1);
    unsigned char *removed = (unsigned char *)calloc((size_t)J, 1);
    int32_t *hcell = (int32_t *)malloc((size_t)J * sizeof(int32_t));
    int32_t *hpos = (int32_t *)malloc((size_t)J * sizeof(int32_t));
    double *old = (double *)malloc((size_t)k * k * sizeof(double));
    unsigned char *unl = lsm ? (unsigned char *)calloc((size_t)nx * ny, 1) : NULL;
    if (!cval || !flags || !removed || !hcell || !hpos || !old || (lsm && !unl)) {
        free(cval); free(flags); free(removed); free(hcell); free(hpos); free(old); free(unl);
        problem_free(&p);
        return ORC_ENOMEM;
    }
    double fmin = INFINITY;
    for (size_t e = 0; e < (size_t)nx * ny; ++e)
        if (p.f[e] < fmin) fmin = p.f[e];
    cell_heap H = {hcell, hpos, 0, cval};
    for (int c = 0; c < J; ++c) {
        cval[c] = INFINITY;
        hpos[c] = -1;
    }
    /* source cells: queued with all four flags, cell value max q over the cell */
    for (size_t e = 0; e < (size_t)nx * ny; ++e) {
        if (!p.src[e]) continue;
        int i = (int)(e % nx), j = (int)(e / nx);
        int c = (j / k) * cxn + i / k;
        if (hpos[c] < 0) {
            cval[c] = p.q[e];
            hcell[H.size] = c;
            hpos[c] = H.size++;
        } else if (p.q[e] > cval[c]) {
            cval[c] = p.q[e];
        }
        flags[c] = 15;
    }
    for (int e = H.size / 2; e >= 0; --e) ch_down(&H, e);
    int64_t removals = 0, sweeps = 0, mono_ok = 0, mono_n = 0, evals = 0;
    while (H.size > 0) {
        int c = hcell[0];
        H.size--;
        if (H.size > 0) {
            hcell[0] = hcell[H.size];
            hpos[hcell[0]] = 0;
            ch_down(&H, 0);
        }
        hpos[c] = -1;
        ++removals;
        const int first = !removed[c];
        removed[c] = 1;
        const int cx = c % cxn, cy = c / cxn;
        const int i0 = cx * k, i1 = i0 + k < nx ? i0 + k : nx, j0 = cy * k, j1 = j0 + k < ny ? j0 + k : ny;
        const int w = i1 - i0;
        for (int j = j0; j < j1; ++j)
            for (int i = i0; i < i1; ++i) old[(j - j0) * w + (i - i0)] = U[(size_t)j * nx + i];
        /* the sweeps */
        int64_t free_nodes = 0;
        for (int j = j0; j < j1; ++j)
            for (int i = i0; i < i1; ++i) free_nodes += !p.src[(size_t)j * nx + i];
        const int fl = flags[c];
        flags[c] = 0;
        if (fast) {
            for (int d = 0; d < 4; ++d)
                if (fl >> d & 1) {
                    sweep_cell(&p, U, i0, i1, j0, j1, d);
                    ++sweeps;
                    evals += free_nodes;
                }
        } else if (lsm) {
            int order[4], no = 0;
            for (int d = 0; d < 4; ++d) if (fl >> d & 1) order[no++] = d;
            for (int d = 0; d < 4; ++d) if (!(fl >> d & 1)) order[no++] = d;
            int64_t n_unl = 0;
            for (int j = j0; j < j1; ++j)
                for (int i = i0; i < i1; ++i) {
                    const size_t q = (size_t)j * nx + i;
                    if (p.src[q]) continue;
                    int u = (i == i0 && i > 0) || (i == i1 - 1 && i1 < nx) || (j == j0 && j > 0) ||
                            (j == j1 - 1 && j1 < ny);
                    if (!u && first)
                        u = (i > i0 && p.src[q - 1]) || (i + 1 < i1 && p.src[q + 1]) ||
                            (j > j0 && p.src[q - nx]) || (j + 1 < j1 && p.src[q + nx]);
                    if (u) {
                        unl[q] = 1;
                        ++n_unl;
                    }
                }
            int s = 0;
            while (n_unl > 0) {
                int d = s < 4 ? order[s] : s % 4;
                sweep_locked(&p, U, unl, i0, i1, j0, j1, d, &evals, &n_unl);
                ++s;
            }
            sweeps += s;
        } else {
            int order[4], no = 0;
            for (int d = 0; d < 4; ++d) if (fl >> d & 1) order[no++] = d;
            for (int d = 0; d < 4; ++d) if (!(fl >> d & 1)) order[no++] = d;
            int s = 0, changed;
            do {
                int d = s < 4 ? order[s] : s % 4;
                changed = sweep_cell(&p, U, i0, i1, j0, j1, d);
                ++s;
            } while (changed);
            sweeps += s;
            evals += s * free_nodes;
        }
        /* the four borders: W, E, S, N */
        for (int sd = 0; sd < 4; ++sd) {
            int ncx = cx + (sd == 0 ? -1 : sd == 1 ? 1 : 0), ncy = cy + (sd == 2 ? -1 : sd == 3 ? 1 : 0);
            if (ncx < 0 || ncy < 0 || ncx >= cxn || ncy >= cyn) continue;
            const int nc = ncy * cxn + ncx;
            const int len = sd < 2 ? j1 - j0 : i1 - i0;
            int act = 0, bmax = -1;
            double vmax = 0.0;
            int nondec = 1, noninc = 1;
            double prev = 0.0;
            for (int b = 0; b < len; ++b) {
                int bi, bj, ai, aj;
                if (sd == 0) { bi = i0; bj = j0 + b; ai = bi - 1; aj = bj; }
                else if (sd == 1) { bi = i1 - 1; bj = j0 + b; ai = i1; aj = bj; }
                else if (sd == 2) { bi = i0 + b; bj = j0; ai = bi; aj = j0 - 1; }
                else { bi = i0 + b; bj = j1 - 1; ai = bi; aj = j1; }
                const size_t qb = (size_t)bj * nx + bi, qa = (size_t)aj * nx + ai;
                const double vb = U[qb];
                const int ch = vb < old[(bj - j0) * w + (bi - i0)];
                if ((ch || (first && p.src[qb])) && vb < U[qa] && !p.src[qa]) act = 1;
                if (isfinite(vb) && (bmax < 0 || vb >= vmax)) { vmax = vb; bmax = b; }
                if (b > 0) {
                    if (vb < prev) nondec = 0;
                    if (vb > prev) noninc = 0;
                }
                prev = vb;
            }
            if (bmax >= 0) {
                int ai, aj;
                if (sd == 0) { ai = i0 - 1; aj = j0 + bmax; }
                else if (sd == 1) { ai = i1; aj = j0 + bmax; }
                else if (sd == 2) { ai = i0 + bmax; aj = j0 - 1; }
                else { ai = i0 + bmax; aj = j1; }
                double fy = p.f[(size_t)aj * nx + ai];
                if (!isfinite(fy)) fy = fmin;
                const double v = vmax + 0.5 * (k + 1) * fy;
                if (v < cval[nc]) {
                    cval[nc] = v;
                    if (hpos[nc] >= 0) ch_up(&H, hpos[nc]);
                }
            }
            if (!act) continue;
            /* the flags pointing away from side sd, and along the border
             * the direction from its smaller values (the Monotonicity Check) */
            int up, down;  /* flag for increasing / decreasing along-border coordinate */
            if (sd == 0) { up = 3; down = 2; }       /* neighbour west: i down */
            else if (sd == 1) { up = 0; down = 1; }  /* neighbour east: i up */
            else if (sd == 2) { up = 1; down = 2; }  /* neighbour south: j down */
            else { up = 0; down = 3; }               /* neighbour north: j up */
            int set;
            if (!fast) {
                set = (1 << up) | (1 << down);
            } else {
                ++mono_n;
                if (noninc) { set = 1 << down; ++mono_ok; }
                else if (nondec) { set = 1 << up; ++mono_ok; }
                else set = (1 << up) | (1 << down);
            }
            flags[nc] |= (unsigned char)set;
            if (hpos[nc] < 0) {
                hcell[H.size] = nc;
                hpos[nc] = H.size++;
                ch_up(&H, hpos[nc]);
            }
        }
    }
    if (stats) {
        stats[0] = removals;
        stats[1] = sweeps;
        stats[2] = mono_ok;
        stats[3] = mono_n;
        stats[4] = evals;
    }
    free(cval); free(flags); free(removed); free(hcell); free(hpos); free(old); free(unl);
    problem_free(&p);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Fast Marching-Sweeping Method, Sec. 4.1 (Alg. FMSM, Remark          */
/* sweeping_in_FMSM, Fig. coarse_sweep_choice), serially.              */
/*   Part I: Alg. FMM on the coarse grid X^c of cell centres: spacing  */
/*   k h, speed F at the centre (the mean of the one, two or four nodes */
/*   nearest to it, clamped to the grid), and as its exit set           */
/*   Q^c the cells that hold sources, each with the smallest q among    */
/*   them.  The acceptance order is the permutation P: Q^c first (by q, */
/*   then index), then the heap's removals, equal values by index; the  */
/*   cells Fast Marching never accepts (infinite coarse value) follow   */
/*   by index.                                                           */
/*   Part II: every cell once, in the order P, on its domain c with the */
/*   current values of N^f(c) as boundary data.  A cell of Q^c is swept */
/*   by Alg. FSM unchanged: the directions of Alg. FSM_order in turn,    */
/*   the full local update, until a sweep changes nothing.  Any other    */
/*   cell gets at most four sweeps, each with the sweep-directional      */
/*   update (the quadrant of the two neighbours behind the sweep): the   */
/*   directions both of whose sides border cells accepted before it, or */
/*   -- when no direction has both -- every direction with one such      */
/*   side, taken in Alg. FSM_order's order.  Directions are numbered as  */
/*   in Alg. FSM_order: 0 (i up, j up: from the SW corner, behind it W   */
/*   and S), 1 (i up, j down: NW; W, N), 2 (i down, j down: NE; E, N),   */
/*   3 (i down, j up: SE; E, S).                                          */
/* ------------------------------------------------------------------ */

/* one sweep of the cell's nodes in direction dir with the sweep-directional update */
static int sweep_cell_directional(const problem *p, double *V, int i0, int i1, int j0, int j1, int dir)
{
    const int i_up = (dir == 0 || dir == 1), j_up = (dir == 0 || dir == 3);
    const int nx = p->nx, ny = p->ny;
    int changed = 0;
    for (int ii = i0; ii < i1; ++ii) {
        int i = i_up ? ii : i1 - 1 - (ii - i0);
        for (int jj = j0; jj < j1; ++jj) {
            int j = j_up ? jj : j1 - 1 - (jj - j0);
            size_t k = (size_t)j * nx + i;
            if (p->src[k]) continue;
            double ux = nb(V, nx, ny, i_up ? i - 1 : i + 1, j);
            double uy = nb(V, nx, ny, i, j_up ? j - 1 : j + 1);
            double t = quadrant_update(ux, uy, p->f[k]);
            if (t < V[k]) {
                V[k] = t;
                changed = 1;
            }
        }
    }
    return changed;
}

/*
 * Uc (may be null): the coarse values, cyn x cxn.  order (may be null): the
 * cells in processing order.  dirs_out (may be null): per cell, the sweep
 * directions taken (bit d: direction d), or 16 for a cell swept by Alg. FSM.
 * stats: [0] cells processed, [1] sweeps, [2] coarse nodes Accepted by Fast
 * Marching (the exit set included).
 */
int orc_fmsm(int nx, int ny, double h, const double *F, int nsrc, const int32_t *si, const int32_t *sj,
             const double *sq, int k, double *U, double *Uc, int32_t *order, int32_t *dirs_out,
             int64_t *stats)
{
    if (k < 1) return ORC_EINVAL;
    problem p;
    int rc = problem_init(&p, nx, ny, h, F, nsrc, si, sj, sq);
    if (rc) return rc;
    const int cxn = (nx + k - 1) / k, cyn = (ny + k - 1) / k, J = cxn * cyn;
    double *Fc = (double *)malloc((size_t)J * sizeof(double));
    double *Vc = (double *)malloc((size_t)J * sizeof(double));
    int32_t *ord = (int32_t *)malloc((size_t)J * sizeof(int32_t));
    int32_t *rank = (int32_t *)malloc((size_t)J * sizeof(int32_t));
    int32_t *csi = (int32_t *)malloc((size_t)(nsrc > 0 ? nsrc : 1) * sizeof(int32_t));
    int32_t *csj = (int32_t *)malloc((size_t)(nsrc > 0 ? nsrc : 1) * sizeof(int32_t));
    double *csq = (double *)malloc((size_t)(nsrc > 0 ? nsrc : 1) * sizeof(double));
    problem pc;
    memset(&pc, 0, sizeof(pc));
    if (!Fc || !Vc || !ord || !rank || !csi || !csj || !csq) {
        rc = ORC_ENOMEM;
        goto done;
    }
    /* ---- Part I: the coarse grid and its Fast Marching */
    for (int cy = 0; cy < cyn; ++cy)
        for (int cx = 0; cx < cxn; ++cx) {
            /* F at the centre, as the mean of the nodes nearest to it (one,
             * two or four of them; exact for a bilinear F) */
            int i0 = cx * k + (k - 1) / 2, i1 = cx * k + k / 2;
            int j0 = cy * k + (k - 1) / 2, j1 = cy * k + k / 2;
            if (i0 > nx - 1) i0 = nx - 1;
            if (i1 > nx - 1) i1 = nx - 1;
            if (j0 > ny - 1) j0 = ny - 1;
            if (j1 > ny - 1) j1 = ny - 1;
            const double a = F[(size_t)j0 * nx + i0], b = F[(size_t)j0 * nx + i1];
            const double c = F[(size_t)j1 * nx + i0], d = F[(size_t)j1 * nx + i1];
            Fc[cy * cxn + cx] = 0.25 * (((a + b) + c) + d);
        }
    for (int s = 0; s < nsrc; ++s) { /* problem_init keeps the smallest q per coarse node */
        csi[s] = si[s] / k;
        csj[s] = sj[s] / k;
        csq[s] = sq[s];
    }
    rc = problem_init(&pc, cxn, cyn, (double)k * h, Fc, nsrc, csi, csj, csq);
    if (rc) { /* problem_init has freed its arrays already */
        memset(&pc, 0, sizeof(pc));
        goto done;
    }
    {
        int64_t acc = fmm_run(&pc, Vc, ord, 1);
        if (acc < 0) {
            rc = (int)acc;
            goto done;
        }
        for (int c = 0; c < J; ++c) rank[c] = -1;
        for (int64_t e = 0; e < acc; ++e) rank[ord[e]] = (int32_t)e;
        int64_t e = acc;
        for (int c = 0; c < J; ++c)
            if (rank[c] < 0) {
                ord[e] = c;
                rank[c] = (int32_t)e++;
            }
        if (stats) stats[2] = acc;
    }
    /* ---- Part II: the cells in order */
    init_values(&p, U);
    int64_t sweeps = 0;
    for (int e = 0; e < J; ++e) {
        const int c = ord[e];
        const int cx = c % cxn, cy = c / cxn;
        const int i0 = cx * k, i1 = i0 + k < nx ? i0 + k : nx, j0 = cy * k, j1 = j0 + k < ny ? j0 + k : ny;
        if (pc.src[c]) {
            /* Alg. FSM on the cell: sweep until a sweep changes nothing */
            for (int s = 0;; ++s) {
                ++sweeps;
                if (!sweep_cell(&p, U, i0, i1, j0, j1, s % 4)) break;
            }
            if (dirs_out) dirs_out[c] = 16;
            continue;
        }
        /* sides W, E, S, N bordering a cell accepted before this one */
        const int w = cx > 0 && rank[c - 1] < e, ea = cx + 1 < cxn && rank[c + 1] < e;
        const int so = cy > 0 && rank[c - cxn] < e, no = cy + 1 < cyn && rank[c + cxn] < e;
        const int xs[4] = {w, w, ea, ea}, ys[4] = {so, no, no, so};
        int dirs = 0;
        for (int d = 0; d < 4; ++d)
            if (xs[d] && ys[d]) dirs |= 1 << d;
        if (!dirs)
            for (int d = 0; d < 4; ++d)
                if (xs[d] || ys[d]) dirs |= 1 << d;
        for (int d = 0; d < 4; ++d)
            if (dirs >> d & 1) {
                sweep_cell_directional(&p, U, i0, i1, j0, j1, d);
                ++sweeps;
            }
        if (dirs_out) dirs_out[c] = dirs;
    }
    if (stats) {
        stats[0] = J;
        stats[1] = sweeps;
    }
    if (Uc) memcpy(Uc, Vc, (size_t)J * sizeof(double));
    if (order) memcpy(order, ord, (size_t)J * sizeof(int32_t));
done:
    free(Fc); free(Vc); free(ord); free(rank); free(csi); free(csj); free(csq);
    problem_free(&pc);
    problem_free(&p);
    return rc;
}
