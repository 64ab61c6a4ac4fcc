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
} heap;

static inline int heap_less(const heap *H, int a, int b)
{
    return H->V[H->node[a]] < H->V[H->node[b]];
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

int orc_fmm(int nx, int ny, double h, const double *F, int nsrc, const int32_t *si,
            const int32_t *sj, const double *sq, double *U, int64_t *n_accepted)
{
    problem p;
    int rc = problem_init(&p, nx, ny, h, F, nsrc, si, sj, sq);
    if (rc)
        return rc;
    size_t m = (size_t)nx * ny;
    unsigned char *label = (unsigned char *)calloc(m, 1);
    heap H;
    H.node = (int32_t *)malloc(m * sizeof(int32_t));
    H.pos = (int32_t *)malloc(m * sizeof(int32_t));
    H.size = 0;
    H.V = U;
    if (!label || !H.node || !H.pos) {
        free(label); free(H.node); free(H.pos); problem_free(&p);
        return ORC_ENOMEM;
    }
    for (size_t k = 0; k < m; ++k)
        H.pos[k] = -1;
    /* Initialisation: Q is Accepted with V = q, everything else Far, +inf. */
    init_values(&p, U);
    for (size_t k = 0; k < m; ++k)
        if (p.src[k])
            label[k] = ACCEPTED;
    /* Far neighbours of Accepted nodes become Considered. */
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
            if (p.src[(size_t)j * nx + i]) {
                fmm_touch(&p, U, label, &H, i + 1, j);
                fmm_touch(&p, U, label, &H, i - 1, j);
                fmm_touch(&p, U, label, &H, i, j + 1);
                fmm_touch(&p, U, label, &H, i, j - 1);
            }
    int64_t acc = 0;
    /* Main loop: accept the smallest Considered node, update its neighbours. */
    while (H.size > 0) {
        int32_t k = heap_pop(&H);
        label[k] = ACCEPTED;
        ++acc;
        int i = k % nx, j = k / nx;
        fmm_touch(&p, U, label, &H, i + 1, j);
        fmm_touch(&p, U, label, &H, i - 1, j);
        fmm_touch(&p, U, label, &H, i, j + 1);
        fmm_touch(&p, U, label, &H, i, j - 1);
    }
    if (n_accepted)
        *n_accepted = acc;
    free(label);
    free(H.node);
    free(H.pos);
    problem_free(&p);
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
