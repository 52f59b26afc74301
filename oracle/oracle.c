/*
 * oracle.c -- plain FP64 CPU oracle for two-dimensional Smart Laplacian
 * smoothing (Zhao, Mei, Xu, Zhang, "On the Accelerating of Two-dimensional
 * Smart Laplacian Smoothing on the GPU").
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the package's smoke check and
 * the benchmark's CPU-baseline leg may load this file.  The library under
 * test (the CUDA path) never calls it, includes it or shares a line with it.
 *
 * Every step is written in the order the paper describes it, with plain
 * sequential loops and no blocking or reordering:
 *   - finding of neighbours and incident triangles      (Section 3.3.2)
 *   - determining of constraints (boundary vertices)     (Section 3.3.3)
 *   - element quality, Lee and Lo's alpha                (Section 3.3.1)
 *   - Laplacian relocation, Form A (Jacobi)              (Section 2.2, Eq. 2)
 *   - the "smart" accept test on the worst incident
 *     element quality                                    (Sections 2.1, 3.3.4)
 *   - refresh of qualities after every full pass         (Section 3.3.4)
 *
 * Readings where the paper is silent (each one is also listed in the design
 * notes of the repository):
 *   R1  neighbour summation order: ascending (x0, y0, index), where (x0, y0)
 *       are the coordinates given when the mesh was created;
 *   R2  alpha = 2*sqrt(3) * cross / (|e1|^2 + |e2|^2 + |e3|^2) with the signed
 *       cross product of the triangle in its stored vertex order, evaluated
 *       with one fixed expression tree (see orc_alpha); 0 when the edge sum
 *       is not positive.  Parity unpinned against the paper for this one
 *       definition: the paper names Lee and Lo's measure but prints neither
 *       its formula nor a value, so alpha is pinned only to textbook values
 *       (equilateral 1, right isosceles sqrt(3)/2, degenerate 0, Heron's
 *       formula);
 *   R3  accept iff q_new >= q_old ("does not get worse"); strict mode uses
 *       q_new > q_old, the paper's "is increased";
 *   R4  stop after max_iter passes, or earlier when tol > 0 and the largest
 *       squared displacement of a pass is below (tol * D)^2, D being the
 *       bounding-box diagonal of the coordinates given at creation;
 *   R5  a node is fixed when it was flagged by the caller, or (no flags
 *       given) when some neighbour shares exactly one triangle with it, or
 *       when it belongs to no triangle.
 *
 * Floating point: FP64 only, compiled with -ffp-contract=off and without
 * -ffast-math, so every + - * / below is one IEEE-754 round-to-nearest
 * operation in the order written.
 *
 * An OpenMP build of this same source (-fopenmp) parallelises the loop over
 * nodes of one pass; Form A reads only the previous pass, so the result is
 * identical to the sequential build.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_INVALID 1
#define ORC_NONMANIFOLD 2
#define ORC_NOMEM 3

/* 2*sqrt(3) rounded to the nearest double; alpha = 4*sqrt(3)*area / sum(l^2)
 * and cross = 2*area. */
static const double ORC_K = 3.4641016151377544;

typedef struct orc_mesh {
    int64_t n, m;
    int32_t *tri;        /* 3m vertex ids, stored order                 */
    double *xy0;         /* 2n coordinates given at creation            */
    uint8_t *fixed;      /* n: 1 = constrained (boundary) node          */
    int64_t *nbr_ptr;    /* n+1: N(i) = nbr[nbr_ptr[i] .. nbr_ptr[i+1]) */
    int32_t *nbr;
    int64_t *tri_ptr;    /* n+1: T(i) = tri_of[tri_ptr[i] .. ]          */
    int32_t *tri_of;
    double diag;         /* D = bounding-box diagonal of xy0            */
} orc_mesh;

/* ---- Section 3.3.1: the element quality (Lee and Lo's alpha) ----------- */

double orc_alpha(double ax, double ay, double bx, double by, double cx, double cy)
{
    double e1x = bx - ax, e1y = by - ay;   /* edge a->b */
    double e2x = cx - ax, e2y = cy - ay;   /* edge a->c */
    double e3x = cx - bx, e3y = cy - by;   /* edge b->c */
    double cross = e1x * e2y - e1y * e2x;  /* twice the signed area */
    double l1 = e1x * e1x + e1y * e1y;
    double l2 = e2x * e2x + e2y * e2y;
    double l3 = e3x * e3x + e3y * e3y;
    double s = (l1 + l2) + l3;
    if (s > 0.0)
        return (ORC_K * cross) / s;
    return 0.0;
}

/* ---- helpers for the neighbour finding ---------------------------------- */

static const double *g_sort_xy; /* coordinates used as the sort key (R1) */

static int cmp_int32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static int cmp_canonical(const void *a, const void *b)
{
    int32_t i = *(const int32_t *)a, j = *(const int32_t *)b;
    double xi = g_sort_xy[2 * (int64_t)i], yi = g_sort_xy[2 * (int64_t)i + 1];
    double xj = g_sort_xy[2 * (int64_t)j], yj = g_sort_xy[2 * (int64_t)j + 1];
    if (xi < xj) return -1;
    if (xi > xj) return 1;
    if (yi < yj) return -1;
    if (yi > yj) return 1;
    return (i > j) - (i < j);
}

void orc_free(orc_mesh *M)
{
    if (!M) return;
    free(M->tri); free(M->xy0); free(M->fixed);
    free(M->nbr_ptr); free(M->nbr); free(M->tri_ptr); free(M->tri_of);
    free(M);
}

/* Builds the mesh: validation, neighbours and incident triangles
 * (Section 3.3.2), constraints (Section 3.3.3), and D (R4).
 * boundary may be NULL (derive the flags).  *status receives ORC_*. */
orc_mesh *orc_create(int64_t n, int64_t m, const double *xy, const int32_t *tri,
                     const uint8_t *boundary, int *status)
{
    *status = ORC_INVALID;
    if (n < 3 || m < 1 || !xy || !tri) return NULL;
    for (int64_t i = 0; i < 2 * n; i++)
        if (!isfinite(xy[i])) return NULL;
    for (int64_t t = 0; t < m; t++) {
        int32_t a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
        if (a < 0 || b < 0 || c < 0 || a >= n || b >= n || c >= n) return NULL;
        if (a == b || b == c || a == c) return NULL;
    }

    orc_mesh *M = (orc_mesh *)calloc(1, sizeof(orc_mesh));
    *status = ORC_NOMEM;
    if (!M) return NULL;
    M->n = n;
    M->m = m;
    M->tri = (int32_t *)malloc(sizeof(int32_t) * 3 * m);
    M->xy0 = (double *)malloc(sizeof(double) * 2 * n);
    M->fixed = (uint8_t *)calloc(n, 1);
    M->tri_ptr = (int64_t *)calloc(n + 1, sizeof(int64_t));
    M->tri_of = (int32_t *)malloc(sizeof(int32_t) * 3 * m);
    M->nbr_ptr = (int64_t *)calloc(n + 1, sizeof(int64_t));
    if (!M->tri || !M->xy0 || !M->fixed || !M->tri_ptr || !M->tri_of || !M->nbr_ptr) {
        orc_free(M);
        return NULL;
    }
    memcpy(M->tri, tri, sizeof(int32_t) * 3 * m);
    memcpy(M->xy0, xy, sizeof(double) * 2 * n);

    /* Section 3.3.2: every triangle is incident to its three vertices.
     * T(i) lists the triangles in ascending triangle id. */
    for (int64_t t = 0; t < m; t++)
        for (int k = 0; k < 3; k++)
            M->tri_ptr[tri[3 * t + k] + 1] += 1;
    for (int64_t i = 0; i < n; i++)
        M->tri_ptr[i + 1] += M->tri_ptr[i];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * n);
        if (!fill) { orc_free(M); return NULL; }
        for (int64_t i = 0; i < n; i++) fill[i] = M->tri_ptr[i];
        for (int64_t t = 0; t < m; t++)
            for (int k = 0; k < 3; k++) {
                int32_t v = tri[3 * t + k];
                M->tri_of[fill[v]++] = (int32_t)t;
            }
        free(fill);
    }

    /* Section 3.3.2: the other two vertices of each incident triangle are
     * neighbours.  Each neighbour across an interior edge is recorded twice
     * (once per triangle on either side of the edge); Section 3.3.3 uses the
     * number of records to find the boundary. */
    int64_t cap = 2 * 3 * m;
    int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * (cap > 0 ? cap : 1));
    int32_t *rec = (int32_t *)malloc(sizeof(int32_t) * (cap > 0 ? cap : 1));
    if (!nb || !rec) { free(nb); free(rec); orc_free(M); return NULL; }
    int64_t nnz = 0;
    int nonmanifold = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t r = 0;
        for (int64_t k = M->tri_ptr[i]; k < M->tri_ptr[i + 1]; k++) {
            int64_t t = M->tri_of[k];
            for (int c = 0; c < 3; c++)
                if (tri[3 * t + c] != i) rec[r++] = tri[3 * t + c];
        }
        qsort(rec, (size_t)r, sizeof(int32_t), cmp_int32);
        int on_boundary = (r == 0); /* R5: a node in no triangle stays put */
        int64_t start = nnz;
        for (int64_t k = 0; k < r;) {
            int64_t e = k;
            while (e < r && rec[e] == rec[k]) e++;
            int64_t times = e - k;      /* triangles sharing edge (i, rec[k]) */
            if (times != 2) on_boundary = 1;
            if (times > 2) nonmanifold = 1;
            nb[nnz++] = rec[k];
            k = e;
        }
        /* R1: canonical summation order of the neighbours */
        g_sort_xy = xy;
        qsort(nb + start, (size_t)(nnz - start), sizeof(int32_t), cmp_canonical);
        M->nbr_ptr[i + 1] = nnz;
        M->fixed[i] = boundary ? (boundary[i] != 0 || r == 0) : (uint8_t)on_boundary;
    }
    free(rec);
    if (nonmanifold) {
        free(nb);
        orc_free(M);
        *status = ORC_NONMANIFOLD;
        return NULL;
    }
    M->nbr = (int32_t *)realloc(nb, sizeof(int32_t) * (nnz > 0 ? nnz : 1));
    if (!M->nbr) { free(nb); orc_free(M); return NULL; }

    /* R4: bounding-box diagonal of the coordinates given at creation */
    double xmin = xy[0], xmax = xy[0], ymin = xy[1], ymax = xy[1];
    for (int64_t i = 1; i < n; i++) {
        double x = xy[2 * i], y = xy[2 * i + 1];
        if (x < xmin) xmin = x;
        if (x > xmax) xmax = x;
        if (y < ymin) ymin = y;
        if (y > ymax) ymax = y;
    }
    M->diag = sqrt((xmax - xmin) * (xmax - xmin) + (ymax - ymin) * (ymax - ymin));
    *status = ORC_OK;
    return M;
}

int64_t orc_n(const orc_mesh *M) { return M->n; }
int64_t orc_m(const orc_mesh *M) { return M->m; }
int64_t orc_nnz(const orc_mesh *M) { return M->nbr_ptr[M->n]; }
double orc_diag(const orc_mesh *M) { return M->diag; }

void orc_get_adjacency(const orc_mesh *M, int64_t *nbr_ptr, int32_t *nbr,
                       int64_t *tri_ptr, int32_t *tri_of, uint8_t *fixed)
{
    if (nbr_ptr) memcpy(nbr_ptr, M->nbr_ptr, sizeof(int64_t) * (M->n + 1));
    if (nbr) memcpy(nbr, M->nbr, sizeof(int32_t) * M->nbr_ptr[M->n]);
    if (tri_ptr) memcpy(tri_ptr, M->tri_ptr, sizeof(int64_t) * (M->n + 1));
    if (tri_of) memcpy(tri_of, M->tri_of, sizeof(int32_t) * M->tri_ptr[M->n]);
    if (fixed) memcpy(fixed, M->fixed, (size_t)M->n);
}

/* ---- Sections 2.1, 2.2 and 3.3.4: one node of one Form-A pass ------------
 * Reads only xy (the coordinates X^q of the previous pass).  Writes the
 * node's coordinates for pass q+1, whether the move was accepted, and the
 * squared displacement (0 when not moved).  Also returns q_old / q_new. */
static void node_update(const orc_mesh *M, const double *xy, int64_t i, int strict,
                        double *out_x, double *out_y, int *accepted, double *d2,
                        double *q_old_out, double *q_new_out, double *cand_out)
{
    double xi = xy[2 * i], yi = xy[2 * i + 1];
    *out_x = xi;
    *out_y = yi;
    *accepted = 0;
    *d2 = 0.0;
    if (q_old_out) *q_old_out = 0.0;
    if (q_new_out) *q_new_out = 0.0;
    if (cand_out) { cand_out[0] = xi; cand_out[1] = yi; }
    if (M->fixed[i]) return; /* Section 3.3.3: constrained nodes never move */

    /* Eq. 2: the geometric centre of the neighbours at pass q */
    int64_t b = M->nbr_ptr[i], e = M->nbr_ptr[i + 1];
    int64_t N = e - b;
    double sx = xy[2 * (int64_t)M->nbr[b]];
    double sy = xy[2 * (int64_t)M->nbr[b] + 1];
    for (int64_t k = b + 1; k < e; k++) {
        sx = sx + xy[2 * (int64_t)M->nbr[k]];
        sy = sy + xy[2 * (int64_t)M->nbr[k] + 1];
    }
    double cx = sx / (double)N;
    double cy = sy / (double)N;
    if (cand_out) { cand_out[0] = cx; cand_out[1] = cy; }

    /* Section 3.3.4: worst quality of the incident triangles before the move
     * (all vertices at pass q) and after it (this node at the centre, the
     * others still at pass q). */
    double q_old = 0.0, q_new = 0.0;
    int first = 1;
    for (int64_t k = M->tri_ptr[i]; k < M->tri_ptr[i + 1]; k++) {
        int64_t t = M->tri_of[k];
        double px[3], py[3], mx[3], my[3];
        for (int c = 0; c < 3; c++) {
            int64_t v = M->tri[3 * t + c];
            px[c] = xy[2 * v];
            py[c] = xy[2 * v + 1];
            mx[c] = (v == i) ? cx : px[c];
            my[c] = (v == i) ? cy : py[c];
        }
        double qb = orc_alpha(px[0], py[0], px[1], py[1], px[2], py[2]);
        double qa = orc_alpha(mx[0], my[0], mx[1], my[1], mx[2], my[2]);
        if (first || qb < q_old) q_old = qb;
        if (first || qa < q_new) q_new = qa;
        first = 0;
    }
    if (q_old_out) *q_old_out = q_old;
    if (q_new_out) *q_new_out = q_new;

    /* Section 2.1 / R3: keep the move only if the local quality does not drop */
    int ok = strict ? (q_new > q_old) : (q_new >= q_old);
    if (ok) {
        double dx = cx - xi, dy = cy - yi;
        *out_x = cx;
        *out_y = cy;
        *accepted = 1;
        *d2 = dx * dx + dy * dy;
    }
}

/* One full Form-A pass: xy_next[i] from xy only.  accept may be NULL. */
void orc_sweep(const orc_mesh *M, const double *xy, double *xy_next, int strict,
               uint8_t *accept, double *maxd2_out, int64_t *nacc_out)
{
    double maxd2 = 0.0;
    int64_t nacc = 0;
    int64_t n = M->n;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) reduction(max : maxd2) reduction(+ : nacc)
#endif
    for (int64_t i = 0; i < n; i++) {
        double x, y, d2;
        int acc;
        node_update(M, xy, i, strict, &x, &y, &acc, &d2, NULL, NULL, NULL);
        xy_next[2 * i] = x;
        xy_next[2 * i + 1] = y;
        if (accept) accept[i] = (uint8_t)acc;
        nacc += acc;
        if (d2 > maxd2) maxd2 = d2;
    }
    *maxd2_out = maxd2;
    *nacc_out = nacc;
}

/* The update of a list of nodes from X^q (same arithmetic as orc_sweep).
 * out_cand (may be NULL) receives each node's candidate position (the centre). */
void orc_update_nodes(const orc_mesh *M, const double *xy, int strict, int64_t k,
                      const int64_t *idx, double *out_xy, uint8_t *out_acc, double *out_d2,
                      double *out_qold, double *out_qnew, double *out_cand)
{
    for (int64_t r = 0; r < k; r++) {
        double x, y, d2, qo, qn;
        int acc;
        node_update(M, xy, idx[r], strict, &x, &y, &acc, &d2, &qo, &qn,
                    out_cand ? out_cand + 2 * r : NULL);
        out_xy[2 * r] = x;
        out_xy[2 * r + 1] = y;
        if (out_acc) out_acc[r] = (uint8_t)acc;
        if (out_d2) out_d2[r] = d2;
        if (out_qold) out_qold[r] = qo;
        if (out_qnew) out_qnew[r] = qn;
    }
}

/* Section 3.3.4 iteration loop, Form A as the paper describes it: compute the
 * pass into a second array, then copy ("swap") it back.  xy is updated in
 * place.  accept_last (may be NULL) gets the decisions of the last pass.
 * Returns 0, or ORC_NOMEM. */
int orc_smooth(const orc_mesh *M, double *xy, int32_t max_iter, double tol, int strict,
               uint8_t *accept_last, int32_t *iterations, int32_t *converged,
               int64_t *nacc_last, double *maxd2_last)
{
    int64_t n = M->n;
    double *next = (double *)malloc(sizeof(double) * 2 * n);
    if (!next) return ORC_NOMEM;
    double thr = (tol * M->diag) * (tol * M->diag); /* R4 */
    int32_t it = 0;
    int32_t conv = 0;
    int64_t nacc = 0;
    double maxd2 = 0.0;
    while (it < max_iter) {
        orc_sweep(M, xy, next, strict, accept_last, &maxd2, &nacc);
        memcpy(xy, next, sizeof(double) * 2 * n);
        it += 1;
        if (tol > 0.0 && maxd2 < thr) {
            conv = 1;
            break;
        }
    }
    free(next);
    *iterations = it;
    *converged = conv;
    *nacc_last = nacc;
    *maxd2_last = maxd2;
    return ORC_OK;
}

/* ---- Eq. 3, Form B, made deterministic: multicolour Gauss-Seidel ---------
 * Form B updates the nodes in place, each reading the newest coordinates of
 * its neighbours (Eq. 3), so a parallel run depends on the update order.  The
 * reading used here (R9): colour the free nodes so that no two neighbours
 * share a colour, then update one colour class after the other, each node
 * reading the coordinates as they are at that moment (neighbours of earlier
 * classes already moved in this sweep).  Nodes of one class are never
 * neighbours, so a class gives the same result in any order.
 *
 * Colouring (R10): Jones-Plassmann rounds.  Priority of node i:
 * splitmix64(seed + i) (Steele, Lea and Flood, OOPSLA 2014), ties by index.
 * In each round, every uncoloured free node whose (priority, index) exceeds
 * that of each uncoloured free neighbour takes the smallest colour not held by
 * a neighbour coloured in an earlier round. */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int beats(uint64_t pi, int64_t i, uint64_t pj, int64_t j)
{
    return pi > pj || (pi == pj && i > j);
}

/* colour[i] = class of free node i, -1 for fixed nodes.  Returns the number of
 * classes in *ncolours and the number of rounds in *rounds.  0 or ORC_NOMEM. */
int orc_colour(const orc_mesh *M, uint64_t seed, int32_t *colour, int32_t *ncolours, int32_t *rounds)
{
    int64_t n = M->n;
    uint64_t *prio = (uint64_t *)malloc(sizeof(uint64_t) * (n > 0 ? n : 1));
    uint8_t *win = (uint8_t *)malloc(n > 0 ? n : 1);
    int64_t maxdeg = 0;
    for (int64_t i = 0; i < n; i++)
        if (M->nbr_ptr[i + 1] - M->nbr_ptr[i] > maxdeg) maxdeg = M->nbr_ptr[i + 1] - M->nbr_ptr[i];
    uint8_t *used = (uint8_t *)malloc((size_t)maxdeg + 1);
    if (!prio || !win || !used) {
        free(prio);
        free(win);
        free(used);
        return ORC_NOMEM;
    }
    int64_t left = 0;
    for (int64_t i = 0; i < n; i++) {
        prio[i] = splitmix64(seed + (uint64_t)i);
        colour[i] = -1;
        if (!M->fixed[i]) left++;
    }
    int32_t nc = 0, r = 0;
    while (left > 0) {
        /* the winners of this round, against the state at its start */
        for (int64_t i = 0; i < n; i++) {
            win[i] = 0;
            if (M->fixed[i] || colour[i] >= 0) continue;
            int w = 1;
            for (int64_t k = M->nbr_ptr[i]; k < M->nbr_ptr[i + 1]; k++) {
                int64_t j = M->nbr[k];
                if (M->fixed[j] || colour[j] >= 0) continue;
                if (!beats(prio[i], i, prio[j], j)) w = 0;
            }
            win[i] = (uint8_t)w;
        }
        /* winners are pairwise non-adjacent: colour them from earlier rounds */
        for (int64_t i = 0; i < n; i++) {
            if (!win[i]) continue;
            int64_t deg = M->nbr_ptr[i + 1] - M->nbr_ptr[i];
            for (int64_t c = 0; c <= deg; c++) used[c] = 0;
            for (int64_t k = M->nbr_ptr[i]; k < M->nbr_ptr[i + 1]; k++) {
                int32_t cj = colour[M->nbr[k]];
                if (cj >= 0 && cj <= deg && !win[M->nbr[k]]) used[cj] = 1;
            }
            int32_t c = 0;
            while (used[c]) c++;
            colour[i] = c;
            if (c + 1 > nc) nc = c + 1;
            left--;
        }
        r++;
    }
    free(prio);
    free(win);
    free(used);
    *ncolours = nc;
    *rounds = r;
    return ORC_OK;
}

/* One Form-B sweep in colour order, in place.  accept may be NULL. */
void orc_sweep_coloured(const orc_mesh *M, double *xy, const int32_t *colour, int32_t ncolours,
                        int strict, uint8_t *accept, double *maxd2_out, int64_t *nacc_out)
{
    double maxd2 = 0.0;
    int64_t nacc = 0;
    int64_t n = M->n;
    if (accept)
        for (int64_t i = 0; i < n; i++) accept[i] = 0;
    for (int32_t c = 0; c < ncolours; c++) {
        for (int64_t i = 0; i < n; i++) {
            if (colour[i] != c) continue;
            double x, y, d2;
            int acc;
            node_update(M, xy, i, strict, &x, &y, &acc, &d2, NULL, NULL, NULL);
            xy[2 * i] = x;
            xy[2 * i + 1] = y;
            if (accept) accept[i] = (uint8_t)acc;
            nacc += acc;
            if (d2 > maxd2) maxd2 = d2;
        }
    }
    *maxd2_out = maxd2;
    *nacc_out = nacc;
}

/* The Form-B iteration: sweeps in colour order with the stop rule R4. */
int orc_smooth_coloured(const orc_mesh *M, double *xy, const int32_t *colour, int32_t ncolours,
                        int32_t max_iter, double tol, int strict, uint8_t *accept_last,
                        int32_t *iterations, int32_t *converged, int64_t *nacc_last, double *maxd2_last)
{
    double thr = (tol * M->diag) * (tol * M->diag); /* R4 */
    int32_t it = 0;
    int32_t conv = 0;
    int64_t nacc = 0;
    double maxd2 = 0.0;
    while (it < max_iter) {
        orc_sweep_coloured(M, xy, colour, ncolours, strict, accept_last, &maxd2, &nacc);
        it += 1;
        if (tol > 0.0 && maxd2 < thr) {
            conv = 1;
            break;
        }
    }
    *iterations = it;
    *converged = conv;
    *nacc_last = nacc;
    *maxd2_last = maxd2;
    return ORC_OK;
}

/* ---- Forms A and B in binary32, the paper's precision (Section 4) --------
 * Reading R11: the coordinates are held as binary32 values (the creation
 * coordinates rounded to nearest) and every operation is one binary32
 * round-to-nearest operation in the order of the FP64 definition above, with
 * K32 the float nearest to 2*sqrt(3).  Summation order (R1) and constraints
 * are those of the mesh; the stop rule compares the largest squared move,
 * widened exactly to double, with (tol * D)^2 computed in double. */
static const float ORC_K32 = 3.46410161514f;

float orc32_alpha(float ax, float ay, float bx, float by, float cx, float cy)
{
    float e1x = bx - ax, e1y = by - ay;
    float e2x = cx - ax, e2y = cy - ay;
    float e3x = cx - bx, e3y = cy - by;
    float cross = e1x * e2y - e1y * e2x;
    float l1 = e1x * e1x + e1y * e1y;
    float l2 = e2x * e2x + e2y * e2y;
    float l3 = e3x * e3x + e3y * e3y;
    float s = (l1 + l2) + l3;
    if (s > 0.0f)
        return (ORC_K32 * cross) / s;
    return 0.0f;
}

/* One node of one pass in binary32 (the steps of node_update). */
static void node_update32(const orc_mesh *M, const float *xy, int64_t i, int strict, float *out_x,
                          float *out_y, int *accepted, float *d2)
{
    float xi = xy[2 * i], yi = xy[2 * i + 1];
    *out_x = xi;
    *out_y = yi;
    *accepted = 0;
    *d2 = 0.0f;
    if (M->fixed[i]) return;
    int64_t b = M->nbr_ptr[i], e = M->nbr_ptr[i + 1];
    int64_t N = e - b;
    float sx = xy[2 * (int64_t)M->nbr[b]];
    float sy = xy[2 * (int64_t)M->nbr[b] + 1];
    for (int64_t k = b + 1; k < e; k++) {
        sx = sx + xy[2 * (int64_t)M->nbr[k]];
        sy = sy + xy[2 * (int64_t)M->nbr[k] + 1];
    }
    float cx = sx / (float)N;
    float cy = sy / (float)N;
    float q_old = 0.0f, q_new = 0.0f;
    int first = 1;
    for (int64_t k = M->tri_ptr[i]; k < M->tri_ptr[i + 1]; k++) {
        int64_t t = M->tri_of[k];
        float px[3], py[3], mx[3], my[3];
        for (int c = 0; c < 3; c++) {
            int64_t v = M->tri[3 * t + c];
            px[c] = xy[2 * v];
            py[c] = xy[2 * v + 1];
            mx[c] = (v == i) ? cx : px[c];
            my[c] = (v == i) ? cy : py[c];
        }
        float qb = orc32_alpha(px[0], py[0], px[1], py[1], px[2], py[2]);
        float qa = orc32_alpha(mx[0], my[0], mx[1], my[1], mx[2], my[2]);
        if (first || qb < q_old) q_old = qb;
        if (first || qa < q_new) q_new = qa;
        first = 0;
    }
    int ok = strict ? (q_new > q_old) : (q_new >= q_old);
    if (ok) {
        float dx = cx - xi, dy = cy - yi;
        *out_x = cx;
        *out_y = cy;
        *accepted = 1;
        *d2 = dx * dx + dy * dy;
    }
}

/* One binary32 sweep: Form A into xy_next (colour == NULL), or Form B in
 * colour order in place (xy_next == xy). */
void orc32_sweep(const orc_mesh *M, float *xy, float *xy_next, const int32_t *colour, int32_t ncolours,
                 int strict, uint8_t *accept, float *maxd2_out, int64_t *nacc_out)
{
    float maxd2 = 0.0f;
    int64_t nacc = 0;
    int64_t n = M->n;
    if (accept)
        for (int64_t i = 0; i < n; i++) accept[i] = 0;
    int32_t classes = colour ? ncolours : 1;
    for (int32_t c = 0; c < classes; c++) {
        for (int64_t i = 0; i < n; i++) {
            if (colour && colour[i] != c) continue;
            float x, y, d2;
            int acc;
            node_update32(M, xy, i, strict, &x, &y, &acc, &d2);
            xy_next[2 * i] = x;
            xy_next[2 * i + 1] = y;
            if (accept) accept[i] = (uint8_t)acc;
            nacc += acc;
            if (d2 > maxd2) maxd2 = d2;
        }
    }
    *maxd2_out = maxd2;
    *nacc_out = nacc;
}

/* The binary32 iteration (Form A with copy-back, or Form B in place). */
int orc32_smooth(const orc_mesh *M, float *xy, const int32_t *colour, int32_t ncolours, int32_t max_iter,
                 double tol, int strict, uint8_t *accept_last, int32_t *iterations, int32_t *converged,
                 int64_t *nacc_last, double *maxd2_last)
{
    int64_t n = M->n;
    float *next = colour ? xy : (float *)malloc(sizeof(float) * 2 * (n > 0 ? n : 1));
    if (!next) return ORC_NOMEM;
    double thr = (tol * M->diag) * (tol * M->diag); /* R4 */
    int32_t it = 0, conv = 0;
    int64_t nacc = 0;
    float maxd2 = 0.0f;
    while (it < max_iter) {
        orc32_sweep(M, xy, next, colour, ncolours, strict, accept_last, &maxd2, &nacc);
        if (!colour) memcpy(xy, next, sizeof(float) * 2 * n);
        it += 1;
        if (tol > 0.0 && (double)maxd2 < thr) {
            conv = 1;
            break;
        }
    }
    if (!colour) free(next);
    *iterations = it;
    *converged = conv;
    *nacc_last = nacc;
    *maxd2_last = (double)maxd2;
    return ORC_OK;
}

/* Quality histogram of all triangles at coordinates xy (Section 3.3.1).
 * bin = floor((q - lo) / (hi - lo) * nbins), clamped to [0, nbins-1];
 * qmean sums the qualities in triangle order. */
void orc_histogram(const orc_mesh *M, const double *xy, int32_t nbins, double lo, double hi,
                   int64_t *counts, double *qmin, double *qmean)
{
    for (int32_t b = 0; b < nbins; b++) counts[b] = 0;
    double mn = 0.0, sum = 0.0;
    for (int64_t t = 0; t < M->m; t++) {
        int64_t a = M->tri[3 * t], b = M->tri[3 * t + 1], c = M->tri[3 * t + 2];
        double q = orc_alpha(xy[2 * a], xy[2 * a + 1], xy[2 * b], xy[2 * b + 1],
                             xy[2 * c], xy[2 * c + 1]);
        double f = floor((q - lo) / (hi - lo) * (double)nbins);
        int32_t bin;
        if (f < 0.0) bin = 0;
        else if (f >= (double)nbins) bin = nbins - 1;
        else bin = (int32_t)f;
        counts[bin] += 1;
        if (t == 0 || q < mn) mn = q;
        sum = sum + q;
    }
    *qmin = mn;
    *qmean = sum / (double)M->m;
}
