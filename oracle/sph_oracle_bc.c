/*
 * sph_oracle_bc.c -- plain CPU reference ("oracle") of
 *   (1) the boundary treatments of the computational domain (Section 3.2.1:
 *       cut-off, symmetric and periodic faces of the axis-aligned box), as
 *       the neighbour images they create;
 *   (2) one time step of Example 1a in the paper's own form (Section 5.1.1,
 *       Eq. SPH_fluid_continuity to Eq. SPH_fluid_momentum, in the equation
 *       order of Appendix A): continuity equation, linear equation of
 *       state, the viscosity Pi_ij with rho_i, symmetric domain walls in
 *       place of boundary particles;
 *   (3) the SPH sampling operator of the performance benchmark (Section 6),
 *       S_i = sum_j A_j m_j / rho_j W_ij.
 * All arithmetic in FP64; the neighbour predicate in FP64 or in the FP32
 * form below.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  It shares no source,
 * header, table or helper with the CUDA library.
 *
 * The step (Appendix A, eq1..eq7), for every particle i:
 *   D_i    = sum_j (m/rho_j) (v_j - v_i) . grad_i W_ij
 *   rho_i' = rho_i + dt (-rho_i D_i)                      (eq1, eq2)
 *   p_i'   = c^2 (rho_i' - rho0)                          (eq3)
 *   a_i    = -sum_j (p_i'/rho_i'^2 + p_j'/rho_j'^2 + Pi_ij) m grad_i W_ij + g
 *   Pi_ij  = -visc c h (v_ji . r_ji) / (rho_i' |r_ji|^2) if v_ji . r_ji < 0,
 *            else 0                                       (eq4, eq5)
 *   v_i'   = v_i + dt a_i,  r_i' = r_i + dt v_i'          (eq6, eq7; fluid only)
 * with grad_i W_ij = (dW/dr)(|r_ij|) r_ij / |r_ij| (0 at r_ij = 0), the
 * Wendland kernel of Section 5.1.1 and the sums over every neighbour image
 * (j, t) with |r_i - r_j^t| < 2h except i itself (t = 0).  visc = 0.1 in
 * Example 1a (the params field visc).
 *
 * Readings of the paper taken here:
 *   - A symmetric face is a mirror plane: every particle j has an image
 *     across it with the position reflected, the velocity component normal
 *     to the face negated and the scalar fields (m, rho, p) unchanged; at a
 *     corner the images across two or three faces are the double / triple
 *     reflections.  Images enter every pair sum as neighbours (i's own image
 *     included) and are never updated themselves.
 *   - A periodic face: the images are the copies shifted by -L or +L,
 *     L = ncell * cs.  A particle that leaves through a periodic face is
 *     shifted back by L (Section 3.2.1); through any other face it is an
 *     error (reported, the state stops at that step).
 *   - A cut-off face has no images.
 *   - Pi_ij = 0 when v_ji . r_ji >= 0, which covers r_ji = 0.
 *   - Boundary particles (kind 1), when present, take part in every sum and
 *     in the continuity equation but are never moved.
 *   - The sampling sum includes j = i.
 *
 * Image codes: per axis t = 0 (the particle itself), 1 (image across the
 * lower face: mirror 2 w_lo - x, or periodic x - L), 2 (image across the
 * upper face: mirror 2 w_hi - x, or periodic x + L); the code of an image is
 * t_x + 3 t_y + 9 t_z.  w_lo = dom_min, w_hi = dom_min + L (the base of
 * cell ncell), L = ncell * cs, each rounded to double.
 *
 * Relative position x_i - x_j^t per axis:
 *   FP64 (also the value every pair sum uses):
 *     t = 0             : x_i - x_j
 *     periodic t = 1, 2 : (x_i + L) - x_j,  (x_i - L) - x_j
 *     symmetric t = 1, 2: (x_i - 2 w_lo) + x_j,  (x_i - 2 w_hi) + x_j
 *   FP32 predicate, from the float cell-relative offsets o = (float)(x -
 *   base(c)) and the cell coordinates c (float products and sums, each
 *   rounded):
 *     t = 0             : (o_i - d cs) - o_j,  d = c_j - c_i
 *     periodic          : the same with d = c_j - ncell - c_i (t = 1) or
 *                         c_j + ncell - c_i (t = 2)
 *     symmetric         : (o_i - S) + o_j,  S = -(c_i + c_j) cs (t = 1) or
 *                         (2 ncell - c_i - c_j) cs (t = 2)
 *   then d2 = fma(z, z, fma(y, y, x*x)) and the test d2 < R2, R2 = (2h)^2 in
 *   the predicate's precision.
 * Only images in the 3^D cells around i's cell are candidates of the cell
 * search; with cs >= 2h that holds every image within the support, which
 * the brute-force search (all j, all image codes) checks.
 *
 * Build: -std=c11 -O2 -ffp-contract=off -fopenmp.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "sph_oracle_bc.h"

/* Wendland kernel and its radial derivative (sph_oracle.c, Section 5.1.1). */
double orc_W(int dim, double h, double r);
double orc_dWdr(int dim, double h, double r);

typedef struct {
    int64_t n_pairs;   /* neighbour images (j, t) != (i, 0) summed, last step */
    double vmax;       /* max |v| over fluid after the last step */
    double amax;       /* max |a| over fluid in the last step */
    double dt_cfl;     /* min(0.25 h/(c + vmax), 0.25 sqrt(h/amax)) */
    int out_of_domain; /* particles outside the grid (or leaving it through a non-periodic face) */
} orc_bc_diag;

/* ---------------------------------------------------------------------- */
/* Grid and images.                                                        */

static double base_of(const orc_bc_params *p, int k, long c)
{
    return p->dom_min[k] + (double)c * p->cs;
}

static double period(const orc_bc_params *p, int k)
{
    return (double)p->ncell[k] * p->cs;
}

/* The largest c with base(c) <= x; -1 outside [base(0), base(ncell)). */
static long cell_of(const orc_bc_params *p, int k, double x)
{
    long nc = p->ncell[k];
    if (!(x >= base_of(p, k, 0)) || !(x < base_of(p, k, nc))) return -1;
    double est = floor((x - p->dom_min[k]) / p->cs);
    long c = (long)(est < 0.0 ? 0.0 : (est > (double)(nc - 1) ? (double)(nc - 1) : est));
    while (c > 0 && base_of(p, k, c) > x) --c;
    while (c + 1 < nc && base_of(p, k, c + 1) <= x) ++c;
    return c;
}

typedef struct {
    int n;
    long ncells;
    long *cc;        /* n x 3 cell coordinates */
    float *off;      /* n x 3 float offsets */
    uint32_t *start; /* ncells + 1 */
    uint32_t *list;  /* particle indices in (cell, id) order */
} grid_t;

static const uint32_t *g_ids;
static int by_id(const void *a, const void *b)
{
    uint32_t x = g_ids[*(const uint32_t *)a], y = g_ids[*(const uint32_t *)b];
    return (x > y) - (x < y);
}

static void grid_free(grid_t *G)
{
    free(G->cc);
    free(G->off);
    free(G->start);
    free(G->list);
    memset(G, 0, sizeof(*G));
}

/* Cells, offsets and the (cell, id) order.  Returns the number of particles
 * outside the grid. */
static int grid_build(const orc_bc_params *p, int n, const double *r, const uint32_t *id, grid_t *G)
{
    int D = p->dim, bad = 0;
    size_t nn = (size_t)(n > 0 ? n : 1);
    G->n = n;
    G->ncells = (long)p->ncell[0] * p->ncell[1] * (D == 3 ? p->ncell[2] : 1);
    G->cc = (long *)calloc(3 * nn, sizeof(long));
    G->off = (float *)calloc(3 * nn, sizeof(float));
    G->start = (uint32_t *)calloc((size_t)G->ncells + 1, sizeof(uint32_t));
    G->list = (uint32_t *)malloc(sizeof(uint32_t) * nn);
    long *lin = (long *)malloc(sizeof(long) * nn);
    for (int i = 0; i < n; ++i) {
        lin[i] = 0;
        for (int k = 0; k < D; ++k) {
            long c = cell_of(p, k, r[(size_t)i * D + k]);
            if (c < 0) {
                lin[i] = -1;
                break;
            }
            G->cc[3 * i + k] = c;
            G->off[3 * i + k] = (float)(r[(size_t)i * D + k] - base_of(p, k, c));
        }
        if (lin[i] < 0) {
            ++bad;
            continue;
        }
        lin[i] = G->cc[3 * i] + (long)p->ncell[0] * (G->cc[3 * i + 1] + (long)p->ncell[1] * G->cc[3 * i + 2]);
        G->start[lin[i] + 1]++;
    }
    for (long c = 0; c < G->ncells; ++c) G->start[c + 1] += G->start[c];
    uint32_t *fill = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(G->ncells > 0 ? G->ncells : 1));
    memcpy(fill, G->start, sizeof(uint32_t) * (size_t)G->ncells);
    for (int i = 0; i < n; ++i)
        if (lin[i] >= 0) G->list[fill[lin[i]]++] = (uint32_t)i;
    g_ids = id;
    for (long c = 0; c < G->ncells; ++c) {
        uint32_t a = G->start[c], b = G->start[c + 1];
        if (b - a > 1) qsort(&G->list[a], b - a, sizeof(uint32_t), by_id);
    }
    free(fill);
    free(lin);
    return bad;
}

typedef orc_image image_t;

/* Relative position of image (j, t[]) seen from i and the predicate.
 * Returns 1 if it is a neighbour. */
static int image_test(const orc_bc_params *p, const double *r, const grid_t *G, int i, int j, const int t[3],
                      image_t *out)
{
    int D = p->dim;
    const double *ri = &r[(size_t)i * D], *rj = &r[(size_t)j * D];
    double x[3] = {0, 0, 0};
    float xf[3] = {0, 0, 0};
    const float csf = (float)p->cs;
    for (int k = 0; k < D; ++k) {
        double L = period(p, k);
        out->vs[k] = 1.0;
        if (t[k] == 0) {
            x[k] = ri[k] - rj[k];
        } else if (p->bc[k] == BC_PERIODIC) {
            x[k] = (t[k] == 1 ? ri[k] + L : ri[k] - L) - rj[k];
        } else { /* symmetric */
            double w = t[k] == 1 ? p->dom_min[k] : base_of(p, k, p->ncell[k]);
            x[k] = (ri[k] - 2.0 * w) + rj[k];
            out->vs[k] = -1.0;
        }
        if (p->fp32) {
            long ci = G->cc[3 * i + k], cj = G->cc[3 * j + k], nc = p->ncell[k];
            float oi = G->off[3 * i + k], oj = G->off[3 * j + k];
            if (t[k] == 0 || p->bc[k] == BC_PERIODIC) {
                long d = cj - ci + (t[k] == 1 ? -nc : (t[k] == 2 ? nc : 0));
                float s = (float)d * csf;
                float a = oi - s;
                xf[k] = a - oj;
            } else {
                long m = t[k] == 1 ? -(ci + cj) : 2 * nc - ci - cj;
                float S = (float)m * csf;
                float a = oi - S;
                xf[k] = a + oj;
            }
        }
    }
    int hit;
    if (p->fp32) {
        float Rf = (float)(2.0 * p->h);
        float d2 = xf[0] * xf[0];
        d2 = fmaf(xf[1], xf[1], d2);
        if (D == 3) d2 = fmaf(xf[2], xf[2], d2);
        hit = d2 < Rf * Rf;
    } else {
        double R = 2.0 * p->h;
        double d2 = fma(x[1], x[1], x[0] * x[0]);
        if (D == 3) d2 = fma(x[2], x[2], d2);
        hit = d2 < R * R;
    }
    out->j = j;
    out->code = t[0] + 3 * t[1] + 9 * t[2];
    out->d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        out->rel[k] = k < D ? x[k] : 0.0;
        if (k >= D) out->vs[k] = 1.0;
        out->d2 += out->rel[k] * out->rel[k];
    }
    return hit;
}

/* Allowed image codes per axis for a brute-force search. */
static int axis_images(const orc_bc_params *p, int k)
{
    return (k < p->dim && p->bc[k] != BC_CUTOFF) ? 3 : 1;
}

typedef struct {
    image_t *v;
    int64_t n, cap;
} image_list;

static void push(image_list *L, const image_t *x)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 64;
        L->v = (image_t *)realloc(L->v, sizeof(image_t) * (size_t)L->cap);
    }
    L->v[L->n++] = *x;
}

/* Neighbour images of i.  method 0: every particle and every image code;
 * 1: the 3^D cells around i's cell, each out-of-grid stencil cell mapped to
 * its image cell (periodic: the cell on the other side; symmetric: i's own
 * cell reflected; cut-off: none). */
static void neighbours_of(const orc_bc_params *p, const double *r, const grid_t *G, int i, int method,
                          image_list *L)
{
    int D = p->dim;
    L->n = 0;
    image_t im;
    if (method == 0) {
        int n0 = axis_images(p, 0), n1 = axis_images(p, 1), n2 = axis_images(p, 2);
        for (int j = 0; j < G->n; ++j)
            for (int t2 = 0; t2 < n2; ++t2)
                for (int t1 = 0; t1 < n1; ++t1)
                    for (int t0 = 0; t0 < n0; ++t0) {
                        int t[3] = {t0, t1, t2};
                        if (j == i && t0 == 0 && t1 == 0 && t2 == 0) continue;
                        if (image_test(p, r, G, i, j, t, &im)) push(L, &im);
                    }
        return;
    }
    const long *ci = &G->cc[3 * i];
    int zlo = D == 3 ? -1 : 0, zhi = D == 3 ? 1 : 0;
    for (int dz = zlo; dz <= zhi; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                int d[3] = {dx, dy, dz};
                long c[3] = {0, 0, 0};
                int t[3] = {0, 0, 0}, skip = 0;
                for (int k = 0; k < D; ++k) {
                    long u = ci[k] + d[k], nc = p->ncell[k];
                    if (u >= 0 && u < nc) {
                        c[k] = u;
                        continue;
                    }
                    if (p->bc[k] == BC_CUTOFF) {
                        skip = 1;
                        break;
                    }
                    t[k] = u < 0 ? 1 : 2;
                    c[k] = p->bc[k] == BC_PERIODIC ? (u < 0 ? u + nc : u - nc) : ci[k];
                }
                if (skip) continue;
                long lc = c[0] + (long)p->ncell[0] * (c[1] + (long)p->ncell[1] * c[2]);
                for (uint32_t q = G->start[lc]; q < G->start[lc + 1]; ++q) {
                    int j = (int)G->list[q];
                    if (j == i && t[0] == 0 && t[1] == 0 && t[2] == 0) continue;
                    if (image_test(p, r, G, i, j, t, &im)) push(L, &im);
                }
            }
}

/* ---------------------------------------------------------------------- */
/* Exported: neighbour images.                                             */

typedef struct {
    uint32_t id;
    uint8_t code;
} id_code;

static int by_id_code(const void *a, const void *b)
{
    const id_code *x = (const id_code *)a, *y = (const id_code *)b;
    if (x->id != y->id) return (x->id > y->id) - (x->id < y->id);
    return (x->code > y->code) - (x->code < y->code);
}

/* Neighbour images of every particle (input order) as (persistent id, image
 * code) pairs sorted by id, then code.  method 0: brute force; 1: cells.
 * offs has n + 1 entries; nbr / img may be NULL to count only.  Returns the
 * total, -1 if a particle is outside the grid, -2 if cap is too small. */
int64_t orc_bc_neighbours(const orc_bc_params *p, int n, const double *r, const uint32_t *id, int method,
                          int64_t *offs, uint32_t *nbr, uint8_t *img, int64_t cap)
{
    grid_t G;
    if (grid_build(p, n, r, id, &G)) {
        grid_free(&G);
        return -1;
    }
    image_list L = {NULL, 0, 0};
    int64_t total = 0;
    offs[0] = 0;
    int rc = 0;
    for (int i = 0; i < n; ++i) {
        neighbours_of(p, r, &G, i, method, &L);
        if (nbr || img) {
            if (total + L.n > cap) {
                rc = -2;
                nbr = NULL;
                img = NULL;
            } else {
                id_code *tmp = (id_code *)malloc(sizeof(id_code) * (size_t)(L.n > 0 ? L.n : 1));
                for (int64_t q = 0; q < L.n; ++q) {
                    tmp[q].id = id[L.v[q].j];
                    tmp[q].code = (uint8_t)L.v[q].code;
                }
                qsort(tmp, (size_t)L.n, sizeof(id_code), by_id_code);
                for (int64_t q = 0; q < L.n; ++q) {
                    if (nbr) nbr[total + q] = tmp[q].id;
                    if (img) img[total + q] = tmp[q].code;
                }
                free(tmp);
            }
        }
        total += L.n;
        offs[i + 1] = total;
    }
    free(L.v);
    grid_free(&G);
    return rc ? rc : total;
}

/* ---------------------------------------------------------------------- */
/* Example 1a in the paper's form.                                          */

static double dot(const double *a, const double *b, int D)
{
    double s = 0.0;
    for (int k = 0; k < D; ++k) s += a[k] * b[k];
    return s;
}

/* grad_i W_ij for relative position rel (0 at rel = 0). */
static void gradW(const orc_bc_params *p, const image_t *im, double gw[3], double *dW)
{
    double rr = sqrt(im->d2);
    *dW = rr > 0.0 ? orc_dWdr(p->dim, p->h, rr) : 0.0;
    for (int k = 0; k < 3; ++k) gw[k] = rr > 0.0 ? *dW * im->rel[k] / rr : 0.0;
}

/* eq1..eq5 at the state (r, v, rho): new density rho1, pressure p1 and
 * acceleration a; per particle the conditioning of the two sums (drho_abs:
 * dt rho_i sum |term| of the continuity sum; aabs: sum |term| + |g| of the
 * momentum sum; asens: change of |a_i| per unit relative error of the
 * densities).  Returns the number of neighbour images, or -1. */
static int64_t eval_1a(const orc_bc_params *p, int n, const double *r, const double *v, const double *rho,
                       const uint8_t *kind, const uint32_t *id, double *rho1, double *p1, double *a,
                       double *drho_abs, double *aabs, double *asens)
{
    grid_t G;
    if (grid_build(p, n, r, id, &G)) {
        grid_free(&G);
        return -1;
    }
    const int D = p->dim;
    const double c2 = p->c * p->c;
    int64_t pairs = 0;
#pragma omp parallel reduction(+ : pairs)
    {
        image_list L = {NULL, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            neighbours_of(p, r, &G, i, 1, &L);
            pairs += L.n;
            const double *vi = &v[(size_t)i * D];
            double Dsum = 0.0, Dabs = 0.0;
            for (int64_t q = 0; q < L.n; ++q) {
                const image_t *im = &L.v[q];
                const double *vj = &v[(size_t)im->j * D];
                double gw[3], dW;
                gradW(p, im, gw, &dW);
                double dv[3] = {0, 0, 0};
                for (int k = 0; k < D; ++k) dv[k] = im->vs[k] * vj[k] - vi[k];
                double term = p->mass / rho[im->j] * dot(dv, gw, D);
                Dsum += term;
                Dabs += fabs(term);
            }
            rho1[i] = rho[i] + p->dt * (-rho[i] * Dsum);
            p1[i] = c2 * (rho1[i] - p->rho0);
            if (drho_abs) drho_abs[i] = p->dt * fabs(rho[i]) * Dabs;
        }
        free(L.v);
    }
    double gnorm = sqrt(dot(p->g, p->g, D));
#pragma omp parallel
    {
        image_list L = {NULL, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            double ai[3] = {0, 0, 0}, absum = 0.0, sens = 0.0;
            if (kind[i] == 0) {
                neighbours_of(p, r, &G, i, 1, &L);
                const double *vi = &v[(size_t)i * D];
                const double Pi_i = p1[i] / (rho1[i] * rho1[i]);
                for (int64_t q = 0; q < L.n; ++q) {
                    const image_t *im = &L.v[q];
                    int j = im->j;
                    const double *vj = &v[(size_t)j * D];
                    double gw[3], dW;
                    gradW(p, im, gw, &dW);
                    /* v_ji . r_ji = (v_j^t - v_i) . (r_j^t - r_i) = v_ij . r_ij */
                    double vr = 0.0;
                    for (int k = 0; k < D; ++k) vr += (vi[k] - im->vs[k] * vj[k]) * im->rel[k];
                    double Pij = 0.0;
                    if (vr < 0.0) Pij = -p->visc * p->c * p->h * vr / (rho1[i] * im->d2);
                    double Pj = p1[j] / (rho1[j] * rho1[j]);
                    double coef = p->mass * (Pi_i + Pj + Pij);
                    for (int k = 0; k < D; ++k) ai[k] -= coef * gw[k];
                    absum += fabs(coef * dW);
                    sens += p->mass * fabs(dW) *
                            (c2 / fabs(rho1[i]) + 2.0 * fabs(p1[i]) / (rho1[i] * rho1[i]) + c2 / fabs(rho1[j]) +
                             2.0 * fabs(p1[j]) / (rho1[j] * rho1[j]) + fabs(Pij));
                }
                for (int k = 0; k < D; ++k) ai[k] += p->g[k];
                absum += gnorm;
            }
            for (int k = 0; k < D; ++k) a[(size_t)i * D + k] = ai[k];
            if (aabs) aabs[i] = absum;
            if (asens) asens[i] = sens;
        }
        free(L.v);
    }
    grid_free(&G);
    return pairs;
}

/* eq1..eq5 without integration (r and v untouched): rho1, p1, a as above,
 * conditioning outputs optional.  Returns the pair count or -1. */
int64_t orc_bc_eval(const orc_bc_params *p, int n, const double *r, const double *v, const double *rho,
                    const uint8_t *kind, const uint32_t *id, double *rho1, double *p1, double *a, double *drho_abs,
                    double *aabs, double *asens)
{
    return eval_1a(p, n, r, v, rho, kind, id, rho1, p1, a, drho_abs, aabs, asens);
}

/* nsteps steps in place on (r, v, rho) (row-major n x dim, input order).
 * p_out / a_out (optional) receive the last step's pressure and
 * acceleration.  Returns 0, or -1 if a particle is outside the grid before
 * a step or leaves it through a non-periodic face (the state then holds the
 * failing step's result). */
int orc_bc_step(const orc_bc_params *p, int n, double *r, double *v, double *rho, const uint8_t *kind,
                const uint32_t *id, int nsteps, double *p_out, double *a_out, orc_bc_diag *diag)
{
    const int D = p->dim;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *rho1 = (double *)malloc(sizeof(double) * nn);
    double *p1 = (double *)malloc(sizeof(double) * nn);
    double *a = (double *)calloc(nn * (size_t)D, sizeof(double));
    int rc = 0;
    if (diag) memset(diag, 0, sizeof(*diag));
    for (int s = 0; s < nsteps && rc == 0; ++s) {
        int64_t pairs = eval_1a(p, n, r, v, rho, kind, id, rho1, p1, a, NULL, NULL, NULL);
        if (pairs < 0) {
            if (diag) diag->out_of_domain = 1;
            rc = -1;
            break;
        }
        double vmax = 0.0, amax = 0.0;
        int left = 0;
        for (int i = 0; i < n; ++i) {
            rho[i] = rho1[i];
            if (kind[i] != 0) continue;
            double v2 = 0.0, a2 = 0.0;
            for (int k = 0; k < D; ++k) {
                size_t q = (size_t)i * D + k;
                v[q] = v[q] + p->dt * a[q];
                r[q] = r[q] + p->dt * v[q];
                v2 += v[q] * v[q];
                a2 += a[q] * a[q];
                double lo = p->dom_min[k], hi = base_of(p, k, p->ncell[k]);
                if (p->bc[k] == BC_PERIODIC) {
                    if (r[q] < lo) r[q] = r[q] + period(p, k);
                    else if (r[q] >= hi) r[q] = r[q] - period(p, k);
                }
                if (!(r[q] >= lo && r[q] < hi)) ++left;
            }
            if (sqrt(v2) > vmax) vmax = sqrt(v2);
            if (sqrt(a2) > amax) amax = sqrt(a2);
        }
        if (diag) {
            diag->n_pairs = pairs;
            diag->vmax = vmax;
            diag->amax = amax;
            double t1 = 0.25 * p->h / (p->c + vmax);
            double t2 = amax > 0.0 ? 0.25 * sqrt(p->h / amax) : INFINITY;
            diag->dt_cfl = t1 < t2 ? t1 : t2;
            diag->out_of_domain = left;
        }
        if (left) rc = -1;
    }
    if (p_out) memcpy(p_out, p1, sizeof(double) * (size_t)n);
    if (a_out) memcpy(a_out, a, sizeof(double) * (size_t)n * (size_t)D);
    free(rho1);
    free(p1);
    free(a);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* The sampling operator of the benchmark of Section 6.                    */

/* S_i = sum over the neighbour images (j, t) of i, i itself included, of
 * A_j m_j / rho_j W(|r_i - r_j^t|); Sabs (optional) the same sum of
 * absolute values.  Returns the number of neighbour images (self excluded)
 * or -1. */
int64_t orc_bc_sample(const orc_bc_params *p, int n, const double *r, const uint32_t *id, const double *A,
                      const double *m, const double *rho, double *S, double *Sabs)
{
    grid_t G;
    if (grid_build(p, n, r, id, &G)) {
        grid_free(&G);
        return -1;
    }
    const double W0 = orc_W(p->dim, p->h, 0.0);
    int64_t pairs = 0;
#pragma omp parallel reduction(+ : pairs)
    {
        image_list L = {NULL, 0, 0};
#pragma omp for schedule(dynamic, 64)
        for (int i = 0; i < n; ++i) {
            neighbours_of(p, r, &G, i, 1, &L);
            pairs += L.n;
            double self = A[i] * m[i] / rho[i] * W0;
            double s = self, sa = fabs(self);
            for (int64_t q = 0; q < L.n; ++q) {
                int j = L.v[q].j;
                double t = A[j] * m[j] / rho[j] * orc_W(p->dim, p->h, sqrt(L.v[q].d2));
                s += t;
                sa += fabs(t);
            }
            S[i] = s;
            if (Sabs) Sabs[i] = sa;
        }
        free(L.v);
    }
    grid_free(&G);
    return pairs;
}

/* ---------------------------------------------------------------------- */
/* Image lists for the other oracle files (sph_oracle_bc.h).               */

int64_t orc_bc_images(const orc_bc_params *p, int n, const double *r, const uint32_t *id, int64_t *offs,
                      orc_image *out, int64_t cap)
{
    grid_t G;
    if (grid_build(p, n, r, id, &G)) {
        grid_free(&G);
        return -1;
    }
    image_list L = {NULL, 0, 0};
    int64_t total = 0;
    int rc = 0;
    offs[0] = 0;
    for (int i = 0; i < n; ++i) {
        neighbours_of(p, r, &G, i, 1, &L);
        if (out && !rc) {
            if (total + L.n > cap) rc = -2;
            else memcpy(out + total, L.v, sizeof(orc_image) * (size_t)L.n);
        }
        total += L.n;
        offs[i + 1] = total;
    }
    free(L.v);
    grid_free(&G);
    return rc ? rc : total;
}
