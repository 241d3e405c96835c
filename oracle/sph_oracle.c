/*
 * sph_oracle.c -- plain CPU reference ("oracle") of one explicit
 * weakly-compressible SPH time step, in FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  It shares no source,
 * header, table or helper with the CUDA library; the two meet only on the
 * seeded input arrays.
 *
 * What it follows (arXiv:1710.08259, "Nauticle"):
 *   - Section 3.2.1: an axis-aligned domain split into a uniform grid of
 *     cells whose edge is at least the influence radius; the neighbour
 *     search only looks at adjacent cells.
 *   - Section 5.1, SPH interpolant <A_i> = sum_j A_j W_ij m_j / rho_j, used
 *     with A = rho (summation density).
 *   - Section 5.1, Eq. (diffop1): symmetric gradient, giving the pressure
 *     term -sum_j (p_i/rho_i^2 + p_j/rho_j^2 + Pi_ij) m_j grad_i W_ij + g of
 *     the momentum equation of Example 1a.
 *   - Section 5.1.1, the artificial viscosity Pi_ij (used in its symmetric
 *     Monaghan form, see the readings below).
 *   - Section 5.1.1, the Wendland kernel W = alpha_D (1 - q/2)^4 (2q + 1),
 *     q = r/h, support 2h, alpha_2 = 7/(4 pi h^2), alpha_3 = 21/(16 pi h^3).
 *   - Section 5.1.1 / Appendix A equation order: first-order semi-implicit
 *     Euler, v updated first and r advanced with the new v.
 *
 * Readings where the paper is silent or differs from the workload:
 * summation density instead of the continuity
 * equation; Tait EOS p = B((rho/rho_ref)^gamma - 1), B = c0^2 rho0 / gamma,
 * negative pressure clamped to 0; rho_ref = m * (lattice sum of W) so that
 * the unperturbed lattice is at rest; Pi_ij = -alpha c0 h (v_ij . r_ij) /
 * (rhobar_ij (|r_ij|^2 + eps h^2)) when v_ij . r_ij < 0, rhobar the mean
 * density; boundary particles join the density sum and the EOS, push on the
 * fluid and never move; the neighbour relation is |r_ij|^2 < (2h)^2, self
 * excluded (density adds the self term W(0) separately).
 *
 * Neighbour predicate, written so that a GPU kernel can take the identical
 * decision bit for bit:
 *   FP64: x_ij = r_i - r_j per axis (RN), d2 = fma(z,z,fma(y,y,x*x)),
 *         neighbour iff d2 < R2, R2 = (2h)*(2h) in double.
 *   FP32: per axis o = (float)(x - base(c)) with base(c) = dom_min + c*cs,
 *         x_ij = (o_i - (float)(c_j - c_i) * (float)cs) - o_j (two float
 *         RN operations, the product being exact for |c_j - c_i| <= 2),
 *         d2 = fmaf chain as above, neighbour iff d2 < Rf*Rf,
 *         Rf = (float)(2h).
 * Cell edge: cs >= 2h (Section 3.2.1: the 3^D adjacent cells) or, for a
 * finer grid, cs >= h with the 5^D cells around a particle's own.
 * Cell of a coordinate: the largest c with base(c) <= x (base computed in
 * double RN, no contraction); outside [0, ncell) is "out of domain".
 *
 * Build: -std=c11 -O2 -ffp-contract=off -fopenmp (no fused multiply-add
 * other than the explicit fma() calls, no reassociation).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    int dim;
    int ncell[3];
    double dom_min[3];
    double cs;
    double h;
    double dx;
    double mass;
    double rho0;
    double c0;
    double gamma;
    double alpha;
    double visc_eps;
    double dt;
    double g[3];
    int rho_ref_lattice; /* 1: rho_ref = m * lattice sum of W; 0: rho_ref = rho0 */
    int clamp_neg_p;     /* 1: p = max(p, 0) */
    int reaction_mode;   /* 1: accelerations on every particle, boundary included */
    int fp32_neighbours; /* 1: neighbour sets from the FP32 predicate */
    int adaptive_dt;     /* 1: step k > 0 of a call takes min(dt, cfl * dt_cfl of step k - 1) */
    double cfl;          /* safety factor of the adaptive step */
} orc_params;

typedef struct {
    int64_t n_pairs;   /* ordered pairs (i, j != i) within the support, last step */
    double vmax;       /* max |v| over fluid after the last step */
    double amax;       /* max |a| over fluid in the last step */
    double dt_cfl;     /* min(0.25 h/(c0 + vmax), 0.25 sqrt(h/amax)) */
    int out_of_domain; /* particles found outside the cell grid */
    double dt;         /* the step size of the last step */
    double time;       /* the sum of the step sizes of the call's steps */
} orc_diag;

/* ---------------------------------------------------------------------- */
/* Wendland kernel, Section 5.1.1.                                         */

double orc_alpha_D(int dim, double h)
{
    if (dim == 1) return 3.0 / (4.0 * h);
    if (dim == 2) return 7.0 / (4.0 * M_PI * h * h);
    return 21.0 / (16.0 * M_PI * h * h * h);
}

double orc_W(int dim, double h, double r)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return orc_alpha_D(dim, h) * t * t * t * t * (2.0 * q + 1.0);
}

/* dW/dr: d/dq [(1-q/2)^4 (2q+1)] = -2(1-q/2)^3(2q+1) + 2(1-q/2)^4
 *      = (1-q/2)^3 (-5q), and dq/dr = 1/h. */
double orc_dWdr(int dim, double h, double r)
{
    double q = r / h;
    if (q >= 2.0) return 0.0;
    double t = 1.0 - 0.5 * q;
    return -5.0 * orc_alpha_D(dim, h) / h * q * t * t * t;
}

/* rho_ref of the LATTICE reading: m * sum over all lattice vectors k of
 * W(|k| dx), self term included, i.e. the summation density of an interior
 * particle of the unperturbed lattice. */
double orc_rho_ref(const orc_params *p)
{
    if (!p->rho_ref_lattice) return p->rho0;
    double R = 2.0 * p->h;
    int K = (int)ceil(R / p->dx) + 1;
    double s = 0.0;
    if (p->dim == 2) {
        for (int b = -K; b <= K; ++b)
            for (int a = -K; a <= K; ++a) {
                double r = sqrt((double)(a * a + b * b)) * p->dx;
                if (r < R) s += orc_W(2, p->h, r);
            }
    } else {
        for (int c = -K; c <= K; ++c)
            for (int b = -K; b <= K; ++b)
                for (int a = -K; a <= K; ++a) {
                    double r = sqrt((double)(a * a + b * b + c * c)) * p->dx;
                    if (r < R) s += orc_W(3, p->h, r);
                }
    }
    return p->mass * s;
}

/* Tait equation of state with the negative-pressure clamp. */
double orc_pressure(const orc_params *p, double rho_ref, double rho)
{
    double B = p->c0 * p->c0 * p->rho0 / p->gamma;
    double pr = B * (pow(rho / rho_ref, p->gamma) - 1.0);
    if (p->clamp_neg_p && pr < 0.0) pr = 0.0;
    return pr;
}

/* ---------------------------------------------------------------------- */
/* Cell grid, Section 3.2.1.                                               */

static double cell_base(const orc_params *p, int k, long c)
{
    return p->dom_min[k] + (double)c * p->cs;
}

/* Cell index along axis k: the largest c with base(c) <= x.  Returns -1 if
 * x is NaN or outside [base(0), base(ncell)). */
static int cell_axis(const orc_params *p, int k, double x, long *out)
{
    long nc = p->ncell[k];
    if (!(x >= cell_base(p, k, 0)) || !(x < cell_base(p, k, nc))) {
        *out = -1;
        return -1;
    }
    double est = floor((x - p->dom_min[k]) / p->cs);
    long c = (long)(est < 0.0 ? 0.0 : (est > (double)(nc - 1) ? (double)(nc - 1) : est));
    while (c > 0 && cell_base(p, k, c) > x) --c;
    while (c + 1 < nc && cell_base(p, k, c + 1) <= x) ++c;
    *out = c;
    return 0;
}

static long n_cells(const orc_params *p)
{
    long nc = (long)p->ncell[0] * p->ncell[1];
    if (p->dim == 3) nc *= p->ncell[2];
    return nc;
}

/* Cell coordinates of particle i (r is row-major n x dim).  Returns 0 or -1. */
static int particle_cell(const orc_params *p, const double *ri, long cc[3])
{
    int bad = 0;
    cc[2] = 0;
    for (int k = 0; k < p->dim; ++k) bad |= cell_axis(p, k, ri[k], &cc[k]);
    return bad;
}

static long linear_cell(const orc_params *p, const long cc[3])
{
    return cc[0] + (long)p->ncell[0] * (cc[1] + (long)p->ncell[1] * cc[2]);
}

typedef struct {
    long ncells;
    uint32_t *start;  /* ncells + 1 */
    uint32_t *list;   /* particle indices, (cell, id) order */
    long *cc;         /* n x 3 cell coordinates */
    float *off;       /* n x 3 FP32 cell-relative offsets */
} cell_list;

static const uint32_t *g_sort_id;
static int cmp_by_id(const void *a, const void *b)
{
    uint32_t ia = g_sort_id[*(const uint32_t *)a], ib = g_sort_id[*(const uint32_t *)b];
    return (ia > ib) - (ia < ib);
}

static void free_cells(cell_list *cl)
{
    free(cl->start);
    free(cl->list);
    free(cl->cc);
    free(cl->off);
    memset(cl, 0, sizeof(*cl));
}

/* Counting sort by linear cell id, then ordering by persistent id inside
 * each cell.  Returns the number of particles outside the grid (they are not
 * listed; callers treat any as an error). */
static int build_cells(const orc_params *p, int n, const double *r, const uint32_t *id,
                       cell_list *cl)
{
    int D = p->dim, bad = 0;
    cl->ncells = n_cells(p);
    cl->start = (uint32_t *)calloc((size_t)cl->ncells + 1, sizeof(uint32_t));
    cl->list = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    cl->cc = (long *)malloc(sizeof(long) * 3 * (size_t)(n > 0 ? n : 1));
    cl->off = (float *)calloc(3 * (size_t)(n > 0 ? n : 1), sizeof(float));
    long *lin = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        long *c = &cl->cc[3 * i];
        if (particle_cell(p, &r[(size_t)i * D], c)) {
            lin[i] = -1;
            ++bad;
            continue;
        }
        lin[i] = linear_cell(p, c);
        for (int k = 0; k < D; ++k)
            cl->off[3 * i + k] = (float)(r[(size_t)i * D + k] - cell_base(p, k, c[k]));
        cl->start[lin[i] + 1]++;
    }
    for (long c = 0; c < cl->ncells; ++c) cl->start[c + 1] += cl->start[c];
    uint32_t *fill = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cl->ncells);
    memcpy(fill, cl->start, sizeof(uint32_t) * (size_t)cl->ncells);
    for (int i = 0; i < n; ++i)
        if (lin[i] >= 0) cl->list[fill[lin[i]]++] = (uint32_t)i;
    g_sort_id = id;
    for (long c = 0; c < cl->ncells; ++c) {
        uint32_t a = cl->start[c], b = cl->start[c + 1];
        if (b - a > 1) qsort(&cl->list[a], b - a, sizeof(uint32_t), cmp_by_id);
    }
    free(fill);
    free(lin);
    return bad;
}

/* ---------------------------------------------------------------------- */
/* Neighbour predicates.                                                   */

static int near_fp64(const orc_params *p, const double *ri, const double *rj)
{
    double R = 2.0 * p->h;
    double R2 = R * R;
    double x = ri[0] - rj[0];
    double y = ri[1] - rj[1];
    double d2 = fma(y, y, x * x);
    if (p->dim == 3) {
        double z = ri[2] - rj[2];
        d2 = fma(z, z, d2);
    }
    return d2 < R2;
}

static int near_fp32(const orc_params *p, const float *oi, const long *ci, const float *oj,
                     const long *cj)
{
    float csf = (float)p->cs;
    float Rf = (float)(2.0 * p->h);
    float R2f = Rf * Rf;
    float x[3] = {0.0f, 0.0f, 0.0f};
    for (int k = 0; k < p->dim; ++k) {
        float shift = (float)(cj[k] - ci[k]) * csf;
        float t = oi[k] - shift;
        x[k] = t - oj[k];
    }
    float d2 = x[0] * x[0];
    d2 = fmaf(x[1], x[1], d2);
    if (p->dim == 3) d2 = fmaf(x[2], x[2], d2);
    return d2 < R2f;
}

static int is_near(const orc_params *p, int fp32, const double *r, const cell_list *cl, int i,
                   int j)
{
    if (fp32) return near_fp32(p, &cl->off[3 * i], &cl->cc[3 * i], &cl->off[3 * j], &cl->cc[3 * j]);
    return near_fp64(p, &r[(size_t)i * p->dim], &r[(size_t)j * p->dim]);
}

/* Stencil radius in cells: the smallest K with K cs >= 2h, so that every
 * particle within the support radius 2h of i lies in one of the (2K+1)^D
 * cells around i's own.  Section 3.2.1 takes cells no smaller than the
 * radius (K = 1, the 3^D adjacent cells); a finer grid (cs >= h, K = 2) finds
 * the same neighbours through more, smaller cells. */
static int stencil_radius(const orc_params *p)
{
    return (int)ceil(2.0 * p->h / p->cs);
}

/* Visit the neighbours j != i of particle i through the (2K+1)^D cells
 * around its own.  Calls fn for each. */
typedef void (*visit_fn)(void *ctx, int i, int j);

static void for_neighbours(const orc_params *p, int fp32, const double *r, const cell_list *cl,
                           int i, visit_fn fn, void *ctx)
{
    const long *ci = &cl->cc[3 * i];
    const int K = stencil_radius(p);
    int zlo = (p->dim == 3) ? -K : 0, zhi = (p->dim == 3) ? K : 0;
    for (int dz = zlo; dz <= zhi; ++dz)
        for (int dy = -K; dy <= K; ++dy)
            for (int dxc = -K; dxc <= K; ++dxc) {
                long c[3] = {ci[0] + dxc, ci[1] + dy, ci[2] + dz};
                if (c[0] < 0 || c[0] >= p->ncell[0] || c[1] < 0 || c[1] >= p->ncell[1]) continue;
                if (p->dim == 3 && (c[2] < 0 || c[2] >= p->ncell[2])) continue;
                long lc = linear_cell(p, c);
                for (uint32_t k = cl->start[lc]; k < cl->start[lc + 1]; ++k) {
                    int j = (int)cl->list[k];
                    if (j == i) continue;
                    if (is_near(p, fp32, r, cl, i, j)) fn(ctx, i, j);
                }
            }
}

/* ---------------------------------------------------------------------- */
/* Exported: cell sort and neighbour lists (for the bit-exact checks).     */

/* Canonical (cell, id) order.  order[k] = input index of the k-th particle;
 * cell_start has ncells + 1 entries; cell_of[k] = linear cell of the k-th
 * sorted particle.  Returns the number of particles outside the grid. */
int orc_sort_cells(const orc_params *p, int n, const double *r, const uint32_t *id,
                   uint32_t *order, uint32_t *cell_start, uint32_t *cell_of)
{
    cell_list cl;
    int bad = build_cells(p, n, r, id, &cl);
    memcpy(cell_start, cl.start, sizeof(uint32_t) * ((size_t)cl.ncells + 1));
    int m = (int)cl.start[cl.ncells];
    for (int k = 0; k < m; ++k) {
        order[k] = cl.list[k];
        cell_of[k] = (uint32_t)linear_cell(p, &cl.cc[3 * cl.list[k]]);
    }
    free_cells(&cl);
    return bad;
}

/* Cell coordinates and FP32 offsets per particle (input order). */
int orc_cell_coords(const orc_params *p, int n, const double *r, int32_t *cc, float *off)
{
    int bad = 0;
    for (int i = 0; i < n; ++i) {
        long c[3];
        int b = particle_cell(p, &r[(size_t)i * p->dim], c);
        bad += b ? 1 : 0;
        for (int k = 0; k < 3; ++k) {
            cc[3 * i + k] = (int32_t)c[k];
            off[3 * i + k] = (!b && k < p->dim) ? (float)(r[(size_t)i * p->dim + k] - cell_base(p, k, c[k])) : 0.0f;
        }
    }
    return bad;
}

typedef struct {
    const uint32_t *id;
    uint32_t *dst;
    int64_t cnt;
} collect_ctx;

static void collect(void *vctx, int i, int j)
{
    (void)i;
    collect_ctx *c = (collect_ctx *)vctx;
    if (c->dst) c->dst[c->cnt] = c->id[j];
    c->cnt++;
}

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

/* Neighbour lists (persistent ids, ascending) of every particle, indexed by
 * input position.  method 0: brute force over all pairs; 1: cell list.
 * fp32 selects the predicate.  offs has n + 1 entries; nbr may be NULL to
 * count only.  Returns the total count, -1 if a particle is outside the grid,
 * -2 if cap is too small. */
int64_t orc_neighbours(const orc_params *p, int n, const double *r, const uint32_t *id, int method,
                       int fp32, int64_t *offs, uint32_t *nbr, int64_t cap)
{
    cell_list cl;
    int bad = build_cells(p, n, r, id, &cl);
    if (bad && (method == 1 || fp32)) {
        free_cells(&cl);
        return -1;
    }
    int64_t total = 0;
    offs[0] = 0;
    for (int i = 0; i < n; ++i) {
        collect_ctx c = {id, NULL, 0};
        uint32_t *dst = (nbr && total <= cap) ? nbr + total : NULL;
        if (method == 0) {
            for (int j = 0; j < n; ++j) {
                if (j == i) continue;
                if (is_near(p, fp32, r, &cl, i, j)) {
                    if (dst && total + c.cnt < cap) dst[c.cnt] = id[j];
                    c.cnt++;
                }
            }
        } else {
            collect_ctx cc2 = {id, NULL, 0};
            for_neighbours(p, fp32, r, &cl, i, collect, &cc2);
            c.cnt = cc2.cnt;
            if (dst && total + c.cnt <= cap) {
                collect_ctx cc3 = {id, dst, 0};
                for_neighbours(p, fp32, r, &cl, i, collect, &cc3);
            }
        }
        if (dst && total + c.cnt <= cap && c.cnt > 1) qsort(dst, (size_t)c.cnt, sizeof(uint32_t), cmp_u32);
        total += c.cnt;
        offs[i + 1] = total;
    }
    free_cells(&cl);
    if (nbr && total > cap) return -2;
    return total;
}

typedef struct {
    uint32_t *dst;
    int64_t cnt;
} idx_ctx;

static void collect_idx(void *vctx, int i, int j)
{
    (void)i;
    idx_ctx *c = (idx_ctx *)vctx;
    if (c->dst) c->dst[c->cnt] = (uint32_t)j;
    c->cnt++;
}

/* Neighbour lists as input indices (cell-list search, the predicate selected
 * by p->fp32_neighbours), CSR in offs (n + 1 entries).  nbr NULL: count only.
 * Returns the total, -1 if a particle is outside the grid, -2 if cap is
 * too small. */
int64_t orc_neighbours_idx(const orc_params *p, int n, const double *r, const uint32_t *id, int64_t *offs,
                           uint32_t *nbr, int64_t cap)
{
    cell_list cl;
    if (build_cells(p, n, r, id, &cl)) {
        free_cells(&cl);
        return -1;
    }
    int64_t total = 0;
    offs[0] = 0;
    for (int i = 0; i < n; ++i) {
        idx_ctx c = {NULL, 0};
        for_neighbours(p, p->fp32_neighbours, r, &cl, i, collect_idx, &c);
        if (nbr) {
            if (total + c.cnt > cap) {
                free_cells(&cl);
                return -2;
            }
            idx_ctx f = {nbr + total, 0};
            for_neighbours(p, p->fp32_neighbours, r, &cl, i, collect_idx, &f);
        }
        total += c.cnt;
        offs[i + 1] = total;
    }
    free_cells(&cl);
    return total;
}

/* ---------------------------------------------------------------------- */
/* The step, Section 5.1 / Example 1a with the readings above.             */

typedef struct {
    const orc_params *p;
    const double *r;
    double sumW;
    int64_t pairs;
} dens_ctx;

static void dens_visit(void *vctx, int i, int j)
{
    dens_ctx *c = (dens_ctx *)vctx;
    int D = c->p->dim;
    const double *ri = &c->r[(size_t)i * D], *rj = &c->r[(size_t)j * D];
    double d2 = 0.0;
    for (int k = 0; k < D; ++k) d2 += (ri[k] - rj[k]) * (ri[k] - rj[k]);
    c->sumW += orc_W(D, c->p->h, sqrt(d2));
    c->pairs++;
}

typedef struct {
    const orc_params *p;
    const double *r, *v, *rho, *pr;
    double a[3];
    double absum; /* sum over pairs of |term_ij| (conditioning of the sum) */
    double sens;  /* first-order change of |a_i| per unit relative density error */
} acc_ctx;

/* One pair term of the momentum equation (Eq. diffop1 form + viscosity):
 * -m (p_i/rho_i^2 + p_j/rho_j^2 + Pi_ij) grad_i W_ij. */
static void acc_visit(void *vctx, int i, int j)
{
    acc_ctx *c = (acc_ctx *)vctx;
    const orc_params *p = c->p;
    int D = p->dim;
    double rij[3] = {0, 0, 0}, vij[3] = {0, 0, 0};
    double r2 = 0.0, vr = 0.0;
    for (int k = 0; k < D; ++k) {
        rij[k] = c->r[(size_t)i * D + k] - c->r[(size_t)j * D + k];
        vij[k] = c->v[(size_t)i * D + k] - c->v[(size_t)j * D + k];
        r2 += rij[k] * rij[k];
        vr += vij[k] * rij[k];
    }
    double rr = sqrt(r2);
    if (rr <= 0.0) return; /* coincident particles: grad W = 0 */
    double dW = orc_dWdr(D, p->h, rr);
    double Pi = 0.0;
    if (vr < 0.0) {
        double rhobar = 0.5 * (c->rho[i] + c->rho[j]);
        Pi = -p->alpha * p->c0 * p->h * vr / (rhobar * (r2 + p->visc_eps * p->h * p->h));
    }
    double coef = p->mass * (c->pr[i] / (c->rho[i] * c->rho[i]) + c->pr[j] / (c->rho[j] * c->rho[j]) + Pi);
    for (int k = 0; k < D; ++k) c->a[k] -= coef * dW * rij[k] / rr;
    c->absum += fabs(coef * dW);
    /* dp/(drho/rho) = gamma (p + B) for the Tait law: the pressure error a
     * relative density error induces, propagated through this pair term */
    double B = p->c0 * p->c0 * p->rho0 / p->gamma;
    c->sens += p->mass * fabs(dW) *
               (p->gamma * (fabs(c->pr[i]) + B) / (c->rho[i] * c->rho[i]) +
                p->gamma * (fabs(c->pr[j]) + B) / (c->rho[j] * c->rho[j]));
}

/* Density (all particles) and pressure.  Returns the ordered pair count, or
 * -1 if a particle is outside the grid. */
static int64_t density_eos(const orc_params *p, int n, const double *r, const cell_list *cl,
                           double *rho, double *pr)
{
    int fp32 = p->fp32_neighbours;
    double rho_ref = orc_rho_ref(p);
    double W0 = orc_W(p->dim, p->h, 0.0);
    int64_t pairs = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : pairs)
    for (int i = 0; i < n; ++i) {
        dens_ctx c = {p, r, 0.0, 0};
        for_neighbours(p, fp32, r, cl, i, dens_visit, &c);
        rho[i] = p->mass * (W0 + c.sumW);
        pr[i] = orc_pressure(p, rho_ref, rho[i]);
        pairs += c.pairs;
    }
    return pairs;
}

static void accel(const orc_params *p, int n, const double *r, const double *v,
                  const uint8_t *kind, const cell_list *cl, const double *rho, const double *pr,
                  double *a, double *aabs, double *asens)
{
    int D = p->dim;
    int fp32 = p->fp32_neighbours;
#pragma omp parallel for schedule(dynamic, 256)
    for (int i = 0; i < n; ++i) {
        acc_ctx c = {p, r, v, rho, pr, {0, 0, 0}, 0.0, 0.0};
        int moving = (kind[i] == 0) || p->reaction_mode;
        if (moving) for_neighbours(p, fp32, r, cl, i, acc_visit, &c);
        if (aabs) {
            double g2 = 0.0;
            for (int k = 0; k < D; ++k) g2 += p->g[k] * p->g[k];
            aabs[i] = moving ? c.absum + (p->reaction_mode ? 0.0 : sqrt(g2)) : 0.0;
        }
        if (asens) asens[i] = moving ? c.sens : 0.0;
        for (int k = 0; k < D; ++k)
            a[(size_t)i * D + k] = moving ? (c.a[k] + (p->reaction_mode ? 0.0 : p->g[k])) : 0.0;
    }
}

/* Density and pressure of every particle at positions r. */
int64_t orc_density(const orc_params *p, int n, const double *r, const uint32_t *id, double *rho,
                    double *pr)
{
    cell_list cl;
    if (build_cells(p, n, r, id, &cl)) {
        free_cells(&cl);
        return -1;
    }
    int64_t pairs = density_eos(p, n, r, &cl, rho, pr);
    free_cells(&cl);
    return pairs;
}

/* Accelerations (fluid; every particle in reaction mode) from given rho, p.
 * aabs (optional): per particle, the sum over pairs of |term_ij| plus |g| --
 * the scale against which the rounding error of the sum is measured.
 * asens (optional): per particle, sum over pairs of m |W'| (gamma(|p_i|+B)/
 * rho_i^2 + gamma(|p_j|+B)/rho_j^2): the first-order change of a_i per unit
 * relative error of the densities (through the equation of state). */
int orc_accel(const orc_params *p, int n, const double *r, const double *v, const uint8_t *kind,
              const uint32_t *id, const double *rho, const double *pr, double *a, double *aabs,
              double *asens)
{
    cell_list cl;
    if (build_cells(p, n, r, id, &cl)) {
        free_cells(&cl);
        return -1;
    }
    accel(p, n, r, v, kind, &cl, rho, pr, a, aabs, asens);
    free_cells(&cl);
    return 0;
}

/* nsteps explicit steps in place on (r, v) (row-major n x dim).  Per step:
 * cell grid, density + EOS, accelerations, v += dt a, r += dt v (fluid
 * only).  The step size is p->dt, or with adaptive_dt the CFL bound of the
 * previous step scaled by cfl and capped by p->dt (the first step of the call
 * takes p->dt): dt_cfl = min(0.25 h/(c0 + vmax), 0.25 sqrt(h/amax)) with
 * vmax over the new velocities and amax over the accelerations of that
 * step.  rho, pr, a (optional) receive the last step's fields.  Returns 0,
 * or -1 if a particle left the grid (state left at the failing step). */
int orc_step(const orc_params *p, int n, double *r, double *v, const uint8_t *kind,
             const uint32_t *id, int nsteps, double *rho_out, double *pr_out, double *a_out,
             orc_diag *diag)
{
    int D = p->dim;
    size_t nn = (size_t)(n > 0 ? n : 1);
    double *rho = (double *)malloc(sizeof(double) * nn);
    double *pr = (double *)malloc(sizeof(double) * nn);
    double *a = (double *)malloc(sizeof(double) * nn * (size_t)D);
    int rc = 0;
    if (diag) memset(diag, 0, sizeof(*diag));
    double dt = p->dt, time = 0.0;
    for (int s = 0; s < nsteps; ++s) {
        cell_list cl;
        int bad = build_cells(p, n, r, id, &cl);
        if (bad) {
            if (diag) diag->out_of_domain = bad;
            free_cells(&cl);
            rc = -1;
            break;
        }
        int64_t pairs = density_eos(p, n, r, &cl, rho, pr);
        accel(p, n, r, v, kind, &cl, rho, pr, a, NULL, NULL);
        free_cells(&cl);
        double vmax = 0.0, amax = 0.0;
        for (int i = 0; i < n; ++i) {
            if (kind[i] != 0) continue;
            double v2 = 0.0, a2 = 0.0;
            for (int k = 0; k < D; ++k) {
                size_t q = (size_t)i * D + k;
                v[q] = v[q] + dt * a[q];
                r[q] = r[q] + dt * v[q];
                v2 += v[q] * v[q];
                a2 += a[q] * a[q];
            }
            if (sqrt(v2) > vmax) vmax = sqrt(v2);
            if (sqrt(a2) > amax) amax = sqrt(a2);
        }
        double t1 = 0.25 * p->h / (p->c0 + vmax);
        double t2 = amax > 0.0 ? 0.25 * sqrt(p->h / amax) : INFINITY;
        double dt_cfl = t1 < t2 ? t1 : t2;
        time += dt;
        if (diag) {
            diag->n_pairs = pairs;
            diag->vmax = vmax;
            diag->amax = amax;
            diag->dt_cfl = dt_cfl;
            diag->dt = dt;
            diag->time = time;
        }
        if (p->adaptive_dt) {
            double next = p->cfl * dt_cfl;
            dt = next < p->dt ? next : p->dt;
        }
    }
    if (rho_out) memcpy(rho_out, rho, sizeof(double) * (size_t)n);
    if (pr_out) memcpy(pr_out, pr, sizeof(double) * (size_t)n);
    if (a_out) memcpy(a_out, a, sizeof(double) * (size_t)n * (size_t)D);
    free(rho);
    free(pr);
    free(a);
    return rc;
}

/* Density, pressure, accelerations and their conditioning (as orc_accel's
 * aabs / asens) at m sampled particles (input indices idx), for inputs too
 * large to evaluate whole: the cell grid is built for all particles, the
 * densities only for the samples and their neighbours.  Outputs are compact
 * (entry k belongs to idx[k]); a is m x dim.  Returns 0 or -1. */
int orc_sampled_forces(const orc_params *p, int n, const double *r, const double *v, const uint8_t *kind,
                       const uint32_t *id, int m, const uint32_t *idx, double *rho_s, double *pr_s, double *a_s,
                       double *aabs_s, double *asens_s)
{
    cell_list cl;
    if (build_cells(p, n, r, id, &cl)) {
        free_cells(&cl);
        return -1;
    }
    const int D = p->dim;
    const int fp32 = p->fp32_neighbours;
    /* closure: the samples and their neighbours */
    unsigned char *need = (unsigned char *)calloc((size_t)(n > 0 ? n : 1), 1);
    for (int k = 0; k < m; ++k) {
        int i = (int)idx[k];
        need[i] = 1;
        idx_ctx c = {NULL, 0};
        for_neighbours(p, fp32, r, &cl, i, collect_idx, &c);
        uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(c.cnt > 0 ? c.cnt : 1));
        idx_ctx f = {tmp, 0};
        for_neighbours(p, fp32, r, &cl, i, collect_idx, &f);
        for (int64_t q = 0; q < f.cnt; ++q) need[tmp[q]] = 1;
        free(tmp);
    }
    double *rho = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    double *pr = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    const double rho_ref = orc_rho_ref(p);
    const double W0 = orc_W(D, p->h, 0.0);
#pragma omp parallel for schedule(dynamic, 256)
    for (int i = 0; i < n; ++i) {
        if (!need[i]) continue;
        dens_ctx c = {p, r, 0.0, 0};
        for_neighbours(p, fp32, r, &cl, i, dens_visit, &c);
        rho[i] = p->mass * (W0 + c.sumW);
        pr[i] = orc_pressure(p, rho_ref, rho[i]);
    }
    double g2 = 0.0;
    for (int k = 0; k < D; ++k) g2 += p->g[k] * p->g[k];
#pragma omp parallel for schedule(dynamic, 16)
    for (int k = 0; k < m; ++k) {
        int i = (int)idx[k];
        acc_ctx c = {p, r, v, rho, pr, {0, 0, 0}, 0.0, 0.0};
        int moving = (kind[i] == 0) || p->reaction_mode;
        if (moving) for_neighbours(p, fp32, r, &cl, i, acc_visit, &c);
        rho_s[k] = rho[i];
        pr_s[k] = pr[i];
        for (int d = 0; d < D; ++d)
            a_s[(size_t)k * D + d] = moving ? c.a[d] + (p->reaction_mode ? 0.0 : p->g[d]) : 0.0;
        if (aabs_s) aabs_s[k] = moving ? c.absum + (p->reaction_mode ? 0.0 : sqrt(g2)) : 0.0;
        if (asens_s) asens_s[k] = moving ? c.sens : 0.0;
    }
    free(need);
    free(rho);
    free(pr);
    free_cells(&cl);
    return 0;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}
