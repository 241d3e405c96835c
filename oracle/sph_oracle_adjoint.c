/*
 * sph_oracle_adjoint.c -- reverse mode (adjoint) of one oracle step, and a
 * complex-step forward step that serves as its independent check.
 *
 * TEST INFRASTRUCTURE ONLY (see sph_oracle.c).  Plain C, FP64.
 *
 * The step being differentiated is the oracle step of sph_oracle.c
 * (arXiv:1710.08259, Section 5.1 / Example 1a with the readings listed
 * there): summation density, Tait EOS with clamp, symmetric pressure term
 * (Eq. diffop1) with artificial viscosity, then v' = v + dt a, r' = r + dt v'
 * on fluid particles.  The neighbour sets are frozen at the step's input
 * positions; W, W' and W'' vanish at the support radius, so set changes
 * carry no derivative.
 *
 * Notation.  r_ij = r_i - r_j, d = |r_ij|, t = 1 - d/(2h), C = 5 alpha_D/h^2,
 * F_ij = m C t^3 (so m grad_i W_ij = -F_ij r_ij), P_i = p_i / rho_i^2,
 * s_ij = P_i + P_j + Pi_ij.  For fluid i: a_i = g + sum_j s_ij F_ij r_ij.
 * Adjoint of one unordered pair {i, j} with abar the acceleration adjoint
 * (zero on boundary particles) and dA = abar_i - abar_j:
 *   sigma = F (r_ij . dA)                 -> Pbar_i, Pbar_j, Pibar += sigma
 *   rbar_i += s [F dA + (r_ij . dA) F'(d) r_ij / d],  rbar_j -= the same
 *   Pi = alpha Pi1, Pi1 = -2 c0 h vr / ((rho_i + rho_j)(d^2 + eps h^2)) when
 *   vr = v_ij . r_ij < 0: its partials in vr, d^2, rho_i, rho_j and alpha.
 * Then rhobar_i += Pbar_i dP/drho(rho_i), and the density adjoint
 *   rbar_i += (rhobar_i + rhobar_j) m grad_i W_ij,  rbar_j -= the same.
 * The oracle evaluates each unordered pair once and scatters to both ends
 * (the GPU evaluates it as a gather from each end: a different order).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

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
    int rho_ref_lattice;
    int clamp_neg_p;
    int reaction_mode;
    int fp32_neighbours;
} orc_params;

/* from sph_oracle.c */
double orc_alpha_D(int dim, double h);
double orc_rho_ref(const orc_params *p);
int64_t orc_neighbours_idx(const orc_params *p, int n, const double *r, const uint32_t *id, int64_t *offs,
                           uint32_t *nbr, int64_t cap);

/* Neighbour lists as input indices (CSR), cell-list search, self excluded. */
static int64_t neighbour_index_lists(const orc_params *p, int n, const double *r, const uint32_t *id,
                                     int64_t **offs, uint32_t **nbr)
{
    *offs = (int64_t *)malloc(sizeof(int64_t) * ((size_t)n + 1));
    int64_t tot = orc_neighbours_idx(p, n, r, id, *offs, NULL, 0);
    if (tot < 0) {
        free(*offs);
        *offs = NULL;
        return tot;
    }
    *nbr = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(tot > 0 ? tot : 1));
    orc_neighbours_idx(p, n, r, id, *offs, *nbr, tot);
    return tot;
}

/* ------------------------------------------------------------------------ */
/* Reverse step.                                                             */

/* Inputs: the state (r, v) at step n (row-major n x dim), kind, id and the
 * adjoint (rbar1, vbar1) of the state at step n+1 (same particle order: the
 * oracle never reorders).  Outputs the adjoint (rbar0, vbar0) of the state at
 * step n and adds dL/dalpha through this step to *alpha_bar.  Boundary
 * particles do not move: their outputs pass their inputs through plus the
 * pair contributions (which a caller may ignore).  Returns 0, or -1 if a
 * particle lies outside the grid. */
static int step_adjoint(const orc_params *p, int n, const double *r, const double *v, const uint8_t *kind,
                        const uint32_t *id, const uint8_t *clamp_in, const double *rbar1, const double *vbar1,
                        double *rbar0, double *vbar0, double *alpha_bar);

int orc_step_adjoint(const orc_params *p, int n, const double *r, const double *v, const uint8_t *kind,
                     const uint32_t *id, const double *rbar1, const double *vbar1, double *rbar0,
                     double *vbar0, double *alpha_bar)
{
    return step_adjoint(p, n, r, v, kind, id, NULL, rbar1, vbar1, rbar0, vbar0, alpha_bar);
}

/* The same reverse step with the pressure clamp's decisions given per
 * particle (clamp_in[i] = 1: p_i was clamped to 0 in the forward step being
 * differentiated, so p_i = 0 and dp_i/drho_i = 0), for differentiating a
 * trajectory that another computation produced (its own rounding decided on
 * which side of the kink p = 0 each particle lay).  clamp_in NULL: the
 * decisions of this step's own densities, as orc_step_adjoint. */
int orc_step_adjoint_clamped(const orc_params *p, int n, const double *r, const double *v, const uint8_t *kind,
                             const uint32_t *id, const uint8_t *clamp_in, const double *rbar1,
                             const double *vbar1, double *rbar0, double *vbar0, double *alpha_bar)
{
    return step_adjoint(p, n, r, v, kind, id, clamp_in, rbar1, vbar1, rbar0, vbar0, alpha_bar);
}

static int step_adjoint(const orc_params *p, int n, const double *r, const double *v, const uint8_t *kind,
                        const uint32_t *id, const uint8_t *clamp_in, const double *rbar1, const double *vbar1,
                        double *rbar0, double *vbar0, double *alpha_bar)
{
    const int D = p->dim;
    int64_t *offs = NULL;
    uint32_t *nbr = NULL;
    if (neighbour_index_lists(p, n, r, id, &offs, &nbr) < 0) return -1;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    double *rho = (double *)calloc(nn, sizeof(double));
    double *pr = (double *)calloc(nn, sizeof(double));
    double *P = (double *)calloc(nn, sizeof(double));
    double *dPdrho = (double *)calloc(nn, sizeof(double));
    double *Pbar = (double *)calloc(nn, sizeof(double));
    double *rhobar = (double *)calloc(nn, sizeof(double));
    double *abar = (double *)calloc(nn * 3, sizeof(double));
    const double h = p->h, m = p->mass;
    const double aD = orc_alpha_D(D, h);
    const double C = 5.0 * aD / (h * h);
    const double B = p->c0 * p->c0 * p->rho0 / p->gamma;
    const double rho_ref = orc_rho_ref(p);
    const double eh2 = p->visc_eps * h * h;

    /* forward quantities: density (self term included) and EOS */
    for (int i = 0; i < n; ++i) {
        double s = 1.0; /* w(0) */
        for (int64_t q = offs[i]; q < offs[i + 1]; ++q) {
            int j = (int)nbr[q];
            double d2 = 0.0;
            for (int k = 0; k < D; ++k) d2 += (r[i * D + k] - r[j * D + k]) * (r[i * D + k] - r[j * D + k]);
            double t = 1.0 - 0.5 * sqrt(d2) / h;
            s += t * t * t * t * (2.0 * sqrt(d2) / h + 1.0);
        }
        rho[i] = m * aD * s;
        double x = rho[i] / rho_ref;
        double praw = B * (pow(x, p->gamma) - 1.0);
        int clamped = clamp_in ? (p->clamp_neg_p && clamp_in[i]) : (p->clamp_neg_p && praw < 0.0);
        pr[i] = clamped ? 0.0 : praw;
        P[i] = pr[i] / (rho[i] * rho[i]);
        double dp = clamped ? 0.0 : B * p->gamma * pow(x, p->gamma - 1.0) / rho_ref;
        dPdrho[i] = dp / (rho[i] * rho[i]) - 2.0 * pr[i] / (rho[i] * rho[i] * rho[i]);
    }
    /* integration: r' = r + dt v', v' = v + dt a */
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < D; ++k) {
            size_t q = (size_t)i * D + k;
            if (kind[i] == 0) {
                double vt = vbar1[q] + p->dt * rbar1[q];
                vbar0[q] = vt;
                abar[(size_t)i * 3 + k] = p->dt * vt;
            } else {
                vbar0[q] = vbar1[q];
            }
            rbar0[q] = rbar1[q];
        }
    /* force terms, each unordered pair once */
    double ab = 0.0;
    for (int i = 0; i < n; ++i) {
        for (int64_t q = offs[i]; q < offs[i + 1]; ++q) {
            int j = (int)nbr[q];
            if (j <= i) continue;
            if (kind[i] != 0 && kind[j] != 0) continue; /* no force on either end */
            double rij[3] = {0, 0, 0}, vij[3] = {0, 0, 0}, dA[3] = {0, 0, 0};
            double d2 = 0.0, vr = 0.0, rdA = 0.0;
            for (int k = 0; k < D; ++k) {
                rij[k] = r[i * D + k] - r[j * D + k];
                vij[k] = v[i * D + k] - v[j * D + k];
                dA[k] = abar[(size_t)i * 3 + k] - abar[(size_t)j * 3 + k];
                d2 += rij[k] * rij[k];
                vr += vij[k] * rij[k];
                rdA += rij[k] * dA[k];
            }
            double d = sqrt(d2);
            double t = 1.0 - 0.5 * d / h;
            double F = m * C * t * t * t;
            double Fp = -1.5 * m * C * t * t / h; /* dF/dd */
            double Pi1 = 0.0, Pi = 0.0;
            if (vr < 0.0) {
                Pi1 = -2.0 * p->c0 * h * vr / ((rho[i] + rho[j]) * (d2 + eh2));
                Pi = p->alpha * Pi1;
            }
            double s = P[i] + P[j] + Pi;
            double sigma = F * rdA;
            Pbar[i] += sigma;
            Pbar[j] += sigma;
            for (int k = 0; k < D; ++k) {
                double gk = s * (F * dA[k] + (d > 0.0 ? rdA * Fp * rij[k] / d : 0.0));
                rbar0[i * D + k] += gk;
                rbar0[j * D + k] -= gk;
            }
            if (vr < 0.0) {
                double den = (rho[i] + rho[j]) * (d2 + eh2);
                double Pi_vr = -2.0 * p->alpha * p->c0 * h / den;
                double Pi_d2 = -Pi / (d2 + eh2);
                double Pi_rho = -Pi / (rho[i] + rho[j]);
                for (int k = 0; k < D; ++k) {
                    double gr = sigma * (Pi_vr * vij[k] + 2.0 * Pi_d2 * rij[k]);
                    rbar0[i * D + k] += gr;
                    rbar0[j * D + k] -= gr;
                    double gv = sigma * Pi_vr * rij[k];
                    vbar0[i * D + k] += gv;
                    vbar0[j * D + k] -= gv;
                }
                rhobar[i] += sigma * Pi_rho;
                rhobar[j] += sigma * Pi_rho;
                ab += sigma * Pi1;
            }
        }
    }
    for (int i = 0; i < n; ++i) rhobar[i] += Pbar[i] * dPdrho[i];
    /* density: rho_i = m sum_j W_ij (self included) */
    for (int i = 0; i < n; ++i) {
        for (int64_t q = offs[i]; q < offs[i + 1]; ++q) {
            int j = (int)nbr[q];
            if (j <= i) continue;
            double rij[3] = {0, 0, 0}, d2 = 0.0;
            for (int k = 0; k < D; ++k) {
                rij[k] = r[i * D + k] - r[j * D + k];
                d2 += rij[k] * rij[k];
            }
            double t = 1.0 - 0.5 * sqrt(d2) / h;
            double F = m * C * t * t * t; /* m grad_i W_ij = -F r_ij */
            for (int k = 0; k < D; ++k) {
                double gk = -(rhobar[i] + rhobar[j]) * F * rij[k];
                rbar0[i * D + k] += gk;
                rbar0[j * D + k] -= gk;
            }
        }
    }
    if (alpha_bar) *alpha_bar += ab;
    free(offs);
    free(nbr);
    free(rho);
    free(pr);
    free(P);
    free(dPdrho);
    free(Pbar);
    free(rhobar);
    free(abar);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Complex-step forward step: the same step evaluated on complex inputs      */
/* r + i hcs dr, v + i hcs dv, alpha + i hcs dalpha (neighbour sets and      */
/* branches from the real parts).  Re(output) is the step; Im(output)/hcs is */
/* the directional derivative J (dr, dv, dalpha) to rounding accuracy.       */

typedef double complex cplx;

int orc_step_cs(const orc_params *p, int n, const double *r, const double *v, const uint8_t *kind,
                const uint32_t *id, const double *dr, const double *dv, double dalpha, double hcs,
                double *r_out, double *v_out, double *dr_out, double *dv_out)
{
    const int D = p->dim;
    int64_t *offs = NULL;
    uint32_t *nbr = NULL;
    if (neighbour_index_lists(p, n, r, id, &offs, &nbr) < 0) return -1;
    const size_t nn = (size_t)(n > 0 ? n : 1);
    cplx *rc = (cplx *)malloc(sizeof(cplx) * nn * D);
    cplx *vc = (cplx *)malloc(sizeof(cplx) * nn * D);
    cplx *rho = (cplx *)malloc(sizeof(cplx) * nn);
    cplx *pr = (cplx *)malloc(sizeof(cplx) * nn);
    for (size_t q = 0; q < (size_t)n * D; ++q) {
        rc[q] = r[q] + I * hcs * dr[q];
        vc[q] = v[q] + I * hcs * dv[q];
    }
    const double h = p->h, m = p->mass;
    const double aD = orc_alpha_D(D, h);
    const double B = p->c0 * p->c0 * p->rho0 / p->gamma;
    const double rho_ref = orc_rho_ref(p);
    const cplx alpha = p->alpha + I * hcs * dalpha;
    for (int i = 0; i < n; ++i) {
        cplx s = aD; /* W(0) */
        for (int64_t q = offs[i]; q < offs[i + 1]; ++q) {
            int j = (int)nbr[q];
            cplx d2 = 0.0;
            for (int k = 0; k < D; ++k) d2 += (rc[i * D + k] - rc[j * D + k]) * (rc[i * D + k] - rc[j * D + k]);
            cplx qq = csqrt(d2) / h;
            cplx t = 1.0 - 0.5 * qq;
            s += aD * t * t * t * t * (2.0 * qq + 1.0);
        }
        rho[i] = m * s;
        cplx x = rho[i] / rho_ref;
        cplx xg = 1.0;
        for (int e = 0; e < (int)p->gamma; ++e) xg *= x; /* integer gamma */
        pr[i] = B * (xg - 1.0);
        if (p->clamp_neg_p && creal(pr[i]) < 0.0) pr[i] = 0.0;
    }
    const double C = 5.0 * aD / (h * h);
    for (int i = 0; i < n; ++i) {
        for (int k = 0; k < D; ++k) {
            r_out[i * D + k] = r[i * D + k];
            v_out[i * D + k] = v[i * D + k];
            dr_out[i * D + k] = dr[i * D + k];
            dv_out[i * D + k] = dv[i * D + k];
        }
        if (kind[i] != 0) continue;
        cplx a[3] = {p->g[0], p->g[1], p->g[2]};
        for (int64_t q = offs[i]; q < offs[i + 1]; ++q) {
            int j = (int)nbr[q];
            cplx rij[3] = {0, 0, 0}, d2 = 0.0, vr = 0.0;
            for (int k = 0; k < D; ++k) {
                rij[k] = rc[i * D + k] - rc[j * D + k];
                d2 += rij[k] * rij[k];
                vr += (vc[i * D + k] - vc[j * D + k]) * rij[k];
            }
            cplx t = 1.0 - 0.5 * csqrt(d2) / h;
            cplx F = m * C * t * t * t;
            cplx Pi = 0.0;
            if (creal(vr) < 0.0)
                Pi = -2.0 * alpha * p->c0 * h * vr / ((rho[i] + rho[j]) * (d2 + p->visc_eps * h * h));
            cplx s = pr[i] / (rho[i] * rho[i]) + pr[j] / (rho[j] * rho[j]) + Pi;
            for (int k = 0; k < D; ++k) a[k] += s * F * rij[k];
        }
        for (int k = 0; k < D; ++k) {
            cplx vn = vc[i * D + k] + p->dt * a[k];
            cplx rn = rc[i * D + k] + p->dt * vn;
            v_out[i * D + k] = creal(vn);
            r_out[i * D + k] = creal(rn);
            dv_out[i * D + k] = cimag(vn) / hcs;
            dr_out[i * D + k] = cimag(rn) / hcs;
        }
    }
    free(offs);
    free(nbr);
    free(rc);
    free(vc);
    free(rho);
    free(pr);
    return 0;
}
