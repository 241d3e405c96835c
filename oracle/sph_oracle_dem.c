/*
 * sph_oracle_dem.c -- plain CPU reference ("oracle") of the DEM particle
 * damper of Example 2 (Section 5.2): the Hertzian contact law with damping
 * and Coulomb friction of Eq. DEM_force and the effective quantities of
 * Eq. effective_quantities between spheres, the tank walls as symmetric
 * domain faces (Section 3.2.1), and the tank oscillator of Eq. tank_ode
 * driven by the wall forces of Eq. boundary_force.  FP64 arithmetic; the
 * neighbour candidates from the FP64 or the FP32 predicate.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load this library.  It shares no source,
 * header, table or helper with the CUDA library.
 *
 * One step from (r, v) and the tank state (Z, Zdot), for every particle i
 * and every neighbour image (j, t) within 2h (h = the largest radius;
 * images of sph_oracle_bc.c) whose overlap delta = R_i + R_j - |r_ij| is
 * positive, with r_ij = r_i - r_j^t, n = r_ij / |r_ij| and v_ij = v_i -
 * v_j^t:
 *   R' = R_i R_j / (R_i + R_j), m' = m_i m_j / (m_i + m_j),
 *   E' = E_i E_j / (E_j (1 - nu_i^2) + E_i (1 - nu_j^2))   (E, nu shared here)
 *   k  = 4/3 sqrt(R') E',  c = sqrt(m' k) / 8
 *   f_n = k delta^(3/2) + c delta^(1/4) ddelta,  ddelta = -(v_ij . n)
 *   v_t = -v_ij + (v_ij . n) n,  f_t = c_f |f_n| v_t / |v_t|  (0 without sliding:
 *   |v_t| <= 1e-5 |v_ij|)
 *   F_i += f_n n + f_t;  an image reflected in a symmetric face (a wall)
 *   adds the same to F^b_i (a periodic image is a neighbour, not a wall).
 * Then F = sum_i F^b_i, Zddot = (-S Z - F . e_z) / M (the tank axis z),
 *   a_i = F_i / m_i + g - Zddot e_z,
 *   v_i += dt a_i, r_i += dt v_i (kind 0 only); Zdot += dt Zddot, Z += dt Zdot.
 *
 * Readings of the paper taken here: the printed normal n_ji is garbled
 * ("r_j - r_j"); the normal force is taken repulsive (pushing i away from
 * j) with the printed magnitude, ddelta the rate at which the overlap grows;
 * the friction acts along the printed v^t (the tangential velocity of j
 * relative to i); its direction is undefined without sliding, and a sliding
 * speed below 1e-5 of the relative speed counts as none (rounding would
 * otherwise give a head-on impact, or a sphere against its own wall image,
 * a full Coulomb force in a random direction); angular velocities are neglected
 * (as the paper states); the tank walls are symmetric faces, so a particle
 * meets the mirror image of itself and of its neighbours with the same law
 * (as the paper states), and F^b_i is the force from those images; the
 * particles move in the tank's frame and feel g - Zddot e_z (the paper's
 * "time-dependent acceleration field superposed with the gravitational
 * acceleration"; its printed particle equation lists g only); the forces of
 * step n use the state of step n, Zddot of step n uses F of step n.
 *
 * Build: -std=c11 -O2 -ffp-contract=off -fopenmp.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "sph_oracle_bc.h"

/* Sliding threshold: |v_t| <= kSlide |v_ij| counts as no sliding. */
static const double kSlide = 1e-5;

typedef struct {
    int dim;
    int ncell[3];
    double dom_min[3];
    double cs;
    double h;        /* largest radius: candidates within 2h */
    double E;        /* Young modulus */
    double nu;       /* Poisson ratio */
    double cf;       /* Coulomb friction coefficient */
    double dt;
    double g[3];
    int bc[3];
    int fp32;
    double tank_M;   /* tank mass; <= 0: no tank (Zddot = 0) */
    double tank_S;   /* spring stiffness */
} orc_dem_params;

typedef struct {
    int64_t n_contacts;  /* contacts (i, image) with positive overlap, last step */
    double vmax, amax;   /* over moving particles, last step */
    double Fb[3];        /* wall force on the particles, last step */
    double Zddot;        /* tank acceleration, last step */
    int out_of_domain;
} orc_dem_diag;

static orc_bc_params to_bc(const orc_dem_params *p)
{
    orc_bc_params q;
    memset(&q, 0, sizeof(q));
    q.dim = p->dim;
    for (int k = 0; k < 3; ++k) {
        q.ncell[k] = p->ncell[k];
        q.dom_min[k] = p->dom_min[k];
        q.bc[k] = p->bc[k];
    }
    q.cs = p->cs;
    q.h = p->h;
    q.fp32 = p->fp32;
    return q;
}

/* Contact forces of every particle: F (n x dim) and the F^b sum.  With
 * Fbound (optional), per particle a bound on the change of F_i when every
 * length the contact law sees carries an absolute rounding error up to
 * Delta = 4 eps max(cs, R_i + R_j) and every other operation a relative
 * error eps: per contact (and per near-contact, -Delta < delta <= 0, whose
 * sign rounding may flip) (1 + c_f) times
 *   1.5 k delta^(1/2) Delta                      (elastic term, Lipschitz)
 * + c |ddelta| min(Delta^(1/4), delta^(-3/4) Delta / 4)
 *                                                (damping: delta^(1/4) is only
 *                                                 Hoelder-continuous at 0)
 * + c delta^(1/4) eps (|v_i| + |v_j|) + 4 eps |f_n|,
 * plus c_f |f_n| min(2, 4 eps (|v_i| + |v_j|) / |v_t|) for the turn of the
 * friction direction.  Returns the contact count or -1. */
static int64_t dem_forces(const orc_dem_params *p, int n, const double *r, const double *v, const double *R,
                          const double *m, const uint32_t *id, double eps, double *F, double Fb[3],
                          double *Fbound)
{
    const int D = p->dim;
    orc_bc_params q = to_bc(p);
    int64_t *offs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t tot = orc_bc_images(&q, n, r, id, offs, NULL, 0);
    if (tot < 0) {
        free(offs);
        return -1;
    }
    orc_image *im = (orc_image *)malloc(sizeof(orc_image) * (size_t)(tot > 0 ? tot : 1));
    orc_bc_images(&q, n, r, id, offs, im, tot);
    const double Ep = p->E * p->E / (p->E * (1.0 - p->nu * p->nu) + p->E * (1.0 - p->nu * p->nu));
    int64_t contacts = 0;
    double fb[3] = {0, 0, 0};
    for (int i = 0; i < n; ++i) {
        double Fi[3] = {0, 0, 0}, fa = 0.0;
        const double *vi = &v[(size_t)i * D];
        for (int64_t s = offs[i]; s < offs[i + 1]; ++s) {
            const orc_image *x = &im[s];
            const int j = x->j;
            const double d = sqrt(x->d2);
            const double delta = R[i] + R[j] - d;
            const double Dl = 4.0 * eps * fmax(p->cs, R[i] + R[j]);
            const double *vj = &v[(size_t)j * D];
            if (!(delta > 0.0) || !(d > 0.0)) {
                if (Fbound && d > 0.0 && delta > -Dl) {
                    /* a near-contact: the rounded overlap may be positive */
                    const double Rp = R[i] * R[j] / (R[i] + R[j]);
                    const double mp = m[i] * m[j] / (m[i] + m[j]);
                    const double kh = 4.0 / 3.0 * sqrt(Rp) * Ep;
                    const double ch = sqrt(mp * kh) / 8.0;
                    double dv2 = 0.0;
                    for (int k = 0; k < D; ++k) dv2 += (vi[k] - x->vs[k] * vj[k]) * (vi[k] - x->vs[k] * vj[k]);
                    fa += (1.0 + p->cf) * (kh * Dl * sqrt(Dl) + ch * sqrt(dv2) * sqrt(sqrt(Dl)));
                }
                continue;
            }
            ++contacts;
            double nrm[3] = {0, 0, 0}, vij[3] = {0, 0, 0};
            double vn = 0.0;
            for (int k = 0; k < D; ++k) {
                nrm[k] = x->rel[k] / d;
                vij[k] = vi[k] - x->vs[k] * vj[k];
                vn += vij[k] * nrm[k];
            }
            const double Rp = R[i] * R[j] / (R[i] + R[j]);
            const double mp = m[i] * m[j] / (m[i] + m[j]);
            const double kh = 4.0 / 3.0 * sqrt(Rp) * Ep;
            const double ch = sqrt(mp * kh) / 8.0;
            const double fn = kh * delta * sqrt(delta) + ch * sqrt(sqrt(delta)) * (-vn);
            double vt[3] = {0, 0, 0}, vt2 = 0.0;
            for (int k = 0; k < D; ++k) {
                vt[k] = -vij[k] + vn * nrm[k];
                vt2 += vt[k] * vt[k];
            }
            /* the direction v_t/|v_t| is undefined without sliding: a sliding
             * speed below kSlide of the relative speed counts as none */
            double vij2 = 0.0;
            for (int k = 0; k < D; ++k) vij2 += vij[k] * vij[k];
            const int slides = vt2 > kSlide * kSlide * vij2;
            const double ft = slides ? p->cf * fabs(fn) / sqrt(vt2) : 0.0;
            for (int k = 0; k < D; ++k) {
                const double f = fn * nrm[k] + ft * vt[k];
                Fi[k] += f;
                if (x->vs[0] < 0.0 || x->vs[1] < 0.0 || x->vs[2] < 0.0) fb[k] += f;
            }
            if (Fbound) {
                double vv = 0.0, ww = 0.0;
                for (int k = 0; k < D; ++k) {
                    vv += vi[k] * vi[k];
                    ww += vj[k] * vj[k];
                }
                const double hold = fmin(sqrt(sqrt(Dl)), 0.25 * Dl / (delta * sqrt(sqrt(delta))));
                fa += (1.0 + p->cf) * (1.5 * kh * sqrt(delta) * Dl + ch * fabs(vn) * hold +
                                       ch * sqrt(sqrt(delta)) * eps * (sqrt(vv) + sqrt(ww)) + 4.0 * eps * fabs(fn));
                /* the friction direction v_t/|v_t| turns by ~eps |v| / |v_t|;
                 * near the sliding threshold rounding may switch it on or off */
                const double turn = vt2 > 4.0 * kSlide * kSlide * vij2
                                        ? 4.0 * eps * (sqrt(vv) + sqrt(ww)) / sqrt(vt2)
                                        : 2.0;
                fa += p->cf * fabs(fn) * fmin(2.0, turn);
            }
        }
        for (int k = 0; k < D; ++k) F[(size_t)i * D + k] = Fi[k];
        if (Fbound) Fbound[i] = fa;
    }
    for (int k = 0; k < 3; ++k) Fb[k] = fb[k];
    free(im);
    free(offs);
    return contacts;
}

/* Contact forces at (r, v) without integration (F n x dim, Fb[3], the
 * rounding bound Fbound for relative precision eps, optional). */
int64_t orc_dem_forces(const orc_dem_params *p, int n, const double *r, const double *v, const double *R,
                       const double *m, const uint32_t *id, double eps, double *F, double *Fb, double *Fbound)
{
    return dem_forces(p, n, r, v, R, m, id, eps, F, Fb, Fbound);
}

/* nsteps steps in place on (r, v) (row-major n x dim, input order) and
 * tank[2] = (Z, Zdot).  F_out (optional, n x dim): the last step's contact
 * forces.  Returns 0, or -1 if a particle is outside the grid (the state
 * stops at that step). */
int orc_dem_step(const orc_dem_params *p, int n, double *r, double *v, const double *R, const double *m,
                 const uint8_t *kind, const uint32_t *id, int nsteps, double *tank, double *F_out,
                 orc_dem_diag *diag)
{
    const int D = p->dim;
    const int ax = D - 1;
    double *F = (double *)calloc((size_t)(n > 0 ? n : 1) * (size_t)D, sizeof(double));
    int rc = 0;
    if (diag) memset(diag, 0, sizeof(*diag));
    for (int s = 0; s < nsteps; ++s) {
        double Fb[3];
        int64_t c = dem_forces(p, n, r, v, R, m, id, 0.0, F, Fb, NULL);
        if (c < 0) {
            if (diag) diag->out_of_domain = 1;
            rc = -1;
            break;
        }
        double Zdd = 0.0;
        if (p->tank_M > 0.0) Zdd = (-p->tank_S * tank[0] - Fb[ax]) / p->tank_M;
        double vmax = 0.0, amax = 0.0;
        for (int i = 0; i < n; ++i) {
            if (kind[i] != 0) continue;
            double v2 = 0.0, a2 = 0.0;
            for (int k = 0; k < D; ++k) {
                size_t q = (size_t)i * D + k;
                double a = F[q] / m[i] + p->g[k] - (k == ax ? Zdd : 0.0);
                v[q] = v[q] + p->dt * a;
                r[q] = r[q] + p->dt * v[q];
                v2 += v[q] * v[q];
                a2 += a * a;
            }
            if (sqrt(v2) > vmax) vmax = sqrt(v2);
            if (sqrt(a2) > amax) amax = sqrt(a2);
        }
        tank[1] = tank[1] + p->dt * Zdd;
        tank[0] = tank[0] + p->dt * tank[1];
        if (diag) {
            diag->n_contacts = c;
            diag->vmax = vmax;
            diag->amax = amax;
            for (int k = 0; k < 3; ++k) diag->Fb[k] = Fb[k];
            diag->Zddot = Zdd;
        }
    }
    if (F_out) memcpy(F_out, F, sizeof(double) * (size_t)n * (size_t)D);
    free(F);
    return rc;
}
