/*
 * sph_oracle_bc.h -- oracle-internal declarations shared by the oracle's C
 * files (test infrastructure only; nothing outside oracle/ includes this).
 * Parameters and neighbour images of the domain faces of Section 3.2.1, as
 * defined in sph_oracle_bc.c.
 */
#ifndef SPH_ORACLE_BC_H
#define SPH_ORACLE_BC_H

#include <stdint.h>

#define BC_CUTOFF 0
#define BC_SYMMETRIC 1
#define BC_PERIODIC 2

typedef struct {
    int dim;
    int ncell[3];
    double dom_min[3];
    double cs;
    double h;
    double mass;
    double rho0;
    double c;      /* speed of sound of the linear EOS */
    double visc;   /* viscosity coefficient (0.1 in Example 1a) */
    double dt;
    double g[3];
    int bc[3];     /* BC_CUTOFF, BC_SYMMETRIC or BC_PERIODIC per axis */
    int fp32;      /* 1: neighbour sets from the FP32 predicate */
} orc_bc_params;

/* One neighbour image of particle i: index j, image code, FP64 relative
 * position r_i - r_j^t, the image's velocity sign per axis (-1: mirrored),
 * and |r_i - r_j^t|^2. */
typedef struct {
    int j;
    int code;
    double rel[3];
    double vs[3];
    double d2;
} orc_image;

/* Neighbour images of every particle within 2h (the predicate of p), i
 * itself excluded, in cell-search order: CSR offsets offs[n + 1] and the
 * images in out[] (out may be NULL to count).  Returns the total, -1 if a
 * particle is outside the grid, -2 if cap is too small. */
int64_t orc_bc_images(const orc_bc_params *p, int n, const double *r, const uint32_t *id, int64_t *offs,
                      orc_image *out, int64_t cap);

#endif
