/*
 * sph.h -- C ABI of the GB300 WCSPH step library (libsph_gb300.so).
 *
 * The library advances a particle system by explicit weakly-compressible
 * SPH time steps: the interaction-law form of arXiv:1710.08259 (Nauticle),
 * Section 2.1 (fields on particles, pair sums over neighbours within an
 * influence radius, particle-wise updates), with the SPH operators of
 * Section 5.1 and the dam-break model of Example 1a (Section 5.1.1).
 *
 * Conventions for every call:
 *   - All particle arrays are DEVICE pointers owned by the caller, laid out
 *     as structure-of-arrays (one contiguous array per component).
 *   - Positions are always double.  Velocity, density and pressure arrays
 *     are float for SPH_PREC_F32 contexts and double for SPH_PREC_F64.
 *   - Every call that takes a stream enqueues work on that stream and
 *     returns without synchronising, unless stated otherwise.  A NULL stream
 *     is the legacy default stream.  Calls on one context must not overlap
 *     on the GPU (they share the context's workspace).
 *   - Return value: SPH_OK (0) or a negative SPH_ERR_* code; the message is
 *     available from sph_last_error().  Host-side argument errors leave the
 *     state untouched.  Errors detected on the device (a particle outside
 *     the domain, a non-finite value, ...) are recorded as bits of the
 *     context's device status word; read them with sph_get_status().
 *   - No call other than sph_create / sph_batch_create allocates device
 *     buffers, so the stepping calls can be captured in a CUDA graph (a
 *     multi-step sph_step records its own step graph on first use, see
 *     below; it does not while its stream is being captured).
 *   - After any call that takes an sph_state, the caller's arrays hold the
 *     particles in the canonical order: by linear cell id (x fastest, then
 *     y, then z) and by persistent id inside a cell.  The `id` array says
 *     which particle is where.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t), opaque here so that the header needs no
 * CUDA include. */
typedef struct CUstream_st *sph_stream_t;

/* Return codes. */
#define SPH_OK 0
#define SPH_ERR_INVALID (-1)  /* bad argument or parameter */
#define SPH_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define SPH_ERR_CAPACITY (-3) /* more particles than the context was created for */
#define SPH_ERR_STATUS (-4)   /* a device status bit is set (see sph_get_status) */

/* Device status bits (sph_get_status). */
#define SPH_STATUS_OUT_OF_DOMAIN 1u   /* a particle lies outside the cell grid (Section 3.2.1) */
#define SPH_STATUS_CELL_OVERFLOW 2u   /* a cell holds more than SPH_MAX_CELL particles */
#define SPH_STATUS_NAN 4u             /* a non-finite position, velocity or acceleration */
#define SPH_STATUS_CFL 8u             /* dt exceeded the CFL bound of the step */
#define SPH_STATUS_BARRIER_TIMEOUT 16u /* a device-wide barrier gave up waiting */
#define SPH_STATUS_DUPLICATE_ID 32u   /* two particles share a persistent id */
#define SPH_STATUS_BOUNDS 64u         /* bounds-checked builds (-DSPH_CHECK) only: an index that would
                                         leave its buffer was caught and the access skipped */

/* Largest cell population that is still ordered canonically; larger cells
 * (a blown-up simulation) keep an arbitrary order and raise CELL_OVERFLOW. */
#define SPH_MAX_CELL 4096

/* Arithmetic of the pair sums. */
#define SPH_PREC_F64 0 /* everything in double */
#define SPH_PREC_F32 1 /* pair sums in float from cell-relative float offsets,
                          Kahan-compensated density; positions, the cell hash
                          and the CFL reduction in double */

/* Reference density of the equation of state. */
#define SPH_RHO_REF_LATTICE 0 /* rho_ref = m * sum over the dx-lattice of W:
                                 the unperturbed lattice is at p = 0 */
#define SPH_RHO_REF_LITERAL 1 /* rho_ref = rho0 */

/* Model of the step (sph_params.model). */
#define SPH_MODEL_WCSPH 0      /* summation density, Tait EOS, symmetric viscosity,
                                  boundary particles (the default) */
#define SPH_MODEL_EXAMPLE_1A 1 /* Example 1a in the paper's own form: continuity
                                  equation, linear EOS, Pi_ij with rho_i */
#define SPH_MODEL_DEM 2        /* Example 2: Hertzian spheres (DEM) in a tank on a
                                  spring */
#define SPH_MODEL_FIELDS 3     /* the particle system only (cells, reorders): pair
                                  sums come from interaction laws compiled by the
                                  caller against this library (sph_law_view);
                                  sph_step and sph_forces are not available */

/* Treatment of a pair of opposite domain faces (Section 3.2.1). */
#define SPH_BC_CUTOFF 0    /* nothing beyond the face; leaving it is an error */
#define SPH_BC_SYMMETRIC 1 /* mirror plane: images with the position reflected and
                              the normal velocity negated */
#define SPH_BC_PERIODIC 2  /* images shifted by the domain edge; particles that
                              leave re-enter on the other side */

/* Particle kinds. */
#define SPH_FLUID 0
#define SPH_BOUNDARY 1

/*
 * Case constants.  Symbols follow Section 5.1.1 of the paper:
 *   W(r, h) = alpha_D (1 - q/2)^4 (2q + 1), q = r/h, support 2h;
 *   rho_i = m (W(0) + sum_{j != i, |r_ij| < 2h} W_ij)          (summation);
 *   p_i = B ((rho_i/rho_ref)^gamma - 1), B = c0^2 rho0 / gamma, p >= 0 if
 *         clamp_neg_p                                           (Tait EOS);
 *   dv_i/dt = -sum_j m (p_i/rho_i^2 + p_j/rho_j^2 + Pi_ij) grad_i W_ij + g
 *         (Eq. diffop1 form), Pi_ij = -alpha c0 h (v_ij . r_ij) /
 *         (rhobar_ij (|r_ij|^2 + visc_eps h^2)) when v_ij . r_ij < 0;
 *   v += dt a; r += dt v (semi-implicit Euler, fluid particles only).
 * The cell grid (Section 3.2.1) has ncell[k] cells of edge cs starting at
 * dom_min[k]; cs must be >= 2h (the neighbours of a particle lie in the 3^D
 * cells around its own), except that SPH_MODEL_WCSPH also takes h <= cs < 2h
 * (the 5^D cells around a particle's own, walked as 5^(D-1) rows of five
 * consecutive cells: fewer candidate pairs to test, the same neighbour sets
 * under the same predicate).  gamma must be an integer in [1, 8].
 */
typedef struct {
    int dim;          /* 2 or 3 (gravity usually along the last axis) */
    int precision;    /* SPH_PREC_F64 or SPH_PREC_F32 */
    int rho_ref_mode; /* SPH_RHO_REF_LATTICE or SPH_RHO_REF_LITERAL */
    int clamp_neg_p;  /* 1: negative pressure clamped to 0 */
    int ncell[3];     /* cells per axis; ncell[2] ignored when dim == 2 */
    double dom_min[3];
    double cs;        /* cell edge (m), >= 2h (>= h for SPH_MODEL_WCSPH) */
    double dx;        /* lattice spacing (m), used by SPH_RHO_REF_LATTICE */
    double h;         /* smoothing length (m) */
    double mass;      /* particle mass (kg) */
    double rho0;      /* rest density (kg/m^dim) */
    double c0;        /* numerical speed of sound (m/s) */
    double gamma;     /* Tait exponent */
    double alpha;     /* artificial viscosity coefficient */
    double visc_eps;  /* viscosity regulariser epsilon */
    double dt;        /* time step (s) */
    double g[3];      /* body acceleration (m/s^2) */
    int model;        /* SPH_MODEL_WCSPH (0), SPH_MODEL_EXAMPLE_1A or SPH_MODEL_DEM */
    int boundary[3];  /* SPH_BC_* per axis; SPH_MODEL_WCSPH takes only SPH_BC_CUTOFF */
    /* SPH_MODEL_DEM only (Section 5.2, Example 2) */
    double young;     /* Young modulus E of the spheres (Pa) */
    double poisson;   /* Poisson ratio nu */
    double friction;  /* Coulomb coefficient c_f */
    double tank_mass; /* M of the tank (kg); 0: no tank, the frame is inertial */
    double tank_stiffness; /* S of its spring (kg/s^2) */
    /* time step control (the CFL bound of Section 5.1.1's explicit scheme;
     * the adaptive step of Example 1b's variables) */
    int dt_mode;      /* SPH_DT_FIXED (0, also a zeroed struct) or SPH_DT_ADAPTIVE */
    double cfl;       /* SPH_DT_ADAPTIVE: safety factor in (0, 1] on the bound */
} sph_params;

/* SPH_DT_FIXED: every step takes dt.  SPH_DT_ADAPTIVE (SPH_MODEL_WCSPH, not in
 * batches or the adjoint): the first step of a context takes dt, every later
 * step min(dt, cfl * dt_cfl) with dt_cfl = min(0.25 h/(c0 + vmax), 0.25
 * sqrt(h/amax)) of the step before it (vmax after it, amax during it; the
 * same FP64 reduction that raises SPH_STATUS_CFL).  The context keeps the
 * next step size and the elapsed time on the device (sph_diag.dt / .time). */
#define SPH_DT_FIXED 0
#define SPH_DT_ADAPTIVE 1

/*
 * SPH_MODEL_EXAMPLE_1A (Section 5.1.1, Eq. SPH_fluid_continuity to
 * Eq. SPH_fluid_momentum, the equation order of Appendix A).  Per step,
 * with sums over the neighbour images (j, t) of i within 2h (i itself
 * excluded; images across symmetric or periodic faces included):
 *   rho_i' = rho_i - dt rho_i sum_j (m/rho_j) (v_j - v_i) . grad_i W_ij
 *   p_i'   = c0^2 (rho_i' - rho0)
 *   dv_i/dt = -sum_j (p_i'/rho_i'^2 + p_j'/rho_j'^2 + Pi_ij) m grad_i W_ij + g,
 *   Pi_ij  = -alpha c0 h (v_ji . r_ji) / (rho_i' |r_ji|^2) if v_ji . r_ji < 0
 *   v += dt a, r += dt v (fluid only), wrapped across periodic faces.
 * c0 is the paper's c, alpha its viscosity coefficient (0.1); gamma,
 * rho_ref_mode, clamp_neg_p, visc_eps and dx are not used.  The state's rho
 * array is the density field: read and advanced by every step (and by
 * sph_forces), carried along by every reorder.  An image across a symmetric
 * face is the particle reflected in the face (velocity component normal to
 * it negated); across a periodic face the particle shifted by the domain
 * edge ncell * cs.  Both are exact images of the relative position in the
 * predicate's precision (FP32: x_ij = (o_i - S) - s o_j per axis with the
 * frame shift S and sign s of the image; FP64: the same on absolute
 * coordinates).
 *
 * SPH_MODEL_DEM (Section 5.2, Eq. DEM_force, Eq. effective_quantities,
 * Eq. tank_ode, Eq. boundary_force).  Spheres with per-particle radius R_i
 * and mass m_i (sph_state.radius / .mass) and shared E, nu, c_f.  h is the
 * largest radius (cs >= 2h); rho0, c0, gamma, alpha, visc_eps, dx are not
 * used.  Per step, over the neighbour images (j, t) of i with overlap
 * delta = R_i + R_j - |r_ij| > 0 (n = r_ij / |r_ij|, v_ij = v_i - v_j^t):
 *   R' = R_i R_j/(R_i + R_j), m' = m_i m_j/(m_i + m_j), E' = E / (2 (1 - nu^2)),
 *   k = 4/3 sqrt(R') E', c = sqrt(m' k) / 8,
 *   f_n = k delta^(3/2) - c delta^(1/4) (v_ij . n)     (pushing i away from j)
 *   v_t = -v_ij + (v_ij . n) n, f_t = c_f |f_n| v_t / |v_t| (0 when
 *   |v_t| <= 1e-5 |v_ij|: no sliding, no direction)
 *   F_i = sum (f_n n + f_t);  F^b = the part of sum_i F_i from mirror images
 *   (the tank walls are the symmetric faces; angular velocities neglected);
 *   Zddot = (-S Z - F^b_z) / M  (z = the last axis; the tank state Z, Zdot
 *   lives in the context, sph_tank_set / sph_tank_get);
 *   a_i = F_i / m_i + g - Zddot e_z   (the particles move in the tank's frame)
 *   v += dt a, r += dt v, Zdot += dt Zddot, Z += dt Zdot.
 * sph_forces writes a_i (with the Zddot of that configuration) and leaves
 * the tank state unchanged.  The SPH status bit CFL is not raised.
 */

/* The particle state.  All pointers are device pointers of n elements.
 * r[2] and v[2] are ignored (may be NULL) when dim == 2.  rho and p receive
 * the density and pressure computed during the last step (outputs only).
 * Boundary particles must have zero velocity; they are never moved. */
typedef struct {
    int n;
    double *r[3];
    void *v[3];   /* float* (F32) or double* (F64); NULL allowed for SPH_MODEL_FIELDS */
    void *rho;    /* float* (F32) or double* (F64) */
    void *p;      /* float* (F32) or double* (F64) */
    uint32_t *id; /* persistent ids, unique */
    uint8_t *kind;/* SPH_FLUID or SPH_BOUNDARY */
    void *radius; /* SPH_MODEL_DEM: radius of each sphere (float / double); else NULL */
    void *mass;   /* SPH_MODEL_DEM: mass of each sphere (float / double); else NULL */
} sph_state;

/* Diagnostics of the last step of a sph_step call. */
typedef struct {
    int64_t n_pairs;  /* ordered pairs (i, j != i) with |r_ij| < 2h, all particles */
    int64_t n_pairs_fluid; /* the same with i a fluid particle (the force pass) */
    double vmax;      /* max |v| over fluid after the step */
    double amax;      /* max |a| over fluid in the step */
    double dt_cfl;    /* min(0.25 h/(c0 + vmax), 0.25 sqrt(h/amax)) */
    uint32_t status;  /* device status bits accumulated so far (not cleared) */
    double dt;        /* the step size of the last step */
    double time;      /* simulated time of all steps of the context so far */
} sph_diag;

typedef struct sph_ctx sph_ctx;

/* Create a context for up to n_capacity particles on the current CUDA
 * device: validates the parameters (SPH_ERR_INVALID) and allocates the
 * whole workspace (cell tables, sort buffers, sorted particle copies).
 * On success *out receives the context, which the caller releases with
 * sph_destroy.  Blocking. */
int sph_create(const sph_params *params, int n_capacity, sph_ctx **out);
int sph_destroy(sph_ctx *ctx);

/* Message of the last error on this context (static storage of the
 * context; "" when none).  ctx may be NULL for errors of sph_create. */
const char *sph_last_error(const sph_ctx *ctx);

/* Reference density the context uses (host value, for reports). */
double sph_rho_ref(const sph_ctx *ctx);

/*
 * Neighbour-search build (Section 3.2.1): cell hash of every particle,
 * sort by (cell, persistent id), cell start table, and the reorder of
 * r, v, id, kind into that order in the caller's arrays.
 */
int sph_build_cells(sph_ctx *ctx, sph_state *s, sph_stream_t stream);

/* Cell start table of the last build: n_cells + 1 entries; the particles of
 * cell c are [start[c], start[c+1]) in the canonical order.  *n_cells
 * receives the number of cells; when cell_start (a device array of
 * n_cells + 1 uint32) is not NULL the table is copied into it on stream. */
int sph_cell_table(sph_ctx *ctx, uint32_t *cell_start, int64_t *n_cells, sph_stream_t stream);

/* Test-only neighbour queries.  Both rebuild the cells first (so the
 * caller's state is left in canonical order).  counts[i] = number of
 * neighbours j != i of the i-th particle (|r_ij| < 2h in the context's
 * precision, the predicate that the pair sums use).  sph_neighbor_list
 * writes, for every particle i, the persistent ids of its neighbours in
 * ascending order to ids[offsets[i] .. offsets[i] + counts[i]); offsets
 * (n entries, int64) is computed by the caller from counts. */
int sph_neighbor_counts(sph_ctx *ctx, sph_state *s, uint32_t *counts, sph_stream_t stream);
int sph_neighbor_list(sph_ctx *ctx, sph_state *s, const int64_t *offsets, uint32_t *ids,
                      sph_stream_t stream);

/* Neighbour images (any model): like sph_neighbor_list, with the image code
 * of every entry in images[] (uint8, same offsets): per axis t = 0 (the
 * particle itself), 1 (its image across the lower face), 2 (across the
 * upper face), code = t_x + 3 t_y + 9 t_z; entries sorted by id, then code.
 * counts for the offsets come from sph_neighbor_counts. */
int sph_neighbor_images(sph_ctx *ctx, sph_state *s, const int64_t *offsets, uint32_t *ids, uint8_t *images,
                        sph_stream_t stream);

/*
 * The SPH sampling operator of the performance benchmark (Section 6):
 *   S_i = sum_j A_j m_j / rho_j W_ij
 * over the neighbour images of i within 2h, i itself included, on the cells
 * of the last sph_build_cells of this context.  The particles must not
 * have moved since that build (no sph_step in between: SPH_ERR_INVALID);
 * A, m, rho (inputs) and S (output) are device arrays of n float (F32) or
 * double (F64) in the state's order after that build (its canonical
 * order), n the count of that build.  It walks the 3^D stencil: the
 * context's cells must have edge cs >= 2h (SPH_ERR_INVALID otherwise).
 */
int sph_sample(sph_ctx *ctx, const void *A, const void *m, const void *rho, void *S, sph_stream_t stream);

/* Pair sums without integration: rebuild, density + EOS into s->rho / s->p,
 * accelerations into a[0..dim-1] (device arrays of n float or double, in
 * the canonical order; zero for boundary particles). */
int sph_forces(sph_ctx *ctx, sph_state *s, void *a[3], sph_stream_t stream);

/* (SPH_MODEL_EXAMPLE_1A: s->rho is advanced by the continuity equation and
 * s->p set, as the first five equations of Appendix A do; r and v are not
 * changed.  SPH_MODEL_DEM: a receives the accelerations of Section 5.2.) */

/* Advance nsteps time steps (each: build, density + EOS, accelerations and
 * integration, CFL reduction).  diag, when not NULL, receives the
 * diagnostics of the last step; the call then synchronises the stream.
 * With nsteps >= 2 the context records one step as a CUDA graph for this
 * state (its pointers and n) the first time and replays it nsteps times, the
 * same kernels in the same order (identical results, without the launch gaps
 * of nine launches per step); a different state records again.  Not while
 * phase profiling is on or the stream is being captured by the caller (the
 * steps are then launched one by one); the graph is the context's and is
 * freed by sph_destroy. */
int sph_step(sph_ctx *ctx, sph_state *s, int nsteps, sph_diag *diag, sph_stream_t stream);

/* sph_step on a state held in HOST memory (the end-to-end call): the arrays
 * of s are host pointers with the meaning and layout of sph_state.  The
 * inputs are copied into device buffers owned by the context (allocated by
 * the first such call, n_capacity particles; copy kernels over the device
 * mapping of page-locked arrays, the driver's copy for pageable ones,
 * spread over 4 copy streams of the context and ordered with `stream`),
 * and the first nsteps - 1 steps run there.  When every array is
 * page-locked (cudaHostAlloc / cudaHostRegister) the last step writes the
 * host arrays directly through their device mapping; otherwise it writes
 * the device buffers, which are then copied back.  Returns when the steps
 * and their copies are complete: the host arrays then hold the new state
 * (r, v, id, kind in canonical order, rho and p; DEM: r, v, id, kind,
 * radius, mass).  Errors as sph_step, plus SPH_ERR_CUDA when the device
 * copy cannot be allocated. */
int sph_step_host(sph_ctx *ctx, sph_state *s, int nsteps, sph_diag *diag, sph_stream_t stream);

/* Apply the permutation of the last build of ctx to a caller field of n
 * elements of elem_bytes bytes each (4, 8, 12, 16, 24 or 32), n the count of
 * that build: out[k] = in[the particle now in canonical slot k].  in and out
 * are device arrays of n elements that must not overlap.  Lets a caller
 * keep fields of its own aligned with a state that sph_build_cells has
 * reordered (Section 3.2.1: the particle system sorts every field). */
int sph_reorder_field(sph_ctx *ctx, const void *in, void *out, int elem_bytes, sph_stream_t stream);

/* The same for nfields fields of one element size in one pass: in and out
 * are host arrays of nfields device pointers (n elements each, the
 * permutation read once per particle).  No output may overlap an input or
 * another output (SPH_ERR_INVALID); nfields = 0 does nothing. */
int sph_reorder_fields(sph_ctx *ctx, int nfields, const void *const *in, void *const *out, int elem_bytes,
                       sph_stream_t stream);

/* The build of SPH_MODEL_FIELDS contexts (the interaction-law compiler)
 * with its outputs in caller arrays: sph_build_cells on the state `in`, but
 * the canonical r, id and kind go to `out` (device arrays of in->n, which
 * must not overlap in's), and nfields caller fields of elem_bytes bytes
 * each (4 or 8) are reordered into fout in the same gather (fout[f][k] =
 * fin[f][the particle in canonical slot k]; no output may overlap an input
 * or another output).  `in` is left as it was, so a caller alternates two
 * states.  Afterwards the cells are current for `out` (sph_reorder_fields
 * and sph_law_view refer to it).  SPH_ERR_INVALID for other models, a size
 * mismatch, NULL arrays or overlaps. */
int sph_build_cells_into(sph_ctx *ctx, const sph_state *in, sph_state *out, int nfields, const void *const *fin,
                         void *const *fout, int elem_bytes, sph_stream_t stream);

/* Views for kernels compiled against this library's internal headers (the
 * interaction-law compiler of the Python package): the sorted particle copy,
 * cell of each sorted particle, cell start table and the context's kernel
 * constants, as left by the last build, and the context's neighbour-mask
 * scratch.  params points to host memory of params_bytes bytes owned by the
 * context (its layout is the internal one; a compiled law checks
 * params_bytes).  The mask scratch (hit masks in the layout of the
 * library's pair passes: blocks of 128 particles x 3^D stencil cells x 128
 * words; a hit count and an overflow flag per particle) is overwritten by
 * every pair pass of the context.  Valid until the next call on ctx. */
typedef struct {
    const void *pos;          /* sorted positions (+ w), float4 (F32) / double4 (F64) */
    const uint32_t *cell_s;   /* cell of each sorted particle */
    const uint32_t *cell_start; /* n_cells + 1 */
    const void *params;       /* host copy of the kernel constants */
    int64_t params_bytes;
    int n;                    /* particles of the last build */
    int precision;
    uint32_t *mask;           /* hit masks (scratch) */
    uint16_t *nnb;            /* hits per particle, self included (scratch) */
    uint8_t *ovf;             /* 1: a cell held more than 32 particles (scratch) */
} sph_law_views;
int sph_law_view(sph_ctx *ctx, sph_law_views *out);

/* Tank of SPH_MODEL_DEM: set (Z, Zdot) (enqueued on stream), or read Z,
 * Zdot, the last step's Zddot and wall force F^b[3] (any pointer may be
 * NULL; synchronises the stream). */
int sph_tank_set(sph_ctx *ctx, double Z, double Zdot, sph_stream_t stream);
int sph_tank_get(sph_ctx *ctx, double *Z, double *Zdot, double *Zddot, double *F_wall, sph_stream_t stream);

/* The context's clock: the step size of its next step (under SPH_DT_FIXED
 * always params.dt) and the simulated time of its steps so far.  get reads
 * both (either pointer may be NULL; synchronises the stream); set replaces
 * them, enqueued on stream (a checkpoint restore): dt_next must be in
 * (0, params.dt] under SPH_DT_ADAPTIVE, params.dt otherwise
 * (SPH_ERR_INVALID). */
int sph_clock_get(sph_ctx *ctx, double *dt_next, double *time, sph_stream_t stream);
int sph_clock_set(sph_ctx *ctx, double dt_next, double time, sph_stream_t stream);

/* Read the device status word into *out (a bit set of SPH_STATUS_*) and
 * clear it.  sync != 0 waits for the context's work on `stream` first;
 * otherwise the value may miss bits of work still in flight. */
int sph_get_status(sph_ctx *ctx, uint32_t *out, int sync, sph_stream_t stream);

/* Adjoint (reverse-mode) variables of a state: dL/dr and dL/dv, device
 * arrays of n elements per component in the order of the state they belong
 * to; r_bar is double, v_bar float (F32) or double (F64). */
typedef struct {
    double *r_bar[3];
    void *v_bar[3];
} sph_grad;

/*
 * Reverse mode of one sph_step (the hand-written adjoint of the density,
 * EOS, pressure + viscosity and integration kernels).  s_n is the state the
 * forward step started from, in any order; it is not modified (its rho and
 * p arrays are not written).  g_np1 is the adjoint of the state that step
 * produced, in that state's order (the canonical order of s_n's cells, which
 * is how sph_step leaves its state).  g_n receives the adjoint of s_n in
 * s_n's order; it must not alias g_np1.  *alpha_bar (a device double, may be
 * NULL) is incremented by dL/dalpha through this step.  The neighbour sets
 * are those of s_n (frozen; the kernel and its first two derivatives vanish
 * at the support radius).  The forward quantities are recomputed inside.
 * SPH_MODEL_WCSPH contexts only.
 */
int sph_step_adjoint(sph_ctx *ctx, const sph_state *s_n, const sph_grad *g_np1, sph_grad *g_n,
                     double *alpha_bar, sph_stream_t stream);

/* The products of the last build and WCSPH density pass -- the sorted
 * copy with densities and P/rho^2, the hit masks, the cell table and the
 * permutation, all that a reverse step reads -- saved to / loaded from
 * device memory, so that a checkpointed reverse sweep need not rebuild what
 * its recomputed forward step already built.  After sph_step these are the
 * products of the step's input state.
 *   sph_build_save: *bytes = their size; with dst != NULL also enqueue the
 *     copy into dst (device, *bytes bytes).  SPH_ERR_INVALID when no density
 *     pass followed the last build, or for a model other than SPH_MODEL_WCSPH.
 *   sph_build_load: enqueue the copy back from src (saved for n particles).
 *   sph_adjoint_of_build: sph_step_adjoint of the state whose products are
 *     loaded (no rebuild); SPH_ERR_INVALID unless products of n particles
 *     are in place. */
int sph_build_save(sph_ctx *ctx, void *dst, int64_t *bytes, sph_stream_t stream);
int sph_build_load(sph_ctx *ctx, const void *src, int n, sph_stream_t stream);
int sph_adjoint_of_build(sph_ctx *ctx, int n, const sph_grad *g_np1, sph_grad *g_n, double *alpha_bar,
                         sph_stream_t stream);
/* sph_build_load followed by sph_adjoint_of_build, without the copy: the
 * reverse step reads the products in place from `saved` (a block written by
 * sph_build_save for n particles on this context, 256-byte aligned, not
 * modified).  The same kernels on the same values: identical results.  The
 * context's own build products are left as they were. */
int sph_adjoint_of_saved(sph_ctx *ctx, const void *saved, int n, const sph_grad *g_np1, sph_grad *g_n,
                         double *alpha_bar, sph_stream_t stream);

/*
 * Batched form: many independent cases advanced together by one persistent
 * cooperative kernel (all phases of all steps in one launch, separated by
 * device-wide barriers with a bounded wait), captured in a CUDA graph the
 * first time a (nsteps, state buffers) combination is stepped.
 *
 * The packed state holds case 0's particles, then case 1's, ...: case c
 * owns [off_c, off_c + cases[c].n) where off_c is the sum of the earlier
 * cases' n; each case stays in its slice (reordered canonically inside it).
 * Every case has its own sph_params (grid, constants, dt); all cases must
 * share dim and precision.  A case evolves bit for bit as it would under
 * sph_step alone.
 */
typedef struct {
    sph_params params;
    int n; /* particles of this case */
} sph_case_desc;

/* Form of the batched step (sph_tune.form). */
#define SPH_BATCH_PERSISTENT 0 /* one cooperative kernel per call, grid barriers between phases */
#define SPH_BATCH_PHASED 1     /* one ordinary launch per phase and step (blocks of 128) */

/* Launch shape (0 = default): threads per block (64, 128 or 256; 128 for the
 * phased form), resident blocks per SM (persistent form; capped by
 * occupancy), the barrier spin limit (persistent form; polls of ~100 ns;
 * default 2^24, i.e. seconds before SPH_STATUS_BARRIER_TIMEOUT) and the
 * form.  Both forms run the same phase bodies and give the same results bit
 * for bit. */
typedef struct {
    int block;
    int blocks_per_sm;
    long long spin_limit;
    int form;
} sph_tune;

typedef struct sph_batch sph_batch;

/* Validates every case (SPH_ERR_INVALID names the case; SPH_MODEL_WCSPH
 * only), allocates the packed workspace and the per-case cell tables.
 * Blocking. */
int sph_batch_create(const sph_case_desc *cases, int ncases, const sph_tune *tune, sph_batch **out);
int sph_batch_destroy(sph_batch *b);
const char *sph_batch_last_error(const sph_batch *b);

/* Advance every case nsteps steps in one launch, or in nsteps x 9 launches
 * for the phased form (through a CUDA graph when capture works on this
 * system, otherwise direct launches).
 * packed->n must equal the sum of the cases' n. */
int sph_batch_step(sph_batch *b, sph_state *packed, int nsteps, sph_stream_t stream);

/* Device status bits of the batch (read and cleared), as sph_get_status. */
int sph_batch_get_status(sph_batch *b, uint32_t *out, int sync, sph_stream_t stream);

/* Synchronises the device; per_case (ncases entries, may be NULL) receives
 * vmax, amax and dt_cfl of each case's last step; *n_pairs_total (may be
 * NULL) the ordered pairs counted since creation. */
int sph_batch_diag(sph_batch *b, sph_diag *per_case, int64_t *n_pairs_total);

/* Launch shape in use (the phased form: block 128, grid = the pair phases'
 * blocks) and whether graphs are used (1), not yet tried (-1) or
 * unavailable (0); n_total = packed particle count. */
int sph_batch_info(const sph_batch *b, int *block, int *grid, int *graph_used, int *n_total);

/* Self-test of the barrier timeout (no GPU fault involved; persistent form
 * only, SPH_ERR_INVALID for the phased one): launches the persistent kernel
 * in a mode where block 0 leaves before the first barrier, so the other
 * blocks' wait can only end by the spin limit; returns the
 * status bits seen (SPH_STATUS_BARRIER_TIMEOUT expected) in *status_out.
 * Synchronises the stream.  The state is not touched. */
int sph_batch_selftest_barrier(sph_batch *b, const sph_state *packed, long long spin_limit, uint32_t *status_out,
                               sph_stream_t stream);

/*
 * The neighbour-search build without a context, for callers that cannot
 * allocate device memory when they need it: code that runs under another
 * component's allocator (a framework's caching pool, a process that reserved
 * its device memory up front), loops that must not stall on cudaMalloc or
 * cudaFree (both can synchronise the device), or plug-ins handed only the
 * particle arrays.  The paper has no counterpart; it is a packaging of
 * sph_build_cells.
 *
 * Same result as sph_build_cells (the caller's r, v, id and kind arrays are
 * left in the canonical order) for a case described by params; the cell
 * start table (ncell product + 1 uint32, device) is copied to cell_start and
 * the status bits (SPH_STATUS_*) to *status (a device uint32) when those are
 * not NULL.  Allocates nothing: the scratch is a fixed array in device memory
 * owned by the library for the life of the process (about 11 MB on every GPU
 * that loads the library), for at most SPH_STATIC_MAX_PARTICLES particles,
 * SPH_STATIC_MAX_CELLS cells and SPH_STATIC_MAX_AXIS_CELLS cells per axis;
 * larger requests fail with SPH_ERR_CAPACITY and a message from
 * sph_static_last_error().  Every call looks up the array's device address
 * (cudaGetSymbolAddress); the first call on a device is the set-up, which may
 * load the library's device code there and with it the array, so make that
 * first call before any stream capture and before the rest of the device
 * memory is reserved.  All calls share the array: calls that overlap on the
 * GPU race with each other and must be serialised by the caller.  As in
 * sph_build_cells, v may be NULL for SPH_MODEL_FIELDS.
 */
#define SPH_STATIC_MAX_PARTICLES 65536
#define SPH_STATIC_MAX_CELLS 262144
#define SPH_STATIC_MAX_AXIS_CELLS 16384
int sph_build_cells_static(const sph_params *params, sph_state *s, uint32_t *cell_start, uint32_t *status,
                           sph_stream_t stream);
/* The message of the calling thread's last failed sph_build_cells_static
 * call (each host thread has its own). */
const char *sph_static_last_error(void);

/*
 * Phase timing with CUDA events (for benchmarks).  sph_profile_begin makes
 * the next max_steps steps of sph_step record events around their phases:
 * SPH_PROF_BUILD (hash, scan, scatter, reorder), SPH_PROF_DENSITY (density +
 * EOS kernel), SPH_PROF_FORCE (acceleration + integration kernel),
 * SPH_PROF_FINISH (CFL reduction epilogue).  sph_profile_end synchronises
 * the stream of the recorded steps, writes the summed device time of each
 * phase in ms to ms[0..SPH_PROF_NPHASE-1] and the number of recorded steps
 * to *steps, and stops recording.  Allocates its events in
 * sph_profile_begin (not during the steps).
 */
#define SPH_PROF_BUILD 0
#define SPH_PROF_DENSITY 1
#define SPH_PROF_FORCE 2
#define SPH_PROF_FINISH 3
#define SPH_PROF_NPHASE 4
int sph_profile_begin(sph_ctx *ctx, int max_steps);
int sph_profile_end(sph_ctx *ctx, double *ms, int64_t *steps);

#ifdef __cplusplus
}
#endif

#endif /* SPH_GB300_H */
