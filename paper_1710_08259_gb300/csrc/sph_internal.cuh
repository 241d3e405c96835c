// sph_internal.cuh -- internal declarations of the GB300 WCSPH library.
//
// Layout in HBM (per context, sized at sph_create):
//   caller state (SoA, canonical order after every call)
//       r[d][n] double, v[d][n] T, rho[n] T, p[n] T, id[n] u32, kind[n] u8
//   binning scratch
//       key[n] u32 (linear cell), rank[n] u32 (arrival slot inside the cell),
//       tmp[n] u32 (particle index in arrival order), cell_count[ncells] u32,
//       cell_start[ncells + 1] u32, block_sums[] u32
//   sorted working copy (gathered by the reorder, read by the pair sums)
//       pos[n]  Vec4<T>: F32: cell-relative float offsets (ox, oy, oz, 0)
//                        F64: absolute positions (x, y, z, 0)
//       vel[n]  Vec4<T>: (vx, vy, vz, rho)  -- rho filled by the density pass
//       phat[n] T: p / rho^2
//       rs[d][n] double positions, cell_s[n] u32, id_s[n] u32, kind_s[n] u8
//   accumulators: n_pairs (u64), max |v|^2, max |a|^2 (double bit patterns),
//       the device status word, the diagnostics of the last step.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/sph.h"

namespace sph {

struct __align__(16) StencilEntry {
    float sx, sy, sz;
    int dcell;  // dx + nc0 * (dy + nc1 * dz)
};

constexpr int kBlock = 128;          // threads per block of the particle kernels
constexpr int kScanThreads = 256;    // scan block
constexpr int kScanItems = 8;        // cells per scan thread
constexpr int kScanTile = kScanThreads * kScanItems;

// Lanes per particle of the pair passes on cells of edge h (small cases): a
// team deals a particle's stencil rows out while the grid stays within about
// one wave of the GPU, n x TEAM <= kTeamLanes threads; 1 for larger cases.
constexpr long long kTeamLanes = 150000;
inline int pair_team(int n)
{
    if ((long long)n * 8 <= kTeamLanes) return 8;
    if ((long long)n * 4 <= kTeamLanes) return 4;
    if ((long long)n * 2 <= kTeamLanes) return 2;
    return 1;
}

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };
template <typename T> using vec4_t = typename Vec4<T>::type;

// Constants of one case, passed by value to every kernel.
struct DevParams {
    int dim;
    int nc[3];
    uint32_t cell_off;  // offset of this case's cells in a shared cell table (0: single case)
    double dom_min[3];
    double cs, inv_cs;
    int K;              // stencil radius in cells: 1 (cs >= 2h, 3^D cells) or 2 (h <= cs < 2h, 5^D cells as rows)
    double dt;
    double R2;          // (2h)^2, FP64 predicate
    float R2f;          // ((float)2h)^2, FP32 predicate
    float csf;          // (float)cs
    double half_inv_h;  // 1 / (2h)
    double S_ref, inv_S_ref;  // reference of the unnormalised density sum
    double mAlpha;      // m * alpha_D  (rho = mAlpha * S)
    double mCg;         // m * 5 alpha_D / h^2  (grad_i W_ij = -(5 alpha_D/h^2) t^3 r_ij)
    double visc_num;    // -2 alpha c0 h
    double eps_h2;      // visc_eps h^2
    double B;           // c0^2 rho0 / gamma
    double binom[9];    // (1+d)^gamma - 1 = d * sum_k binom[k] d^k
    int gamma;
    int clamp;
    double g[3];
    // cell base tables: base[k][c] = dom_min[k] + c * cs (double RN, no
    // contraction), c = 0..nc[k]; bkey = the same values as order-preserving
    // signed 64-bit keys, so that the hash compares integers, not doubles
    const double *bval[3];
    const long long *bkey[3];
    float lof[3];       // (float)dom_min, for the float estimate of the cell
    float inv_csf;      // (float)(1 / cs)
    // the 3^D stencil cells in stencil order (dz, dy, dx): frame shifts
    // (float)d * (float)cs per axis (exact products) and the cell-index delta
    const struct StencilEntry *stab;
    // adjoint / CFL constants
    double h, c0, alpha;
    double visc_num1;   // -2 c0 h: viscosity numerator per unit alpha
    double inv_rho_ref; // 1 / rho_ref
    double Bg_rho_ref;  // B gamma / rho_ref
    // model and domain faces (SPH_MODEL_*, SPH_BC_* per axis)
    int model;
    int bc[3];
    double per[3];      // ncell * cs: the period of a periodic axis
    double hi[3];       // dom_min + ncell * cs: the upper face
    // SPH_MODEL_EXAMPLE_1A constants
    double c2;          // c0^2 (linear EOS)
    double rho0;
    double visc1a;      // -alpha c0 h (Pi_ij numerator per v_ij . r_ij)
    double alphaD;      // alpha_D of the kernel (sampling operator)
    // SPH_MODEL_DEM constants
    double demEp;       // E' = E / (2 (1 - nu^2))
    double demCf;       // Coulomb coefficient
    double tankM, tankS;
    // bounds-checked builds: where violations are recorded (null: unchecked)
    // and the particle capacity of the buffers
    uint32_t *chk_status;
    uint32_t chk_cap;
    // SPH_DT_ADAPTIVE: the step size of the next step lives on the device
    // (DiagDev::dt_next of the context); dt is then its upper bound
    int adaptive;
    double cfl;
    const double *dt_next;
};

// Checked builds (-DSPH_CHECK): an index that would leave its buffer sets
// SPH_STATUS_BOUNDS in the context's status word and the caller skips the
// access; in the normal build the test compiles away.
#ifdef SPH_CHECK
__device__ __forceinline__ bool sph_in_bounds(const DevParams &P, bool ok)
{
    if (!ok && P.chk_status) atomicOr(P.chk_status, SPH_STATUS_BOUNDS);
    return ok || !P.chk_status;
}
#define SPH_IN_BOUNDS(P, cond) ::sph::sph_in_bounds((P), (cond))
#else
#define SPH_IN_BOUNDS(P, cond) true
#endif

// Tank of SPH_MODEL_DEM (device): state, last acceleration, last wall force.
struct TankDev {
    double Z, Zdot, Zddot;
    double Fb[3];
    unsigned int done;  // blocks of the wall-force sum that finished (0 between steps)
    unsigned int pad;
};

// Accumulator block (device).
struct Accum {
    unsigned long long n_pairs;
    unsigned long long vmax2;  // bit pattern of a non-negative double
    unsigned long long amax2;
    unsigned long long n_pairs_fluid;
};

struct DiagDev {
    long long n_pairs;
    long long n_pairs_fluid;
    double vmax, amax, dt_cfl;
    unsigned int status;
    unsigned int pad;
    double dt;       // the step size of the last step
    double time;     // simulated time of the context's steps
    double dt_next;  // the step size of the next step (SPH_DT_ADAPTIVE)
};

// Host values of the stencil table in stencil order; 27 entries (2D uses the
// first 9, dz = 0).  K = 2: the 5^(D-1) rows (dz, dy) of the 5^D stencil, the
// cell offset of a row's cell at dx = 0 and its y / z frame shifts (25
// entries in 3D, 5 in 2D).
inline void stencil_table(int dim, double cs, const int nc[3], StencilEntry out[27], int K = 1)
{
    const float csf = (float)cs;
    int idx = 0;
    if (K == 2) {
        for (int dz = (dim == 3 ? -2 : 0); dz <= (dim == 3 ? 2 : 0); ++dz)
            for (int dy = -2; dy <= 2; ++dy) {
                out[idx].sx = 0.f;
                out[idx].sy = (float)dy * csf;
                out[idx].sz = (float)dz * csf;
                out[idx].dcell = nc[0] * (dy + nc[1] * dz);
                ++idx;
            }
        for (; idx < 27; ++idx) out[idx] = StencilEntry{0.f, 0.f, 0.f, 0};
        return;
    }
    for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                out[idx].sx = (float)dx * csf;
                out[idx].sy = (float)dy * csf;
                out[idx].sz = (float)dz * csf;
                out[idx].dcell = dx + nc[0] * (dy + nc[1] * dz);
                ++idx;
            }
    for (; idx < 27; ++idx) out[idx] = StencilEntry{0.f, 0.f, 0.f, 0};
}

// Derive the kernel constants of one case (validates p; fills everything but
// the base-table pointers and cell_off).  Returns false with a reason.
bool make_dev_params(const sph_params *p, DevParams *d, double *rho_ref, std::string &why);

// ---- launchers (sph_cells.cu) -------------------------------------------
struct CellBufs {
    uint32_t *key, *rank, *tmp, *cell_count, *cell_start, *block_sums;
    int64_t ncells;
    int scan_blocks;
};

struct SortedBufs {
    void *pos, *vel, *phat;
    double *rs[3];
    uint32_t *cell_s, *id_s;
    uint8_t *kind_s;
    uint32_t *mask;  // neighbour hit masks, one word per (particle, stencil cell), block-major
    uint8_t *ovf;    // 1: a stencil cell held > 32 particles (slow path)
    uint32_t *src;   // caller index of each canonical slot (the reorder's permutation)
    uint16_t *nnb;   // hits of each particle in its masks (neighbours + self)
};

// Adjoint scratch (sorted order): abar (Vec4<T>), vtilde (Vec4<T>), rhobar (T),
// per-block partial sums of alphabar (double) and the count of blocks that
// have written theirs.
struct AdjBufs {
    void *abar, *vt, *rhobar;
    double *alpha_part;
    unsigned int *alpha_ticket;  // blocks of k_adj_rho done (0 between launches)
};

// Words of neighbour masks for n particles: blocks x stencil cells x kBlock
// (the 3^D stencil's count, which also holds the 5^(D-1) rows of K = 2).
inline size_t mask_words(int dim, size_t n)
{
    const size_t nb = (n + kBlock - 1) / kBlock;
    return nb * (dim == 3 ? 27 : 9) * kBlock;
}

cudaError_t launch_build(const DevParams &P, bool f32, int n, const sph_state &s, const CellBufs &cb,
                         const SortedBufs &sb, uint32_t *status, cudaStream_t st);
cudaError_t launch_writeback(const DevParams &P, bool f32, int n, const sph_state &s,
                             const SortedBufs &sb, cudaStream_t st);
// out[k] = in[src[k]] for elements of elem_bytes
cudaError_t launch_reorder_field(int n, const uint32_t *src, const void *in, void *out, int elem_bytes,
                                 cudaStream_t st);
// Up to kMaxFields caller fields reordered in one launch.
constexpr int kMaxFields = 8;
struct FieldSet {
    const uint32_t *in[kMaxFields];
    uint32_t *out[kMaxFields];
    int nf;
};
cudaError_t launch_reorder_fields(int n, const uint32_t *src, const FieldSet &fs, int elem_bytes, cudaStream_t st);
// A build whose gather writes the canonical r / id / kind through sb's rs /
// id_s / kind_s (caller arrays) and reorders the fields of fs (elem_bytes 4
// or 8) in the same pass.
cudaError_t launch_build_into(const DevParams &P, bool f32, int n, const sph_state &s, const CellBufs &cb,
                              const SortedBufs &sb, const FieldSet &fs, int elem_bytes, uint32_t *status,
                              cudaStream_t st);
// Copy bytes between device memory and the device mapping of page-locked
// host memory with a kernel (both addresses 16-byte aligned).
cudaError_t launch_copy_bytes(const void *src, void *dst, size_t bytes, int sms, cudaStream_t st);
// Up to 16 device-to-device copies (16-byte aligned starts) in one launch.
struct CopySections {
    const void *src[16];
    void *dst[16];
    size_t bytes[16];
    int m;
};
cudaError_t launch_copy_sections(const CopySections &cs, cudaStream_t st);
// fill bval / bkey (device arrays of nc[k] + 1 entries per axis)
cudaError_t launch_base_tables(const DevParams &P, double *bval[3], long long *bkey[3], cudaStream_t st);

// ---- launchers (sph_pairs.cu) -------------------------------------------
cudaError_t launch_density(const DevParams &P, bool f32, int n, const CellBufs &cb,
                           const SortedBufs &sb, void *rho_out, void *p_out, Accum *acc,
                           cudaStream_t st);
// a_out != nullptr: write accelerations (sph_forces); otherwise integrate and
// write the new state to s (sph_step).
cudaError_t launch_force(const DevParams &P, bool f32, int n, const CellBufs &cb,
                         const SortedBufs &sb, const sph_state &s, void *const *a_out, Accum *acc,
                         uint32_t *status, cudaStream_t st);
cudaError_t launch_finish(const DevParams &P, double h, double c0, Accum *acc, uint32_t *status,
                          DiagDev *diag, int step, cudaStream_t st);
// ---- launchers (sph_adjoint.cu) -----------------------------------------
cudaError_t launch_adjoint(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                           const AdjBufs &ab, const sph_grad &g1, const sph_grad &g0, double *alpha_bar,
                           cudaStream_t st);
// neighbour sets found by the last density pass: counts (if not null) and
// ascending id lists at offsets (if ids not null)
cudaError_t launch_nbr(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                       uint32_t *counts, const int64_t *offsets, uint32_t *ids, cudaStream_t st,
                       uint8_t *images = nullptr);

// ---- launchers (sph_model.cu): Example 1a form, domain faces, sampling ----
// continuity + linear EOS over the neighbour images (records the masks);
// rho1 / p1 (canonical order, may be null) receive rho' and p'.
cudaError_t launch_cont(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                        void *rho1, void *p1, Accum *acc, cudaStream_t st);
// momentum over the masks of launch_cont; a_out != nullptr: accelerations
// only, otherwise integrate into s (periodic faces wrap).
cudaError_t launch_mom(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                       const sph_state &s, const void *rho1, void *const *a_out, Accum *acc, uint32_t *status,
                       cudaStream_t st);
// neighbour images from the masks of the last pair pass (either model)
cudaError_t launch_nbr_img(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                           uint32_t *counts, const int64_t *offsets, uint32_t *ids, uint8_t *img, cudaStream_t st);
// ---- launchers (sph_dem.cu): Example 2 ------------------------------------
// contact forces into F (sorted Vec4<T>), per-block wall-force partials into
// fbp (3 doubles per block), contact count into acc->n_pairs
cudaError_t launch_dem_force(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                             void *F, double *fbp, Accum *acc, cudaStream_t st);
// the tank: sum of the partials in a fixed order, Zddot; advance (Z, Zdot)
// when advance != 0
cudaError_t launch_dem_tank(const DevParams &P, int n, double *fbp, TankDev *tank, int advance, cudaStream_t st);
// bytes of the wall-force partials buffer for n spheres
size_t dem_partials_bytes(int n);
// accelerations a = F/m + g - Zddot e_z; a_out != nullptr: write them,
// otherwise integrate into s
cudaError_t launch_dem_integrate(const DevParams &P, bool f32, int n, const SortedBufs &sb, const void *F,
                                 const TankDev *tank, const sph_state &s, void *const *a_out, Accum *acc,
                                 uint32_t *status, cudaStream_t st);

// S_i = sum_j A_j m_j / rho_j W_ij on the sorted copy of the last build
cudaError_t launch_sample(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                          const void *A, const void *m, const void *rho, void *S, cudaStream_t st);

}  // namespace sph
