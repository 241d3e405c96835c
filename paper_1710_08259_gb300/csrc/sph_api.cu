// sph_api.cu -- the C ABI (include/sph.h): context, workspace, step driver.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sph_internal.cuh"

using namespace sph;

struct sph_ctx {
    sph_params prm;
    int cap = 0;
    bool f32 = false;
    DevParams dp{};
    double rho_ref = 0.0;
    CellBufs cb{};
    SortedBufs sb{};
    Accum *acc = nullptr;
    uint32_t *status = nullptr;
    DiagDev *diag_dev = nullptr;
    DiagDev *diag_host = nullptr;  // pinned
    AdjBufs ab{};
    StencilEntry *stab = nullptr;
    double *bval[3] = {nullptr, nullptr, nullptr};
    long long *bkey[3] = {nullptr, nullptr, nullptr};
    std::string err;
    // the sorted copy and cell table belong to the caller's current
    // positions (set by a build that moved nothing, cleared by sph_step)
    bool cells_current = false;
    int cells_n = 0;
    // particles of the last WCSPH density pass whose products (sorted copy,
    // densities, P/rho^2, masks, cell table, permutation) are still in the
    // buffers (-1: none): what sph_build_save / sph_adjoint_of_build use
    int dens_n = -1;
    // SPH_MODEL_DEM: contact forces (sorted Vec4), wall-force partials per
    // block, the tank
    void *dem_F = nullptr;
    double *dem_fbp = nullptr;
    TankDev *tank = nullptr;
    // phase profiling (sph_profile_begin / _end)
    std::vector<cudaEvent_t> ev;  // 5 per recorded step
    int prof_cap = 0, prof_steps = 0;
    bool prof_on = false;
    cudaStream_t prof_stream = nullptr;
    // sph_step_host: the device copy of a host state (allocated by the first
    // call, capacity cap) and the copy streams with their join events
    sph_state hs{};
    std::vector<void *> hs_bufs;
    cudaStream_t cs[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ce[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // sph_step with nsteps >= 2: one step recorded as a CUDA graph (for the
    // state gstate) and replayed, which removes the launch gaps between the
    // step's nine kernels (2D 64 x 64 dam break: 0.063 -> 0.042 ms per FP32
    // step); gfailed: recording failed once, the context steps eagerly
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    sph_state gstate{};
    bool gfailed = false;
};

static const int kCopyStreams = 4;

static const int kEvPerStep = 5;

// NVTX range over a host scope (phases of a step show up by name in nsys /
// ncu; a no-op without an attached tool).
struct NvtxScope {
    explicit NvtxScope(const char *name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope &) = delete;
    NvtxScope &operator=(const NvtxScope &) = delete;
};

static void prof_mark(sph_ctx *ctx, int k, cudaStream_t st)
{
    if (!ctx->prof_on || ctx->prof_steps >= ctx->prof_cap) return;
    cudaEventRecord(ctx->ev[(size_t)ctx->prof_steps * kEvPerStep + k], st);
    ctx->prof_stream = st;
}

static std::string g_create_error;

static int fail(sph_ctx *c, int code, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return code;
}

static int cuda_fail(sph_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, SPH_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

// Wendland normalisation alpha_D (Section 5.1.1).
static double alpha_D(int dim, double h)
{
    if (dim == 2) return 7.0 / (4.0 * M_PI * h * h);
    return 21.0 / (16.0 * M_PI * h * h * h);
}

// Unnormalised kernel sum over the dx-lattice around an interior particle,
// self included: sum_k w(|k| dx / h), w(q) = (1 - q/2)^4 (2q + 1), |k| dx < 2h.
static double lattice_w_sum(int dim, double dx, double h)
{
    const double R = 2.0 * h;
    const int K = (int)std::ceil(R / dx) + 1;
    double s = 0.0;
    for (int c = (dim == 3 ? -K : 0); c <= (dim == 3 ? K : 0); ++c)
        for (int b = -K; b <= K; ++b)
            for (int a = -K; a <= K; ++a) {
                const double r = std::sqrt((double)(a * a + b * b + c * c)) * dx;
                if (r >= R) continue;
                const double q = r / h;
                const double t = 1.0 - 0.5 * q;
                s += t * t * t * t * (2.0 * q + 1.0);
            }
    return s;
}

static double binomial(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

static int validate(const sph_params *p, std::string &why)
{
    if (!p) return why = "params is NULL", 0;
    if (p->dim != 2 && p->dim != 3) return why = "dim must be 2 or 3", 0;
    if (p->precision != SPH_PREC_F64 && p->precision != SPH_PREC_F32) return why = "bad precision", 0;
    if (p->model != SPH_MODEL_WCSPH && p->model != SPH_MODEL_EXAMPLE_1A && p->model != SPH_MODEL_DEM &&
        p->model != SPH_MODEL_FIELDS)
        return why = "bad model", 0;
    const bool dem = p->model == SPH_MODEL_DEM;
    if (dem) {
        if (!(p->young > 0.0) || !std::isfinite(p->young)) return why = "DEM: Young modulus must be > 0", 0;
        if (!(p->poisson >= 0.0 && p->poisson < 0.5)) return why = "DEM: Poisson ratio must be in [0, 0.5)", 0;
        if (!(p->friction >= 0.0) || !std::isfinite(p->friction)) return why = "DEM: friction must be >= 0", 0;
        if (!(p->tank_mass >= 0.0) || !(p->tank_stiffness >= 0.0) || !std::isfinite(p->tank_mass) ||
            !std::isfinite(p->tank_stiffness))
            return why = "DEM: tank mass and stiffness must be >= 0", 0;
    }
    for (int k = 0; k < p->dim; ++k) {
        const int b = p->boundary[k];
        if (b != SPH_BC_CUTOFF && b != SPH_BC_SYMMETRIC && b != SPH_BC_PERIODIC) return why = "bad boundary", 0;
        if (p->model == SPH_MODEL_WCSPH && b != SPH_BC_CUTOFF)
            return why = "SPH_MODEL_WCSPH uses boundary particles: every boundary must be SPH_BC_CUTOFF", 0;
    }
    const bool wc = p->model == SPH_MODEL_WCSPH;
    if (wc && p->rho_ref_mode != SPH_RHO_REF_LATTICE && p->rho_ref_mode != SPH_RHO_REF_LITERAL)
        return why = "bad rho_ref_mode", 0;
    if (!(p->h > 0.0) || !std::isfinite(p->h)) return why = "h must be > 0", 0;
    // cells no smaller than the support radius 2h (Section 3.2.1: the 3^D
    // adjacent cells); the WCSPH step also takes cells of edge in [h, 2h),
    // searched through the 5^D cells around a particle's own
    if (!std::isfinite(p->cs)) return why = "cell edge cs must be finite", 0;
    // (the field model's compiled laws walk the rows too, when no face has images)
    bool all_cut = true;
    for (int k = 0; k < p->dim; ++k) all_cut = all_cut && p->boundary[k] == SPH_BC_CUTOFF;
    const bool rows_ok = wc || (p->model == SPH_MODEL_FIELDS && all_cut);
    if (rows_ok && !(p->cs >= p->h)) return why = "cell edge cs must be >= h", 0;
    if (!rows_ok && !(p->cs >= 2.0 * p->h)) return why = "cell edge cs must be >= 2h for this model", 0;
    if (wc && p->rho_ref_mode == SPH_RHO_REF_LATTICE && !(p->dx > 0.0)) return why = "dx must be > 0", 0;
    const bool fields = p->model == SPH_MODEL_FIELDS;
    if (!dem && !fields && (!(p->mass > 0.0) || !(p->rho0 > 0.0) || !(p->c0 > 0.0)))
        return why = "mass, rho0, c0 must be > 0", 0;
    if (!(p->dt >= 0.0) || !std::isfinite(p->dt) || (wc && !(p->dt > 0.0))) return why = "dt must be > 0", 0;
    if (!(p->alpha >= 0.0) || !std::isfinite(p->alpha)) return why = "alpha must be >= 0", 0;
    if (wc && !(p->visc_eps > 0.0)) return why = "visc_eps must be > 0", 0;
    double gi = std::floor(p->gamma);
    if (wc && (gi != p->gamma || gi < 1.0 || gi > 8.0)) return why = "gamma must be an integer in [1, 8]", 0;
    double ncells = 1.0;
    for (int k = 0; k < p->dim; ++k) {
        if (p->ncell[k] < 1) return why = "ncell must be >= 1", 0;
        if (!std::isfinite(p->dom_min[k])) return why = "dom_min must be finite", 0;
        ncells *= (double)p->ncell[k];
    }
    if (ncells > 2.0e9) return why = "too many cells", 0;
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(p->g[k])) return why = "g must be finite", 0;
    if (p->dt_mode != SPH_DT_FIXED && p->dt_mode != SPH_DT_ADAPTIVE) return why = "bad dt_mode", 0;
    if (p->dt_mode == SPH_DT_ADAPTIVE) {
        if (!wc) return why = "SPH_DT_ADAPTIVE steps SPH_MODEL_WCSPH only", 0;
        if (!(p->cfl > 0.0 && p->cfl <= 1.0)) return why = "cfl must be in (0, 1]", 0;
    }
    return 1;
}

namespace sph {

bool make_dev_params(const sph_params *pp, DevParams *dd, double *rho_ref, std::string &why)
{
    if (!validate(pp, why)) return false;
    const sph_params &p = *pp;
    DevParams &d = *dd;
    d = DevParams{};
    d.dim = p.dim;
    for (int k = 0; k < 3; ++k) {
        d.nc[k] = k < p.dim ? p.ncell[k] : 1;
        d.dom_min[k] = k < p.dim ? p.dom_min[k] : 0.0;
        d.g[k] = p.g[k];
    }
    d.cell_off = 0;
    d.cs = p.cs;
    d.inv_cs = 1.0 / p.cs;
    d.K = p.cs >= 2.0 * p.h ? 1 : 2;
    d.dt = p.dt;
    d.adaptive = p.dt_mode == SPH_DT_ADAPTIVE;
    d.cfl = p.cfl;
    d.dt_next = nullptr;  // (set by the context that owns the step size)
    const double R = 2.0 * p.h;
    d.R2 = R * R;
    const float Rf = (float)R;
    d.R2f = Rf * Rf;
    d.csf = (float)p.cs;
    d.half_inv_h = 1.0 / (2.0 * p.h);
    const double aD = alpha_D(p.dim, p.h);
    d.mAlpha = p.mass * aD;
    d.mCg = p.mass * 5.0 * aD / (p.h * p.h);
    d.visc_num = -2.0 * p.alpha * p.c0 * p.h;
    d.eps_h2 = p.visc_eps * p.h * p.h;
    const bool wc = p.model == SPH_MODEL_WCSPH;
    const double gam = wc ? p.gamma : 1.0;  // the Tait constants are unused by Example 1a
    d.B = p.c0 * p.c0 * p.rho0 / gam;
    d.gamma = (int)gam;
    for (int k = 0; k < 9; ++k) d.binom[k] = k < d.gamma ? binomial(d.gamma, k + 1) : 0.0;
    d.S_ref = (wc && p.rho_ref_mode == SPH_RHO_REF_LATTICE) ? lattice_w_sum(p.dim, p.dx, p.h)
              : (p.mass > 0.0 && p.rho0 > 0.0)                 ? p.rho0 / (p.mass * aD)
                                                               : 1.0;
    d.inv_S_ref = 1.0 / d.S_ref;
    d.clamp = p.clamp_neg_p ? 1 : 0;
    *rho_ref = d.mAlpha * d.S_ref;
    for (int k = 0; k < 3; ++k) d.lof[k] = (float)d.dom_min[k];
    d.inv_csf = (float)(1.0 / p.cs);
    d.h = p.h;
    d.c0 = p.c0;
    d.alpha = p.alpha;
    d.visc_num1 = -2.0 * p.c0 * p.h;
    d.inv_rho_ref = 1.0 / *rho_ref;
    d.Bg_rho_ref = d.B * gam / *rho_ref;
    d.model = p.model;
    for (int k = 0; k < 3; ++k) {
        d.bc[k] = k < p.dim ? p.boundary[k] : SPH_BC_CUTOFF;
        d.per[k] = (double)d.nc[k] * p.cs;
        d.hi[k] = d.dom_min[k] + d.per[k];
    }
    d.c2 = p.c0 * p.c0;
    d.rho0 = p.rho0;
    d.visc1a = -p.alpha * p.c0 * p.h;
    d.alphaD = aD;
    d.demEp = p.model == SPH_MODEL_DEM ? p.young / (2.0 * (1.0 - p.poisson * p.poisson)) : 0.0;
    d.demCf = p.friction;
    d.tankM = p.tank_mass;
    d.tankS = p.tank_stiffness;
    return true;
}

}  // namespace sph

extern "C" {

const char *sph_last_error(const sph_ctx *ctx)
{
    return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

double sph_rho_ref(const sph_ctx *ctx) { return ctx ? ctx->rho_ref : 0.0; }

int sph_destroy(sph_ctx *ctx)
{
    if (!ctx) return SPH_OK;
    void *bufs[] = {ctx->cb.key, ctx->cb.rank, ctx->cb.tmp, ctx->cb.cell_count, ctx->cb.cell_start,
                    ctx->cb.block_sums, ctx->sb.pos, ctx->sb.vel, ctx->sb.phat, ctx->sb.rs[0],
                    ctx->sb.rs[1], ctx->sb.rs[2], ctx->sb.cell_s, ctx->sb.id_s, ctx->sb.kind_s,
                    ctx->acc, ctx->status, ctx->diag_dev, ctx->sb.mask, ctx->sb.ovf, ctx->bval[0],
                    ctx->bval[1], ctx->bval[2], ctx->bkey[0], ctx->bkey[1], ctx->bkey[2], ctx->sb.src,
                    ctx->ab.abar, ctx->ab.vt, ctx->ab.rhobar, ctx->ab.alpha_part, ctx->ab.alpha_ticket, ctx->stab,
                    ctx->sb.nnb,
                    ctx->dem_F, ctx->dem_fbp, ctx->tank};
    for (void *b : bufs)
        if (b) cudaFree(b);
    if (ctx->diag_host) cudaFreeHost(ctx->diag_host);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    for (void *b : ctx->hs_bufs) cudaFree(b);
    for (cudaStream_t c : ctx->cs)
        if (c) cudaStreamDestroy(c);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    for (cudaEvent_t e : ctx->ce)
        if (e) cudaEventDestroy(e);
    delete ctx;
    return SPH_OK;
}

int sph_create(const sph_params *params, int n_capacity, sph_ctx **out)
{
    if (!out) return fail(nullptr, SPH_ERR_INVALID, "out is NULL");
    *out = nullptr;
    std::string why;
    if (!validate(params, why)) return fail(nullptr, SPH_ERR_INVALID, why);
    if (n_capacity < 1 || n_capacity > (1 << 30)) return fail(nullptr, SPH_ERR_INVALID, "bad n_capacity");
    sph_ctx *ctx = new (std::nothrow) sph_ctx();
    if (!ctx) return fail(nullptr, SPH_ERR_INVALID, "out of host memory");
    ctx->prm = *params;
    const sph_params &p = *params;
    ctx->cap = n_capacity;
    ctx->f32 = p.precision == SPH_PREC_F32;
    DevParams &d = ctx->dp;
    make_dev_params(params, &d, &ctx->rho_ref, why);
    int64_t ncells = 1;
    for (int k = 0; k < 3; ++k) ncells *= d.nc[k];

    CellBufs &cb = ctx->cb;
    cb.ncells = ncells;
    cb.scan_blocks = (int)((ncells + kScanTile - 1) / kScanTile);
    const size_t padded = (size_t)cb.scan_blocks * kScanTile;
    const size_t n = (size_t)n_capacity;
    const size_t tsz = ctx->f32 ? sizeof(float) : sizeof(double);
    auto alloc = [&](void **ptr, size_t bytes) -> cudaError_t { return cudaMalloc(ptr, bytes > 0 ? bytes : 16); };
    cudaError_t e = cudaSuccess;
#define AL(ptr, bytes)                                                     \
    if (e == cudaSuccess) {                                                \
        e = alloc((void **)&(ptr), (bytes));                               \
        if (e != cudaSuccess) {                                            \
            fail(nullptr, SPH_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e)); \
        }                                                                  \
    }
    AL(cb.key, n * 4);
    AL(cb.rank, n * 4);
    AL(cb.tmp, n * 4);
    AL(cb.cell_count, padded * 4);
    AL(cb.cell_start, ((size_t)ncells + 1) * 4);
    AL(cb.block_sums, (size_t)cb.scan_blocks * 4);
    AL(ctx->sb.pos, n * 4 * tsz);
    AL(ctx->sb.vel, n * 4 * tsz);
    AL(ctx->sb.phat, n * tsz);
    for (int k = 0; k < 3; ++k) {
        if (k < p.dim) AL(ctx->sb.rs[k], n * 8);
    }
    AL(ctx->sb.cell_s, n * 4);
    AL(ctx->sb.id_s, n * 4);
    AL(ctx->sb.kind_s, n);
    AL(ctx->sb.mask, mask_words(p.dim, n) * 4);
    AL(ctx->sb.ovf, n);
    AL(ctx->sb.src, n * 4);
    AL(ctx->stab, 27 * sizeof(StencilEntry));
    AL(ctx->sb.nnb, n * 2);
    AL(ctx->ab.abar, n * 4 * tsz);
    AL(ctx->ab.vt, n * 4 * tsz);
    AL(ctx->ab.rhobar, n * tsz);
    // (one partial per block of the adjoint density kernel: a block per 128
    // particles, or per 128 / TEAM particles of a team kernel)
    AL(ctx->ab.alpha_part, ((n + kBlock - 1) / kBlock + (kTeamLanes + kBlock - 1) / kBlock) * 8);
    AL(ctx->ab.alpha_ticket, sizeof(unsigned int));
    for (int k = 0; k < p.dim; ++k) {
        AL(ctx->bval[k], ((size_t)p.ncell[k] + 1) * 8);
        AL(ctx->bkey[k], ((size_t)p.ncell[k] + 1) * 8);
    }
    if (p.model == SPH_MODEL_DEM) {
        AL(ctx->dem_F, n * 4 * tsz);
        AL(ctx->dem_fbp, dem_partials_bytes(n));
        AL(ctx->tank, sizeof(TankDev));
    }
    AL(ctx->acc, sizeof(Accum));
    AL(ctx->status, sizeof(uint32_t));
    AL(ctx->diag_dev, sizeof(DiagDev));
#undef AL
    d.chk_status = ctx->status;  // used by bounds-checked builds only
    d.chk_cap = (uint32_t)n_capacity;
    d.dt_next = ctx->diag_dev ? &ctx->diag_dev->dt_next : nullptr;
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->diag_host, sizeof(DiagDev));
    if (e == cudaSuccess) e = cudaMemset(cb.cell_count, 0, padded * 4);
    if (e == cudaSuccess) e = cudaMemset(cb.cell_start, 0, ((size_t)ncells + 1) * 4);
    if (e == cudaSuccess) e = cudaMemset(ctx->acc, 0, sizeof(Accum));
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(ctx->ab.alpha_ticket, 0, sizeof(unsigned int));
    if (e == cudaSuccess) {
        // (the first step of a context takes dt)
        DiagDev d0{};
        d0.dt_next = p.dt;
        e = cudaMemcpy(ctx->diag_dev, &d0, sizeof(d0), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && ctx->tank) e = cudaMemset(ctx->tank, 0, sizeof(TankDev));
    if (e == cudaSuccess) {
        StencilEntry sh[27];
        stencil_table(p.dim, p.cs, d.nc, sh, d.K);
        e = cudaMemcpy(ctx->stab, sh, sizeof(sh), cudaMemcpyHostToDevice);
        d.stab = ctx->stab;
    }
    if (e == cudaSuccess) {
        for (int k = 0; k < 3; ++k) {
            d.bval[k] = ctx->bval[k];
            d.bkey[k] = ctx->bkey[k];
        }
        e = launch_base_tables(d, ctx->bval, ctx->bkey, 0);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        std::string msg = std::string("sph_create: ") + cudaGetErrorString(e);
        sph_destroy(ctx);
        return fail(nullptr, SPH_ERR_CUDA, msg);
    }
    *out = ctx;
    return SPH_OK;
}

static int check_state(sph_ctx *ctx, const sph_state *s)
{
    if (!ctx) return SPH_ERR_INVALID;
    if (!s) return fail(ctx, SPH_ERR_INVALID, "state is NULL");
    if (s->n < 0) return fail(ctx, SPH_ERR_INVALID, "negative particle count");
    if (s->n > ctx->cap) return fail(ctx, SPH_ERR_CAPACITY, "more particles than the context capacity");
    if (s->n == 0) return SPH_OK;
    // the field model's state is positions only: its fields are the caller's
    const bool need_v = ctx->prm.model != SPH_MODEL_FIELDS;
    for (int k = 0; k < ctx->prm.dim; ++k)
        if (!s->r[k] || (need_v && !s->v[k])) return fail(ctx, SPH_ERR_INVALID, "NULL r or v component");
    if (!s->id || !s->kind) return fail(ctx, SPH_ERR_INVALID, "NULL id or kind");
    if (ctx->prm.model == SPH_MODEL_EXAMPLE_1A && !s->rho)
        return fail(ctx, SPH_ERR_INVALID, "SPH_MODEL_EXAMPLE_1A needs the density field rho");
    if (ctx->prm.model == SPH_MODEL_DEM && (!s->radius || !s->mass))
        return fail(ctx, SPH_ERR_INVALID, "SPH_MODEL_DEM needs the radius and mass arrays");
    return SPH_OK;
}

static bool model_1a(const sph_ctx *ctx) { return ctx->prm.model == SPH_MODEL_EXAMPLE_1A; }
static bool model_dem(const sph_ctx *ctx) { return ctx->prm.model == SPH_MODEL_DEM; }

static int build(sph_ctx *ctx, const sph_state *s, cudaStream_t st)
{
    ctx->cells_current = false;
    ctx->dens_n = -1;
    CK(launch_build(ctx->dp, ctx->f32, s->n, *s, ctx->cb, ctx->sb, ctx->status, st));
    return SPH_OK;
}

// A build whose state is then written back unmoved: the cells stay current.
static void mark_current(sph_ctx *ctx, const sph_state *s)
{
    ctx->cells_current = true;
    ctx->cells_n = s->n;
}

// The first pass of the model: candidate tests + masks and the density
// (summation + Tait, or continuity + linear EOS).
// Whether the model's first pass records image masks (the 3^D image
// stencil of sph_model.cu) rather than the WCSPH masks (3^D cells or rows):
// Example 1a, DEM, and the field model on cells of edge >= 2h.  A field model
// on cells of edge h (cut-off faces) searches as the WCSPH step does.
static bool uses_images(const sph_ctx *ctx)
{
    return model_1a(ctx) || model_dem(ctx) || (ctx->prm.model == SPH_MODEL_FIELDS && ctx->dp.K == 1);
}

static int pair_pass1(sph_ctx *ctx, const sph_state *s, void *rho_out, void *p_out, cudaStream_t st)
{
    // the DEM and field models' neighbour queries take the masks of a first
    // pass whose density outputs go nowhere
    if (model_dem(ctx) || ctx->prm.model == SPH_MODEL_FIELDS) rho_out = p_out = nullptr;
    if (uses_images(ctx)) {
        CK(launch_cont(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, rho_out, p_out, ctx->acc, st));
    } else {
        CK(launch_density(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, rho_out, p_out, ctx->acc, st));
        if (ctx->prm.model == SPH_MODEL_WCSPH) ctx->dens_n = s->n;
    }
    return SPH_OK;
}

int sph_build_cells(sph_ctx *ctx, sph_state *s, sph_stream_t stream)
{
    int rc = check_state(ctx, s);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = build(ctx, s, st))) return rc;
    CK(launch_writeback(ctx->dp, ctx->f32, s->n, *s, ctx->sb, st));
    mark_current(ctx, s);
    return SPH_OK;
}

int sph_cell_table(sph_ctx *ctx, uint32_t *cell_start, int64_t *n_cells, sph_stream_t stream)
{
    if (!ctx || !n_cells) return SPH_ERR_INVALID;
    *n_cells = ctx->cb.ncells;
    if (cell_start)
        CK(cudaMemcpyAsync(cell_start, ctx->cb.cell_start, ((size_t)ctx->cb.ncells + 1) * sizeof(uint32_t),
                           cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return SPH_OK;
}

int sph_neighbor_counts(sph_ctx *ctx, sph_state *s, uint32_t *counts, sph_stream_t stream)
{
    int rc = check_state(ctx, s);
    if (rc) return rc;
    if (!counts && s->n > 0) return fail(ctx, SPH_ERR_INVALID, "counts is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = build(ctx, s, st))) return rc;
    // the Example 1a pass writes no field here: the state's density stays
    const bool img = uses_images(ctx);
    if ((rc = pair_pass1(ctx, s, img ? nullptr : s->rho, img ? nullptr : s->p, st))) return rc;
    if (img)
        CK(launch_nbr_img(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, counts, nullptr, nullptr, nullptr, st));
    else
        CK(launch_nbr(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, counts, nullptr, nullptr, st));
    CK(launch_finish(ctx->dp, ctx->prm.h, ctx->prm.c0, ctx->acc, ctx->status, ctx->diag_dev, 0, st));
    CK(launch_writeback(ctx->dp, ctx->f32, s->n, *s, ctx->sb, st));
    mark_current(ctx, s);
    return SPH_OK;
}

int sph_neighbor_list(sph_ctx *ctx, sph_state *s, const int64_t *offsets, uint32_t *ids,
                      sph_stream_t stream)
{
    int rc = check_state(ctx, s);
    if (rc) return rc;
    if ((!offsets || !ids) && s->n > 0) return fail(ctx, SPH_ERR_INVALID, "offsets or ids is NULL");
    return sph_neighbor_images(ctx, s, offsets, ids, nullptr, stream);
}

int sph_neighbor_images(sph_ctx *ctx, sph_state *s, const int64_t *offsets, uint32_t *ids, uint8_t *images,
                        sph_stream_t stream)
{
    int rc = check_state(ctx, s);
    if (rc) return rc;
    if ((!offsets || !ids) && s->n > 0) return fail(ctx, SPH_ERR_INVALID, "offsets or ids is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = build(ctx, s, st))) return rc;
    const bool img = uses_images(ctx);
    if ((rc = pair_pass1(ctx, s, img ? nullptr : s->rho, img ? nullptr : s->p, st))) return rc;
    // (the WCSPH model has cut-off faces only: every image code is 0)
    if (img)
        CK(launch_nbr_img(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, nullptr, offsets, ids, images, st));
    else
        CK(launch_nbr(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, nullptr, offsets, ids, st, images));
    CK(launch_finish(ctx->dp, ctx->prm.h, ctx->prm.c0, ctx->acc, ctx->status, ctx->diag_dev, 0, st));
    CK(launch_writeback(ctx->dp, ctx->f32, s->n, *s, ctx->sb, st));
    mark_current(ctx, s);
    return SPH_OK;
}

int sph_forces(sph_ctx *ctx, sph_state *s, void *a[3], sph_stream_t stream)
{
    int rc = check_state(ctx, s);
    if (rc) return rc;
    if (ctx->prm.model == SPH_MODEL_FIELDS)
        return fail(ctx, SPH_ERR_INVALID, "SPH_MODEL_FIELDS has no built-in forces: run compiled laws");
    if (s->n > 0 && !model_dem(ctx) && (!s->rho || !s->p)) return fail(ctx, SPH_ERR_INVALID, "NULL rho or p");
    if (s->n > 0 && (!a || !a[0] || !a[1] || (ctx->prm.dim == 3 && !a[2])))
        return fail(ctx, SPH_ERR_INVALID, "NULL acceleration array");
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = build(ctx, s, st))) return rc;
    if (model_dem(ctx)) {
        CK(launch_dem_force(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, ctx->dem_F, ctx->dem_fbp, ctx->acc, st));
        CK(launch_dem_tank(ctx->dp, s->n, ctx->dem_fbp, ctx->tank, 0, st));
        CK(launch_dem_integrate(ctx->dp, ctx->f32, s->n, ctx->sb, ctx->dem_F, ctx->tank, *s, a, ctx->acc,
                                ctx->status, st));
        CK(launch_writeback(ctx->dp, ctx->f32, s->n, *s, ctx->sb, st));
        CK(launch_finish(ctx->dp, ctx->prm.h, ctx->prm.c0, ctx->acc, ctx->status, ctx->diag_dev, 0, st));
        mark_current(ctx, s);
        return SPH_OK;
    }
    if ((rc = pair_pass1(ctx, s, s->rho, s->p, st))) return rc;
    if (model_1a(ctx)) {
        CK(launch_mom(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, *s, s->rho, a, ctx->acc, ctx->status, st));
        // the density field was advanced in place: the writeback must not
        // restore the gathered (old) values
        sph_state w = *s;
        w.rho = nullptr;
        CK(launch_writeback(ctx->dp, ctx->f32, s->n, w, ctx->sb, st));
    } else {
        CK(launch_force(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, *s, a, ctx->acc, ctx->status, st));
        CK(launch_writeback(ctx->dp, ctx->f32, s->n, *s, ctx->sb, st));
    }
    CK(launch_finish(ctx->dp, ctx->prm.h, ctx->prm.c0, ctx->acc, ctx->status, ctx->diag_dev, 0, st));
    mark_current(ctx, s);
    return SPH_OK;
}

static bool model_fields(const sph_ctx *ctx) { return ctx->prm.model == SPH_MODEL_FIELDS; }

// One time step.  The build reads the state `in`; every later phase reads
// the sorted copy and writes the state `s` (the same arrays, or `in` staged
// on the device while `s` is the caller's host state).
static int step_once(sph_ctx *ctx, const sph_state *in, sph_state *s, cudaStream_t st)
{
    int rc;
    prof_mark(ctx, 0, st);
    {
        NvtxScope r("sph.build");
        if ((rc = build(ctx, in, st))) return rc;
    }
    prof_mark(ctx, 1, st);
    if (model_dem(ctx)) {
        CK(launch_dem_force(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, ctx->dem_F, ctx->dem_fbp, ctx->acc, st));
        prof_mark(ctx, 2, st);
        CK(launch_dem_tank(ctx->dp, s->n, ctx->dem_fbp, ctx->tank, 1, st));
        CK(launch_dem_integrate(ctx->dp, ctx->f32, s->n, ctx->sb, ctx->dem_F, ctx->tank, *s, nullptr, ctx->acc,
                                ctx->status, st));
        prof_mark(ctx, 3, st);
    } else {
        {
            NvtxScope r("sph.density");
            if ((rc = pair_pass1(ctx, s, s->rho, s->p, st))) return rc;
        }
        prof_mark(ctx, 2, st);
        NvtxScope rf("sph.force");
        if (model_1a(ctx))
            CK(launch_mom(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, *s, s->rho, nullptr, ctx->acc, ctx->status,
                          st));
        else
            CK(launch_force(ctx->dp, ctx->f32, s->n, ctx->cb, ctx->sb, *s, nullptr, ctx->acc, ctx->status, st));
        prof_mark(ctx, 3, st);
    }
    CK(launch_finish(ctx->dp, ctx->prm.h, ctx->prm.c0, ctx->acc, ctx->status, ctx->diag_dev, 1, st));
    prof_mark(ctx, 4, st);
    if (ctx->prof_on && ctx->prof_steps < ctx->prof_cap) ++ctx->prof_steps;
    return SPH_OK;
}

// Record one step_once on the context's capture stream into the step graph.
static int record_step_graph(sph_ctx *ctx, sph_state *s)
{
    if (ctx->gexec) {
        cudaGraphExecDestroy(ctx->gexec);
        ctx->gexec = nullptr;
    }
    if (!ctx->gstream) CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
    const int rc = step_once(ctx, s, s, ctx->gstream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->gstream, &g);
    if (rc || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc ? rc : cuda_fail(ctx, e, "cudaStreamEndCapture");
    }
    e = cudaGraphInstantiate(&ctx->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        ctx->gexec = nullptr;
        return cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    ctx->gstate = *s;
    return SPH_OK;
}

int sph_step(sph_ctx *ctx, sph_state *s, int nsteps, sph_diag *diag, sph_stream_t stream)
{
    int rc = check_state(ctx, s);
    if (rc) return rc;
    if (model_fields(ctx))
        return fail(ctx, SPH_ERR_INVALID, "SPH_MODEL_FIELDS has no built-in step: run compiled laws");
    if (nsteps < 0) return fail(ctx, SPH_ERR_INVALID, "negative nsteps");
    if (s->n > 0 && !model_dem(ctx) && (!s->rho || !s->p)) return fail(ctx, SPH_ERR_INVALID, "NULL rho or p");
    cudaStream_t st = (cudaStream_t)stream;
    NvtxScope range("sph_step");
    // a multi-step call replays the recorded step, unless phase profiling is
    // on (events per phase) or the caller is capturing this stream itself
    bool done = false;
    if (nsteps >= 2 && !ctx->prof_on && !ctx->gfailed && s->n > 0) {
        cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cst) == cudaSuccess && cst == cudaStreamCaptureStatusNone) {
            if (!ctx->gexec || std::memcmp(&ctx->gstate, s, sizeof(sph_state)) != 0) {
                if (record_step_graph(ctx, s)) ctx->gfailed = true;
            }
            if (ctx->gexec) {
                for (int it = 0; it < nsteps; ++it) CK(cudaGraphLaunch(ctx->gexec, st));
                done = true;
            }
        } else {
            cudaGetLastError();
        }
    }
    if (!done)
        for (int it = 0; it < nsteps; ++it)
            if ((rc = step_once(ctx, s, s, st))) return rc;
    if (diag) {
        CK(cudaMemcpyAsync(ctx->diag_host, ctx->diag_dev, sizeof(DiagDev), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        diag->n_pairs = ctx->diag_host->n_pairs;
        diag->n_pairs_fluid = ctx->diag_host->n_pairs_fluid;
        diag->vmax = ctx->diag_host->vmax;
        diag->amax = ctx->diag_host->amax;
        diag->dt_cfl = ctx->diag_host->dt_cfl;
        diag->status = ctx->diag_host->status;
        diag->dt = ctx->diag_host->dt;
        diag->time = ctx->diag_host->time;
    }
    return SPH_OK;
}

// One array copy of a host step: device, host, bytes.
struct HostCopy {
    void *dev;
    void *host;
    size_t bytes;
};

// The arrays of a state that exist, as (device array of ctx->hs, host
// array, bytes); inputs: what a step reads, outputs: what it writes.
static int host_copies(const sph_ctx *ctx, const sph_state *h, bool out, HostCopy *c)
{
    const size_t n = (size_t)h->n, tsz = ctx->f32 ? 4 : 8;
    const sph_state &d = ctx->hs;
    int m = 0;
    for (int k = 0; k < ctx->prm.dim; ++k) {
        c[m++] = {d.r[k], h->r[k], n * 8};
        c[m++] = {d.v[k], h->v[k], n * tsz};
    }
    c[m++] = {d.id, h->id, n * 4};
    c[m++] = {d.kind, h->kind, n};
    const bool dem = ctx->prm.model == SPH_MODEL_DEM;
    if (ctx->prm.model == SPH_MODEL_EXAMPLE_1A || (out && !dem)) c[m++] = {d.rho, h->rho, n * tsz};
    if (out && !dem) c[m++] = {d.p, h->p, n * tsz};
    if (dem) {  // per-sphere arrays: read, and reordered with their spheres
        c[m++] = {d.radius, h->radius, n * tsz};
        c[m++] = {d.mass, h->mass, n * tsz};
    }
    return m;
}

// Copies spread over the copy streams (each its own DMA queue), joined back
// into st: every copy stream waits for st's work so far, st waits for them.
static int spread_copies(sph_ctx *ctx, const HostCopy *c, int m, bool to_device, cudaStream_t st)
{
    CK(cudaEventRecord(ctx->ce[kCopyStreams], st));
    for (int q = 0; q < kCopyStreams; ++q) CK(cudaStreamWaitEvent(ctx->cs[q], ctx->ce[kCopyStreams], 0));
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    for (int i = 0; i < m; ++i) {
        cudaStream_t cq = ctx->cs[i % kCopyStreams];
        // page-locked host memory with a device mapping: a copy kernel over
        // the mapping; pageable memory: the driver's staged copy
        cudaPointerAttributes at{};
        void *mapped = nullptr;
        if (cudaPointerGetAttributes(&at, c[i].host) == cudaSuccess && at.type == cudaMemoryTypeHost)
            mapped = at.devicePointer;
        else
            cudaGetLastError();  // (an unregistered pointer is not an error here)
        const bool aligned = !((reinterpret_cast<uintptr_t>(mapped) | reinterpret_cast<uintptr_t>(c[i].dev)) & 15u);
        if (mapped && aligned) {
            if (to_device)
                CK(launch_copy_bytes(mapped, c[i].dev, c[i].bytes, sms, cq));
            else
                CK(launch_copy_bytes(c[i].dev, mapped, c[i].bytes, sms, cq));
        } else if (to_device) {  // (Default: the driver infers the direction from the addresses)
            CK(cudaMemcpyAsync(c[i].dev, c[i].host, c[i].bytes, cudaMemcpyDefault, cq));
        } else {
            CK(cudaMemcpyAsync(c[i].host, c[i].dev, c[i].bytes, cudaMemcpyDefault, cq));
        }
    }
    for (int q = 0; q < kCopyStreams; ++q) {
        CK(cudaEventRecord(ctx->ce[q], ctx->cs[q]));
        CK(cudaStreamWaitEvent(st, ctx->ce[q], 0));
    }
    return SPH_OK;
}

// The device copy of a host state (capacity cap) and the copy streams,
// made by the first call that stages a host state.
static int ensure_stage(sph_ctx *ctx)
{
    if (!ctx->hs_bufs.empty()) return SPH_OK;
    const size_t n = (size_t)ctx->cap, tsz = ctx->f32 ? 4 : 8;
    auto al = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        ctx->hs_bufs.push_back(p);
        return p;
    };
    bool ok = true;
    for (int k = 0; k < ctx->prm.dim; ++k) {
        ok = ok && (ctx->hs.r[k] = static_cast<double *>(al(n * 8)));
        ok = ok && (ctx->hs.v[k] = al(n * tsz));
    }
    ok = ok && (ctx->hs.rho = al(n * tsz)) && (ctx->hs.p = al(n * tsz));
    ok = ok && (ctx->hs.id = static_cast<uint32_t *>(al(n * 4))) && (ctx->hs.kind = static_cast<uint8_t *>(al(n)));
    if (model_dem(ctx)) ok = ok && (ctx->hs.radius = al(n * tsz)) && (ctx->hs.mass = al(n * tsz));
    for (int q = 0; q < kCopyStreams && ok; ++q)
        ok = cudaStreamCreateWithFlags(&ctx->cs[q], cudaStreamNonBlocking) == cudaSuccess;
    for (int q = 0; q <= kCopyStreams && ok; ++q)
        ok = cudaEventCreateWithFlags(&ctx->ce[q], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        for (void *b : ctx->hs_bufs) cudaFree(b);
        ctx->hs_bufs.clear();
        ctx->hs = sph_state{};
        return fail(ctx, SPH_ERR_CUDA, "sph_step_host: device allocation failed");
    }
    return SPH_OK;
}

static int host_diag(sph_ctx *ctx, sph_diag *diag, cudaStream_t st)
{
    if (diag) CK(cudaMemcpyAsync(ctx->diag_host, ctx->diag_dev, sizeof(DiagDev), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (diag) {
        diag->n_pairs = ctx->diag_host->n_pairs;
        diag->n_pairs_fluid = ctx->diag_host->n_pairs_fluid;
        diag->vmax = ctx->diag_host->vmax;
        diag->amax = ctx->diag_host->amax;
        diag->dt_cfl = ctx->diag_host->dt_cfl;
        diag->status = ctx->diag_host->status;
        diag->dt = ctx->diag_host->dt;
        diag->time = ctx->diag_host->time;
    }
    return SPH_OK;
}

int sph_step_host(sph_ctx *ctx, sph_state *s, int nsteps, sph_diag *diag, sph_stream_t stream)
{
    int rc = check_state(ctx, s);
    if (rc) return rc;
    if (model_fields(ctx))
        return fail(ctx, SPH_ERR_INVALID, "SPH_MODEL_FIELDS has no built-in step: run compiled laws");
    if (nsteps < 0) return fail(ctx, SPH_ERR_INVALID, "negative nsteps");
    if (s->n > 0 && !model_dem(ctx) && (!s->rho || !s->p)) return fail(ctx, SPH_ERR_INVALID, "NULL rho or p");
    cudaStream_t st = (cudaStream_t)stream;
    NvtxScope range("sph_step_host");
    if (nsteps == 0) return host_diag(ctx, diag, st);
    if ((rc = ensure_stage(ctx))) return rc;
    ctx->hs.n = s->n;
    HostCopy c[16];
    int m = host_copies(ctx, s, false, c);
    {
        // the inputs are staged on the device (copy kernels over the device
        // mapping of page-locked arrays, the driver's copy otherwise), so the
        // build's scattered reads stay in HBM
        NvtxScope r("sph.stage_in");
        if ((rc = spread_copies(ctx, c, m, true, st))) return rc;
    }
    for (int it = 0; it + 1 < nsteps; ++it)
        if ((rc = step_once(ctx, &ctx->hs, &ctx->hs, st))) return rc;
    // every array page-locked: the last step writes the host state directly
    // through its device mapping (the stores cross the host link overlapped
    // with the arithmetic instead of a copy after the step)
    sph_state z = *s;
    bool all = true;
    auto map = [&](void *h) -> void * {
        if (!h) return nullptr;
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, h) != cudaSuccess || at.type != cudaMemoryTypeHost) {
            cudaGetLastError();  // (an unregistered pointer is not an error here)
            all = false;
            return nullptr;
        }
        return at.devicePointer;
    };
    for (int k = 0; k < 3; ++k) {
        z.r[k] = static_cast<double *>(map(s->r[k]));
        z.v[k] = map(s->v[k]);
    }
    z.rho = map(s->rho);
    z.p = map(s->p);
    z.id = static_cast<uint32_t *>(map(s->id));
    z.kind = static_cast<uint8_t *>(map(s->kind));
    z.radius = map(s->radius);
    z.mass = map(s->mass);
    if (all) {
        if ((rc = step_once(ctx, &ctx->hs, &z, st))) return rc;
    } else {
        if ((rc = step_once(ctx, &ctx->hs, &ctx->hs, st))) return rc;
        m = host_copies(ctx, s, true, c);
        if ((rc = spread_copies(ctx, c, m, false, st))) return rc;
    }
    return host_diag(ctx, diag, st);
}

// The buffers holding the products of a build + density pass for n
// particles (what the reverse step reads), in a fixed order (the views of
// sph_adjoint_of_saved follow it).
struct Section {
    void *p;
    size_t bytes;
};
static int build_sections(const sph_ctx *ctx, int n, Section *sec)
{
    const size_t N = (size_t)n, tsz = ctx->f32 ? 4 : 8;
    int m = 0;
    sec[m++] = {ctx->sb.pos, N * 4 * tsz};
    sec[m++] = {ctx->sb.vel, N * 4 * tsz};
    sec[m++] = {ctx->sb.phat, N * tsz};
    sec[m++] = {ctx->sb.kind_s, N};
    sec[m++] = {ctx->sb.cell_s, N * 4};
    sec[m++] = {ctx->sb.src, N * 4};
    sec[m++] = {ctx->sb.ovf, N};
    sec[m++] = {ctx->sb.nnb, N * 2};
    sec[m++] = {ctx->sb.mask, mask_words(ctx->prm.dim, N) * 4};
    sec[m++] = {ctx->cb.cell_start, ((size_t)ctx->cb.ncells + 1) * 4};
    return m;
}
static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int sph_build_save(sph_ctx *ctx, void *dst, int64_t *bytes, sph_stream_t stream)
{
    if (!ctx || !bytes) return SPH_ERR_INVALID;
    if (model_1a(ctx) || model_dem(ctx) || model_fields(ctx))
        return fail(ctx, SPH_ERR_INVALID, "sph_build_save covers SPH_MODEL_WCSPH only");
    if (ctx->dens_n < 0) return fail(ctx, SPH_ERR_INVALID, "sph_build_save: no density pass since the last build");
    Section sec[16];
    const int m = build_sections(ctx, ctx->dens_n, sec);
    size_t total = 0;
    for (int k = 0; k < m; ++k) total += align256(sec[k].bytes);
    *bytes = (int64_t)total;
    if (!dst) return SPH_OK;
    if (reinterpret_cast<uintptr_t>(dst) & 255u) return fail(ctx, SPH_ERR_INVALID, "sph_build_save: dst not 256-byte aligned");
    char *d = static_cast<char *>(dst);
    CopySections cs{};
    for (int k = 0; k < m; ++k) {
        cs.src[cs.m] = sec[k].p;
        cs.dst[cs.m] = d;
        cs.bytes[cs.m] = sec[k].bytes;
        ++cs.m;
        d += align256(sec[k].bytes);
    }
    CK(launch_copy_sections(cs, (cudaStream_t)stream));  // one launch for all sections
    return SPH_OK;
}

int sph_build_load(sph_ctx *ctx, const void *src, int n, sph_stream_t stream)
{
    if (!ctx || !src) return SPH_ERR_INVALID;
    if (model_1a(ctx) || model_dem(ctx) || model_fields(ctx))
        return fail(ctx, SPH_ERR_INVALID, "sph_build_load covers SPH_MODEL_WCSPH only");
    if (n < 0 || n > ctx->cap) return fail(ctx, SPH_ERR_CAPACITY, "sph_build_load: bad particle count");
    if (reinterpret_cast<uintptr_t>(src) & 255u) return fail(ctx, SPH_ERR_INVALID, "sph_build_load: src not 256-byte aligned");
    Section sec[16];
    const int m = build_sections(ctx, n, sec);
    const char *s = static_cast<const char *>(src);
    CopySections cs{};
    for (int k = 0; k < m; ++k) {
        cs.src[cs.m] = s;
        cs.dst[cs.m] = sec[k].p;
        cs.bytes[cs.m] = sec[k].bytes;
        ++cs.m;
        s += align256(sec[k].bytes);
    }
    CK(launch_copy_sections(cs, (cudaStream_t)stream));
    ctx->cells_current = false;  // the caller's state is not known to match
    ctx->cells_n = n;
    ctx->dens_n = n;
    return SPH_OK;
}

int sph_adjoint_of_build(sph_ctx *ctx, int n, const sph_grad *g_np1, sph_grad *g_n, double *alpha_bar,
                         sph_stream_t stream)
{
    if (!ctx) return SPH_ERR_INVALID;
    if (!g_np1 || !g_n) return fail(ctx, SPH_ERR_INVALID, "NULL gradient");
    if (model_1a(ctx) || model_dem(ctx) || model_fields(ctx))
        return fail(ctx, SPH_ERR_INVALID, "the adjoint covers SPH_MODEL_WCSPH only");
    if (ctx->dp.adaptive) return fail(ctx, SPH_ERR_INVALID, "the adjoint takes a fixed dt (SPH_DT_FIXED)");
    if (ctx->dens_n != n)
        return fail(ctx, SPH_ERR_INVALID, "sph_adjoint_of_build: no build products of n particles (sph_build_load)");
    if (n > 0) {
        for (int k = 0; k < ctx->prm.dim; ++k) {
            if (!g_np1->r_bar[k] || !g_np1->v_bar[k] || !g_n->r_bar[k] || !g_n->v_bar[k])
                return fail(ctx, SPH_ERR_INVALID, "NULL gradient component");
            if (g_np1->r_bar[k] == g_n->r_bar[k] || g_np1->v_bar[k] == g_n->v_bar[k])
                return fail(ctx, SPH_ERR_INVALID, "g_n aliases g_np1");
        }
    }
    NvtxScope range("sph_adjoint_of_build");
    CK(launch_adjoint(ctx->dp, ctx->f32, n, ctx->cb, ctx->sb, ctx->ab, *g_np1, *g_n, alpha_bar,
                      (cudaStream_t)stream));
    return SPH_OK;
}

int sph_adjoint_of_saved(sph_ctx *ctx, const void *saved, int n, const sph_grad *g_np1, sph_grad *g_n,
                         double *alpha_bar, sph_stream_t stream)
{
    if (!ctx) return SPH_ERR_INVALID;
    if (!g_np1 || !g_n) return fail(ctx, SPH_ERR_INVALID, "NULL gradient");
    if (model_1a(ctx) || model_dem(ctx) || model_fields(ctx))
        return fail(ctx, SPH_ERR_INVALID, "the adjoint covers SPH_MODEL_WCSPH only");
    if (ctx->dp.adaptive) return fail(ctx, SPH_ERR_INVALID, "the adjoint takes a fixed dt (SPH_DT_FIXED)");
    if (n < 0 || n > ctx->cap) return fail(ctx, SPH_ERR_CAPACITY, "sph_adjoint_of_saved: bad particle count");
    if (n > 0 && !saved) return fail(ctx, SPH_ERR_INVALID, "sph_adjoint_of_saved: saved is NULL");
    if (reinterpret_cast<uintptr_t>(saved) & 255u)
        return fail(ctx, SPH_ERR_INVALID, "sph_adjoint_of_saved: saved not 256-byte aligned");
    if (n > 0) {
        for (int k = 0; k < ctx->prm.dim; ++k) {
            if (!g_np1->r_bar[k] || !g_np1->v_bar[k] || !g_n->r_bar[k] || !g_n->v_bar[k])
                return fail(ctx, SPH_ERR_INVALID, "NULL gradient component");
            if (g_np1->r_bar[k] == g_n->r_bar[k] || g_np1->v_bar[k] == g_n->v_bar[k])
                return fail(ctx, SPH_ERR_INVALID, "g_n aliases g_np1");
        }
    }
    // views of the saved products, in the order and alignment of
    // sph_build_save (the reverse step only reads them)
    Section sec[16];
    const int m = build_sections(ctx, n, sec);
    SortedBufs sb = ctx->sb;
    CellBufs cb = ctx->cb;
    void **view[10] = {&sb.pos,
                       &sb.vel,
                       &sb.phat,
                       reinterpret_cast<void **>(&sb.kind_s),
                       reinterpret_cast<void **>(&sb.cell_s),
                       reinterpret_cast<void **>(&sb.src),
                       reinterpret_cast<void **>(&sb.ovf),
                       reinterpret_cast<void **>(&sb.nnb),
                       reinterpret_cast<void **>(&sb.mask),
                       reinterpret_cast<void **>(&cb.cell_start)};
    if (m != 10) return fail(ctx, SPH_ERR_INVALID, "sph_adjoint_of_saved: section layout");
    const char *p = static_cast<const char *>(saved);
    for (int k = 0; k < m; ++k) {
        *view[k] = const_cast<char *>(p);
        p += align256(sec[k].bytes);
    }
    NvtxScope range("sph_adjoint_of_saved");
    CK(launch_adjoint(ctx->dp, ctx->f32, n, cb, sb, ctx->ab, *g_np1, *g_n, alpha_bar, (cudaStream_t)stream));
    return SPH_OK;
}

int sph_step_adjoint(sph_ctx *ctx, const sph_state *s_n, const sph_grad *g_np1, sph_grad *g_n,
                     double *alpha_bar, sph_stream_t stream)
{
    int rc = check_state(ctx, s_n);
    if (rc) return rc;
    if (!g_np1 || !g_n) return fail(ctx, SPH_ERR_INVALID, "NULL gradient");
    if (model_1a(ctx) || model_dem(ctx)) return fail(ctx, SPH_ERR_INVALID, "the adjoint covers SPH_MODEL_WCSPH only");
    if (ctx->dp.adaptive) return fail(ctx, SPH_ERR_INVALID, "the adjoint takes a fixed dt (SPH_DT_FIXED)");
    if (s_n->n > 0) {
        for (int k = 0; k < ctx->prm.dim; ++k) {
            if (!g_np1->r_bar[k] || !g_np1->v_bar[k] || !g_n->r_bar[k] || !g_n->v_bar[k])
                return fail(ctx, SPH_ERR_INVALID, "NULL gradient component");
            if (g_np1->r_bar[k] == g_n->r_bar[k] || g_np1->v_bar[k] == g_n->v_bar[k])
                return fail(ctx, SPH_ERR_INVALID, "g_n aliases g_np1");
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    NvtxScope range("sph_step_adjoint");
    if ((rc = build(ctx, s_n, st))) return rc;
    CK(launch_density(ctx->dp, ctx->f32, s_n->n, ctx->cb, ctx->sb, nullptr, nullptr, ctx->acc, st));
    ctx->dens_n = s_n->n;
    CK(launch_adjoint(ctx->dp, ctx->f32, s_n->n, ctx->cb, ctx->sb, ctx->ab, *g_np1, *g_n, alpha_bar, st));
    return SPH_OK;
}

int sph_sample(sph_ctx *ctx, const void *A, const void *m, const void *rho, void *S, sph_stream_t stream)
{
    if (!ctx) return SPH_ERR_INVALID;
    if (!ctx->cells_current)
        return fail(ctx, SPH_ERR_INVALID,
                    "sph_sample needs the cells of the particles' current positions: call sph_build_cells first");
    if (ctx->cells_n > 0 && (!A || !m || !rho || !S)) return fail(ctx, SPH_ERR_INVALID, "NULL field");
    if (ctx->dp.K != 1)
        return fail(ctx, SPH_ERR_INVALID, "sph_sample walks the 3^D stencil: it needs cells of edge cs >= 2h");
    CK(launch_sample(ctx->dp, ctx->f32, ctx->cells_n, ctx->cb, ctx->sb, A, m, rho, S, (cudaStream_t)stream));
    return SPH_OK;
}

int sph_reorder_field(sph_ctx *ctx, const void *in, void *out, int elem_bytes, sph_stream_t stream)
{
    if (!ctx) return SPH_ERR_INVALID;
    if (!(elem_bytes == 4 || elem_bytes == 8 || elem_bytes == 12 || elem_bytes == 16 || elem_bytes == 24 ||
          elem_bytes == 32))
        return fail(ctx, SPH_ERR_INVALID, "elem_bytes must be 4, 8, 12, 16, 24 or 32");
    if (!ctx->cells_current)
        return fail(ctx, SPH_ERR_INVALID, "sph_reorder_field needs a build (sph_build_cells) first");
    if (ctx->cells_n > 0 && (!in || !out)) return fail(ctx, SPH_ERR_INVALID, "NULL field");
    const char *a = static_cast<const char *>(in);
    const char *b = static_cast<const char *>(out);
    const size_t bytes = (size_t)ctx->cells_n * (size_t)elem_bytes;
    if (ctx->cells_n > 0 && a < b + bytes && b < a + bytes)
        return fail(ctx, SPH_ERR_INVALID, "sph_reorder_field: in and out overlap");
    CK(launch_reorder_field(ctx->cells_n, ctx->sb.src, in, out, elem_bytes, (cudaStream_t)stream));
    return SPH_OK;
}

// [a, a + bytes) and [b, b + bytes) overlap
static bool overlap(const void *a, const void *b, size_t bytes)
{
    const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
    return x < y + bytes && y < x + bytes;
}

int sph_build_cells_into(sph_ctx *ctx, const sph_state *in, sph_state *out, int nfields, const void *const *fin,
                         void *const *fout, int elem_bytes, sph_stream_t stream)
{
    int rc = check_state(ctx, in);
    if (rc) return rc;
    if (!model_fields(ctx)) return fail(ctx, SPH_ERR_INVALID, "sph_build_cells_into serves SPH_MODEL_FIELDS");
    if (!out || out->n != in->n) return fail(ctx, SPH_ERR_INVALID, "out must be a state of in->n particles");
    if (nfields < 0 || (nfields > 0 && (!fin || !fout)))
        return fail(ctx, SPH_ERR_INVALID, "bad field list");
    if (nfields > 0 && elem_bytes != 4 && elem_bytes != 8)
        return fail(ctx, SPH_ERR_INVALID, "elem_bytes must be 4 or 8");
    const size_t n = (size_t)in->n;
    if (n > 0) {
        for (int k = 0; k < ctx->prm.dim; ++k) {
            if (!out->r[k]) return fail(ctx, SPH_ERR_INVALID, "NULL output position");
            for (int q = 0; q < ctx->prm.dim; ++q)
                if (overlap(out->r[k], in->r[q], n * 8)) return fail(ctx, SPH_ERR_INVALID, "out overlaps in");
        }
        if (!out->id || !out->kind) return fail(ctx, SPH_ERR_INVALID, "NULL output id or kind");
        if (overlap(out->id, in->id, n * 4) || overlap(out->kind, in->kind, n))
            return fail(ctx, SPH_ERR_INVALID, "out overlaps in");
        const size_t fb = n * (size_t)elem_bytes;
        for (int f = 0; f < nfields; ++f) {
            if (!fin[f] || !fout[f]) return fail(ctx, SPH_ERR_INVALID, "NULL field");
            for (int g = 0; g < nfields; ++g) {
                if (overlap(fout[f], fin[g], fb) || (g != f && overlap(fout[f], fout[g], fb)))
                    return fail(ctx, SPH_ERR_INVALID, "sph_build_cells_into: a field output overlaps");
            }
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    SortedBufs sbx = ctx->sb;
    for (int k = 0; k < ctx->prm.dim; ++k) sbx.rs[k] = out->r[k];
    sbx.id_s = out->id;
    sbx.kind_s = out->kind;
    FieldSet fs{};
    fs.nf = nfields < kMaxFields ? nfields : kMaxFields;
    for (int f = 0; f < fs.nf; ++f) {
        fs.in[f] = static_cast<const uint32_t *>(fin[f]);
        fs.out[f] = static_cast<uint32_t *>(fout[f]);
    }
    ctx->cells_current = false;
    ctx->dens_n = -1;
    {
        NvtxScope r("sph.build");
        CK(launch_build_into(ctx->dp, ctx->f32, in->n, *in, ctx->cb, sbx, fs, elem_bytes ? elem_bytes : 4,
                             ctx->status, st));
    }
    mark_current(ctx, out);
    // fields beyond the first kMaxFields: through the permutation
    for (int f0 = kMaxFields; f0 < nfields; f0 += kMaxFields) {
        FieldSet rest{};
        rest.nf = nfields - f0 < kMaxFields ? nfields - f0 : kMaxFields;
        for (int f = 0; f < rest.nf; ++f) {
            rest.in[f] = static_cast<const uint32_t *>(fin[f0 + f]);
            rest.out[f] = static_cast<uint32_t *>(fout[f0 + f]);
        }
        CK(launch_reorder_fields(in->n, ctx->sb.src, rest, elem_bytes, st));
    }
    return SPH_OK;
}

int sph_reorder_fields(sph_ctx *ctx, int nfields, const void *const *in, void *const *out, int elem_bytes,
                       sph_stream_t stream)
{
    if (!ctx) return SPH_ERR_INVALID;
    if (nfields < 0) return fail(ctx, SPH_ERR_INVALID, "negative field count");
    if (nfields == 0) return SPH_OK;
    if (!in || !out) return fail(ctx, SPH_ERR_INVALID, "NULL field list");
    if (!(elem_bytes == 4 || elem_bytes == 8 || elem_bytes == 12 || elem_bytes == 16 || elem_bytes == 24 ||
          elem_bytes == 32))
        return fail(ctx, SPH_ERR_INVALID, "elem_bytes must be 4, 8, 12, 16, 24 or 32");
    if (!ctx->cells_current)
        return fail(ctx, SPH_ERR_INVALID, "sph_reorder_fields needs a build (sph_build_cells) first");
    const size_t bytes = (size_t)ctx->cells_n * (size_t)elem_bytes;
    if (ctx->cells_n > 0) {
        // every output must be disjoint from every input and every other output
        for (int f = 0; f < nfields; ++f) {
            if (!in[f] || !out[f]) return fail(ctx, SPH_ERR_INVALID, "NULL field");
            const char *b = static_cast<const char *>(out[f]);
            for (int g = 0; g < nfields; ++g) {
                const char *a = static_cast<const char *>(in[g]);
                if (a < b + bytes && b < a + bytes)
                    return fail(ctx, SPH_ERR_INVALID, "sph_reorder_fields: an output overlaps an input");
                const char *c = static_cast<const char *>(out[g]);
                if (g != f && c < b + bytes && b < c + bytes)
                    return fail(ctx, SPH_ERR_INVALID, "sph_reorder_fields: two outputs overlap");
            }
        }
    }
    for (int f0 = 0; f0 < nfields; f0 += kMaxFields) {
        FieldSet fs{};
        fs.nf = nfields - f0 < kMaxFields ? nfields - f0 : kMaxFields;
        for (int f = 0; f < fs.nf; ++f) {
            fs.in[f] = static_cast<const uint32_t *>(in[f0 + f]);
            fs.out[f] = static_cast<uint32_t *>(out[f0 + f]);
        }
        CK(launch_reorder_fields(ctx->cells_n, ctx->sb.src, fs, elem_bytes, (cudaStream_t)stream));
    }
    return SPH_OK;
}

int sph_law_view(sph_ctx *ctx, sph_law_views *out)
{
    if (!ctx || !out) return SPH_ERR_INVALID;
    if (!ctx->cells_current) return fail(ctx, SPH_ERR_INVALID, "sph_law_view needs a build (sph_build_cells) first");
    out->pos = ctx->sb.pos;
    out->cell_s = ctx->sb.cell_s;
    out->cell_start = ctx->cb.cell_start;
    out->params = &ctx->dp;
    out->params_bytes = (int64_t)sizeof(DevParams);
    out->n = ctx->cells_n;
    out->precision = ctx->prm.precision;
    out->mask = ctx->sb.mask;
    out->nnb = ctx->sb.nnb;
    out->ovf = ctx->sb.ovf;
    return SPH_OK;
}

int sph_clock_get(sph_ctx *ctx, double *dt_next, double *time, sph_stream_t stream)
{
    if (!ctx) return SPH_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(ctx->diag_host, ctx->diag_dev, sizeof(DiagDev), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (dt_next) *dt_next = ctx->dp.adaptive ? ctx->diag_host->dt_next : ctx->prm.dt;
    if (time) *time = ctx->diag_host->time;
    return SPH_OK;
}

int sph_clock_set(sph_ctx *ctx, double dt_next, double time, sph_stream_t stream)
{
    if (!ctx) return SPH_ERR_INVALID;
    if (!std::isfinite(time) || !std::isfinite(dt_next)) return fail(ctx, SPH_ERR_INVALID, "non-finite clock");
    if (ctx->dp.adaptive ? !(dt_next > 0.0 && dt_next <= ctx->prm.dt) : dt_next != ctx->prm.dt)
        return fail(ctx, SPH_ERR_INVALID, "dt_next outside (0, params.dt] (params.dt itself for a fixed dt)");
    cudaStream_t st = (cudaStream_t)stream;
    // (two doubles of the device record, from a pinned staging slot that
    // the stream orders: the host record is not used by the device)
    CK(cudaStreamSynchronize(st));
    ctx->diag_host->dt_next = dt_next;
    ctx->diag_host->time = time;
    CK(cudaMemcpyAsync(&ctx->diag_dev->time, &ctx->diag_host->time, sizeof(double), cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(&ctx->diag_dev->dt_next, &ctx->diag_host->dt_next, sizeof(double), cudaMemcpyHostToDevice,
                       st));
    CK(cudaStreamSynchronize(st));
    return SPH_OK;
}

int sph_tank_set(sph_ctx *ctx, double Z, double Zdot, sph_stream_t stream)
{
    if (!ctx) return SPH_ERR_INVALID;
    if (!ctx->tank) return fail(ctx, SPH_ERR_INVALID, "the context has no tank (SPH_MODEL_DEM only)");
    TankDev t{};
    t.Z = Z;
    t.Zdot = Zdot;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(ctx->tank, &t, sizeof(t), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));  // t lives on this stack
    return SPH_OK;
}

int sph_tank_get(sph_ctx *ctx, double *Z, double *Zdot, double *Zddot, double *F_wall, sph_stream_t stream)
{
    if (!ctx) return SPH_ERR_INVALID;
    if (!ctx->tank) return fail(ctx, SPH_ERR_INVALID, "the context has no tank (SPH_MODEL_DEM only)");
    cudaStream_t st = (cudaStream_t)stream;
    TankDev t{};
    CK(cudaMemcpyAsync(&t, ctx->tank, sizeof(t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (Z) *Z = t.Z;
    if (Zdot) *Zdot = t.Zdot;
    if (Zddot) *Zddot = t.Zddot;
    if (F_wall)
        for (int k = 0; k < 3; ++k) F_wall[k] = t.Fb[k];
    return SPH_OK;
}

int sph_get_status(sph_ctx *ctx, uint32_t *out, int sync, sph_stream_t stream)
{
    if (!ctx || !out) return SPH_ERR_INVALID;
    cudaStream_t st = (cudaStream_t)stream;
    if (sync) CK(cudaStreamSynchronize(st));
    uint32_t v = 0;
    CK(cudaMemcpy(&v, ctx->status, sizeof(v), cudaMemcpyDeviceToHost));
    CK(cudaMemset(ctx->status, 0, sizeof(uint32_t)));
    *out = v;
    return SPH_OK;
}

int sph_profile_begin(sph_ctx *ctx, int max_steps)
{
    if (!ctx || max_steps < 1 || max_steps > (1 << 20)) return SPH_ERR_INVALID;
    size_t need = (size_t)max_steps * kEvPerStep;
    while (ctx->ev.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        ctx->ev.push_back(e);
    }
    ctx->prof_cap = max_steps;
    ctx->prof_steps = 0;
    ctx->prof_on = true;
    return SPH_OK;
}

int sph_profile_end(sph_ctx *ctx, double *ms, int64_t *steps)
{
    if (!ctx || !ms || !steps) return SPH_ERR_INVALID;
    ctx->prof_on = false;
    for (int k = 0; k < SPH_PROF_NPHASE; ++k) ms[k] = 0.0;
    *steps = ctx->prof_steps;
    if (ctx->prof_steps == 0) return SPH_OK;
    CK(cudaEventSynchronize(ctx->ev[(size_t)ctx->prof_steps * kEvPerStep - 1]));
    for (int s = 0; s < ctx->prof_steps; ++s) {
        for (int k = 0; k < SPH_PROF_NPHASE; ++k) {
            float t = 0.f;
            CK(cudaEventElapsedTime(&t, ctx->ev[(size_t)s * kEvPerStep + k], ctx->ev[(size_t)s * kEvPerStep + k + 1]));
            ms[k] += (double)t;
        }
    }
    ctx->prof_steps = 0;
    return SPH_OK;
}

}  // extern "C"
