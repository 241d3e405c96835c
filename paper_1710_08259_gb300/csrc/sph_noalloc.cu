// sph_noalloc.cu -- the neighbour-search build for callers that cannot
// allocate device memory (sph_build_cells_static).
//
// Who needs it.  sph_build_cells works on a context whose workspace
// sph_create obtains with cudaMalloc.  Some callers cannot do that where they
// need a build: code that runs under someone else's allocator (a framework
// whose caching pool owns the device memory and must not be bypassed, or a
// process that reserved all of it up front), loops that must not stall on
// cudaMalloc / cudaFree (both can synchronise the device), and plug-ins that
// are handed only the particle arrays.  This entry point sorts their
// particles and fills the cell start table with no context and no allocation:
// its scratch is one fixed array that the library keeps in device memory.
//
// The array is g_static_scratch below, sized for SPH_STATIC_MAX_PARTICLES
// particles and SPH_STATIC_MAX_CELLS cells (about 11 MB).  Every GPU that
// loads the library holds it until the process exits.  In host code its name
// is only a host-side stand-in; every call asks the runtime for the device
// address with cudaGetSymbolAddress and passes that to the kernels.  The
// first call on a device is the set-up: the lookup may load the library's
// device code there (and with it the array), so it should come before any
// stream capture and before the rest of the device memory is reserved.
// Later lookups are cheap, and asking every time (rather than caching per
// device ordinal) stays right if the device's primary context is torn down
// and recreated, which can move the array.  Every call shares the array, so
// calls that overlap on the GPU (different streams, or different host
// threads) race with each other; each call clears what must start at zero.
#include <cuda_runtime.h>

#include <string>

#include "sph_internal.cuh"

using namespace sph;

namespace {

constexpr size_t kMaxN = SPH_STATIC_MAX_PARTICLES;
constexpr size_t kMaxC = SPH_STATIC_MAX_CELLS;
constexpr size_t kMaxAxis = SPH_STATIC_MAX_AXIS_CELLS;

constexpr size_t al(size_t b) { return (b + 255) / 256 * 256; }

// byte layout of the scratch
constexpr size_t kCountWords = (kMaxC + 2048) / 2048 * 2048 + 2048;
constexpr size_t oKey = 0;
constexpr size_t oRank = oKey + al(4 * kMaxN);
constexpr size_t oTmp = oRank + al(4 * kMaxN);
constexpr size_t oCount = oTmp + al(4 * kMaxN);
constexpr size_t oStart = oCount + al(4 * kCountWords);
constexpr size_t oBlockSums = oStart + al(4 * (kMaxC + 1));
constexpr size_t oPos = oBlockSums + al(4 * (kMaxC / 512 + 2));
constexpr size_t oVel = oPos + al(32 * kMaxN);
constexpr size_t oPhat = oVel + al(32 * kMaxN);
constexpr size_t oRs = oPhat + al(8 * kMaxN);
constexpr size_t oCellS = oRs + 3 * al(8 * kMaxN);
constexpr size_t oIdS = oCellS + al(4 * kMaxN);
constexpr size_t oSrc = oIdS + al(4 * kMaxN);
constexpr size_t oKindS = oSrc + al(4 * kMaxN);
constexpr size_t oBval = oKindS + al(kMaxN);
constexpr size_t oBkey = oBval + 3 * al(8 * (kMaxAxis + 1));
constexpr size_t oStatus = oBkey + 3 * al(8 * (kMaxAxis + 1));
constexpr size_t kScratchBytes = oStatus + 256;

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

namespace {

// The message of the calling thread's last failure (sph_static_last_error):
// one string per host thread, so a failure on another thread never replaces
// or frees the string a caller is reading.
thread_local std::string g_err;

int fail(int code, const std::string &m)
{
    g_err = m;
    return code;
}

// Device address of the scratch on the current device.
int scratch_address(unsigned char **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return fail(SPH_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = static_cast<unsigned char *>(p);
    return SPH_OK;
}

}  // namespace

extern "C" {

const char *sph_static_last_error(void)
{
    return g_err.c_str();
}

int sph_build_cells_static(const sph_params *params, sph_state *s, uint32_t *cell_start, uint32_t *status,
                           sph_stream_t stream)
{
    if (!params || !s) return fail(SPH_ERR_INVALID, "params or state is NULL");
    DevParams d;
    double rho_ref = 0.0;
    std::string why;
    if (!make_dev_params(params, &d, &rho_ref, why)) return fail(SPH_ERR_INVALID, why);
    if (s->n < 0) return fail(SPH_ERR_INVALID, "negative particle count");
    if ((size_t)s->n > kMaxN)
        return fail(SPH_ERR_CAPACITY, "sph_build_cells_static: " + std::to_string(s->n) +
                                          " particles exceed the static limit of " + std::to_string(kMaxN));
    size_t ncells = 1;
    for (int k = 0; k < params->dim; ++k) {
        if ((size_t)params->ncell[k] > kMaxAxis)
            return fail(SPH_ERR_CAPACITY, "sph_build_cells_static: " + std::to_string(params->ncell[k]) +
                                              " cells along an axis exceed the static limit of " +
                                              std::to_string(kMaxAxis));
        ncells *= (size_t)params->ncell[k];
    }
    if (ncells > kMaxC)
        return fail(SPH_ERR_CAPACITY, "sph_build_cells_static: " + std::to_string(ncells) +
                                          " cells exceed the static limit of " + std::to_string(kMaxC));
    if (s->n > 0) {
        // (the field model carries no velocity, as in sph_build_cells)
        const bool need_v = params->model != SPH_MODEL_FIELDS;
        for (int k = 0; k < params->dim; ++k)
            if (!s->r[k] || (need_v && !s->v[k])) return fail(SPH_ERR_INVALID, "NULL r or v component");
        if (!s->id || !s->kind) return fail(SPH_ERR_INVALID, "NULL id or kind");
    }
    unsigned char *base = nullptr;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const bool f32 = params->precision == SPH_PREC_F32;

    CellBufs cb{};
    cb.key = reinterpret_cast<uint32_t *>(base + oKey);
    cb.rank = reinterpret_cast<uint32_t *>(base + oRank);
    cb.tmp = reinterpret_cast<uint32_t *>(base + oTmp);
    cb.cell_count = reinterpret_cast<uint32_t *>(base + oCount);
    cb.cell_start = reinterpret_cast<uint32_t *>(base + oStart);
    cb.block_sums = reinterpret_cast<uint32_t *>(base + oBlockSums);
    cb.ncells = (int64_t)ncells;
    cb.scan_blocks = (int)((ncells + kScanTile - 1) / kScanTile);
    SortedBufs sb{};
    sb.pos = base + oPos;
    sb.vel = base + oVel;
    sb.phat = base + oPhat;
    for (int k = 0; k < 3; ++k) sb.rs[k] = reinterpret_cast<double *>(base + oRs + k * al(8 * kMaxN));
    sb.cell_s = reinterpret_cast<uint32_t *>(base + oCellS);
    sb.id_s = reinterpret_cast<uint32_t *>(base + oIdS);
    sb.src = reinterpret_cast<uint32_t *>(base + oSrc);
    sb.kind_s = base + oKindS;
    sb.mask = nullptr;
    sb.ovf = nullptr;
    double *bval[3];
    long long *bkey[3];
    for (int k = 0; k < 3; ++k) {
        bval[k] = reinterpret_cast<double *>(base + oBval + k * al(8 * (kMaxAxis + 1)));
        bkey[k] = reinterpret_cast<long long *>(base + oBkey + k * al(8 * (kMaxAxis + 1)));
        d.bval[k] = bval[k];
        d.bkey[k] = bkey[k];
    }
    uint32_t *stat = reinterpret_cast<uint32_t *>(base + oStatus);
    d.chk_status = stat;  // used by bounds-checked builds only
    d.chk_cap = (uint32_t)s->n;

    // what must start at zero: the cell counts (consumed by the scan) and the
    // status word; the rest is fully rewritten by this call
    const size_t count_words = (size_t)cb.scan_blocks * kScanTile;
    cudaError_t e = cudaMemsetAsync(cb.cell_count, 0, count_words * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(stat, 0, 4, st);
    if (e == cudaSuccess) e = launch_base_tables(d, bval, bkey, st);
    if (e == cudaSuccess) e = launch_build(d, f32, s->n, *s, cb, sb, stat, st);
    if (e == cudaSuccess) e = launch_writeback(d, f32, s->n, *s, sb, st);
    if (e == cudaSuccess && cell_start)
        e = cudaMemcpyAsync(cell_start, cb.cell_start, (ncells + 1) * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && status) e = cudaMemcpyAsync(status, stat, 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(SPH_ERR_CUDA, std::string("sph_build_cells_static: ") + cudaGetErrorString(e));
    return SPH_OK;
}

}  // extern "C"
