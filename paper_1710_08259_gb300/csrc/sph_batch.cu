// sph_batch.cu -- many independent WCSPH cases advanced together by one
// persistent cooperative kernel (sph_batch_step), captured in a CUDA graph.
//
// The cases (arXiv:1710.08259 Example 1a style dam breaks of uneven size) are
// packed one after another in a single state: case c owns particles
// [off_c, off_c + n_c) and cells [cell_off_c, cell_off_c + ncells_c) of one
// shared cell table.  Because every case's particles and cells are contiguous
// and in case order, ONE exclusive scan over the shared count table gives
// every case's cell start table in packed particle indices, and every phase
// runs over all cases at once: a thread takes the constants of its particle's
// case (DevParams of that case) and otherwise executes exactly the per-phase
// bodies of the one-case path (sph_phases.cuh), so a batched case evolves bit
// for bit like the same case stepped alone.
//
// One launch runs nsteps steps; the phases of a step are separated by a
// software grid barrier (all blocks are co-resident: cooperative launch).
// Each barrier spins a bounded number of times; past the limit the block sets
// SPH_STATUS_BARRIER_TIMEOUT and an abort flag, and every block leaves the
// kernel at its next barrier, so a lost block can never hang the GPU.
// Work in the pair phases is split in tiles of blockDim particles taken in
// grid-stride order, which balances uneven cases by particle count.
//
// The phased form (sph_tune.form = SPH_BATCH_PHASED) runs the same phase
// bodies as one ordinary launch per phase, captured in the same kind of
// graph: no barrier, and every phase gets its own launch shape and register
// budget.  The autotuner times both forms.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "sph_internal.cuh"
#include "sph_phases.cuh"

using namespace sph;

namespace sph {

struct BarrierState {
    unsigned int count;
    unsigned int gen;
    unsigned int abort;
    unsigned int pad;
};

// Grid-wide barrier with a bounded wait.  Returns false when the kernel must
// stop (a timeout here or in another block).
__device__ __forceinline__ bool grid_barrier(BarrierState *b, long long limit, uint32_t *status)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int g = atomicAdd(&b->gen, 0u);
        __threadfence();
        if (atomicAdd(&b->count, 1u) == gridDim.x - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            long long it = 0;
            while (atomicAdd(&b->gen, 0u) == g) {
                if (atomicAdd(&b->abort, 0u)) {
                    ok = 0;
                    break;
                }
                if (++it > limit) {
                    atomicOr(status, SPH_STATUS_BARRIER_TIMEOUT);
                    atomicExch(&b->abort, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        if (atomicAdd(&b->abort, 0u)) ok = 0;
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

struct BatchArgs {
    int n;
    int ncases;
    const DevParams *cp;
    const uint16_t *case_of;
    sph_state s;
    CellBufs cb;
    SortedBufs sb;
    int ntiles_scan;
    unsigned long long *vmax2;  // per case
    unsigned long long *amax2;  // per case
    DiagDev *diag;              // per case, after the last step
    unsigned long long *n_pairs;
    uint32_t *status;
    BarrierState *bar;
    long long spin_limit;
    int nsteps;
    int selftest;  // 1: block 0 never reaches the first barrier (barrier timeout test)
};

// ---- the phases of one step over all cases.  Every loop is grid-stride,
// so the same body serves the persistent kernel (a grid of resident blocks,
// phases separated by grid barriers) and the phased form (one launch per
// phase with a grid covering the work).

template <int D>
__device__ __forceinline__ void bp_hash(const BatchArgs &A)
{
    // warp-uniform trip count for the match/ballot inside
    const int lane = threadIdx.x & 31;
    const int nthreads = gridDim.x * blockDim.x;
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) - lane; base < A.n; base += nthreads) {
        const int k = base + lane;
        const bool act = k < A.n;
        const DevParams &P = A.cp[act ? A.case_of[k] : 0];
        dev_hash<D>(P, k, act, A.s, A.cb.key, A.cb.rank, A.cb.cell_count, A.status);
    }
}

__device__ __forceinline__ void bp_scan_reduce(const BatchArgs &A, uint32_t *ws)
{
    for (int t = blockIdx.x; t < A.ntiles_scan; t += gridDim.x) dev_scan_reduce(A.cb.cell_count, A.cb.block_sums, t, ws);
}

__device__ __forceinline__ void bp_scan_apply(const BatchArgs &A, uint32_t *ws)
{
    for (int t = blockIdx.x; t < A.ntiles_scan; t += gridDim.x)
        dev_scan_apply(A.cb.cell_count, A.cb.block_sums, A.cb.cell_start, A.cb.ncells, t, ws);
}

__device__ __forceinline__ void bp_scatter(const BatchArgs &A)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < A.n; k += gridDim.x * blockDim.x)
        dev_scatter(k, A.cb.key, A.cb.rank, A.cb.cell_start, A.cb.tmp);
}

template <int D, typename T>
__device__ __forceinline__ void bp_gather(const BatchArgs &A)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < A.n; t += gridDim.x * blockDim.x) {
        const DevParams &P = A.cp[A.case_of[A.cb.tmp[t]]];
        dev_order_gather<D, T>(P, t, A.s, A.cb.key, A.cb.cell_start, A.cb.tmp, A.sb, A.status);
    }
}

// density + EOS over tiles of blockDim particles
template <int D, typename T, int K>
__device__ __forceinline__ void bp_density(const BatchArgs &A)
{
    constexpr int NC = Sten<D, K>::NC;
    using V4 = vec4_t<T>;
    const int bd = blockDim.x, tid = threadIdx.x;
    const V4 *pos = static_cast<const V4 *>(A.sb.pos);
    V4 *vel = static_cast<V4 *>(A.sb.vel);
    T *phat = static_cast<T *>(A.sb.phat);
    unsigned long long pairs = 0;
    for (int tile = blockIdx.x; (long long)tile * bd < A.n; tile += gridDim.x) {
        const int i = tile * bd + tid;
        if (i < A.n)
            pairs += dev_density<D, T, K>(A.cp[A.case_of[i]], i, pos, A.sb.cell_s, A.cb.cell_start, vel, phat,
                                       static_cast<T *>(A.s.rho), static_cast<T *>(A.s.p),
                                       A.sb.mask + (size_t)tile * NC * bd + tid, bd, A.sb.ovf, A.sb.nnb);
    }
    pairs = warp_sum(pairs);
    if ((tid & 31) == 0 && pairs) atomicAdd(A.n_pairs, pairs);
}

// forces + integration; per-case maxima of |v|^2, |a|^2
template <int D, typename T, int K>
__device__ __forceinline__ void bp_force(const BatchArgs &A)
{
    constexpr int NC = Sten<D, K>::NC;
    using V4 = vec4_t<T>;
    const int bd = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    const V4 *pos = static_cast<const V4 *>(A.sb.pos);
    V4 *vel = static_cast<V4 *>(A.sb.vel);
    T *phat = static_cast<T *>(A.sb.phat);
    for (int tile = blockIdx.x; (long long)tile * bd < A.n; tile += gridDim.x) {
        const int i = tile * bd + tid;
        const bool act = i < A.n;
        ForceOut<T> o{(T)0, (T)0, 0u, false};
        unsigned int cid = 0;
        if (act) {
            cid = A.case_of[i];
            o = dev_force<D, T, true, K>(A.cp[cid], i, pos, vel, phat, A.sb.cell_s, A.cb.cell_start,
                                      A.sb.mask + (size_t)tile * NC * bd + tid, bd, A.sb.ovf, A.sb, A.s, nullptr,
                                      nullptr, nullptr);
            if (o.bad) atomicOr(A.status, SPH_STATUS_NAN);
        }
        const unsigned act_mask = __ballot_sync(0xffffffffu, act);
        if (act) {
            const unsigned peers = __match_any_sync(act_mask, cid);
            T mv = o.v2, ma = o.a2;
            if (peers == act_mask) {
                // whole warp in one case (the common case): shuffle reduction
                for (int off = 16; off > 0; off >>= 1) {
                    const T ov = __shfl_xor_sync(act_mask, mv, off);
                    const T oa = __shfl_xor_sync(act_mask, ma, off);
                    if ((act_mask >> (lane ^ off)) & 1u) {
                        mv = fmax(mv, ov);
                        ma = fmax(ma, oa);
                    }
                }
                if (lane == __ffs(act_mask) - 1) {
                    raise_max(&A.vmax2[cid], (double)mv);
                    raise_max(&A.amax2[cid], (double)ma);
                }
            } else {
                raise_max(&A.vmax2[cid], (double)mv);
                raise_max(&A.amax2[cid], (double)ma);
            }
        }
    }
}

// per-case CFL check of a step (one block), then the maxima restart
__device__ __forceinline__ void bp_cfl(const BatchArgs &A, int step)
{
    for (int c = threadIdx.x; c < A.ncases; c += blockDim.x) {
        const DevParams &P = A.cp[c];
        const double vmax = sqrt(__longlong_as_double((long long)A.vmax2[c]));
        const double amax = sqrt(__longlong_as_double((long long)A.amax2[c]));
        const double dtc = fmin(0.25 * P.h / (P.c0 + vmax), amax > 0.0 ? 0.25 * sqrt(P.h / amax) : INFINITY);
        if (P.dt > dtc) atomicOr(A.status, SPH_STATUS_CFL);
        if (step == A.nsteps - 1) {
            A.diag[c].vmax = vmax;
            A.diag[c].amax = amax;
            A.diag[c].dt_cfl = dtc;
        }
        A.vmax2[c] = 0;
        A.amax2[c] = 0;
    }
}

template <int D, typename T, int K>
__device__ __forceinline__ void batch_steps(const BatchArgs &A)
{
    extern __shared__ uint32_t smem[];
    uint32_t *ws = smem;  // 33 words of scan scratch
    if (A.selftest) {
        // a barrier that block 0 never reaches: every other block must give
        // up after spin_limit rounds, flag the timeout and leave
        if (blockIdx.x == 0) return;
        grid_barrier(A.bar, A.spin_limit, A.status);
        return;
    }
    for (int step = 0; step < A.nsteps; ++step) {
        bp_hash<D>(A);
        if (!grid_barrier(A.bar, A.spin_limit, A.status)) return;
        bp_scan_reduce(A, ws);
        if (!grid_barrier(A.bar, A.spin_limit, A.status)) return;
        if (blockIdx.x == 0) dev_scan_top(A.cb.block_sums, A.ntiles_scan, A.cb.cell_start + A.cb.ncells, ws);
        if (!grid_barrier(A.bar, A.spin_limit, A.status)) return;
        bp_scan_apply(A, ws);
        if (!grid_barrier(A.bar, A.spin_limit, A.status)) return;
        bp_scatter(A);
        if (!grid_barrier(A.bar, A.spin_limit, A.status)) return;
        bp_gather<D, T>(A);
        if (!grid_barrier(A.bar, A.spin_limit, A.status)) return;
        bp_density<D, T, K>(A);
        if (!grid_barrier(A.bar, A.spin_limit, A.status)) return;
        bp_force<D, T, K>(A);
        if (!grid_barrier(A.bar, A.spin_limit, A.status)) return;
        // (block 0; the next use of the maxima is several barriers away)
        if (blockIdx.x == 0) bp_cfl(A, step);
    }
}

template <int D, typename T, int K>
__global__ void k_batch(BatchArgs A)
{
    batch_steps<D, T, K>(A);
}

// The 2D FP32 kernel, held to the register budget of 6 resident blocks of
// 256 threads (40 registers, that of the 2D pair kernels at 12 x 128): its
// pair phases are latency-bound and gain more from the occupancy than the
// memory phases lose to a few spills (256-case workload: 1.13 -> 1.04 ms per
// step)
template <int K>
__global__ void __launch_bounds__(256, 6) k_batch_2f(BatchArgs A)
{
    batch_steps<2, float, K>(A);
}

// ---- the phased form: one ordinary launch per phase, no grid barrier; the
// pair phases take the one-case kernels' register budget (blocks of 128, 9
// resident per SM in 3D, 12 in 2D: 1.21 -> 1.10 ms per step of the 256-case
// 2D workload against 9)
constexpr int kPhasedBlock = 128;

template <int D>
__global__ void __launch_bounds__(256) k_bp_hash(BatchArgs A)
{
    bp_hash<D>(A);
}
__global__ void k_bp_scan_reduce(BatchArgs A)
{
    __shared__ uint32_t ws[33];
    bp_scan_reduce(A, ws);
}
__global__ void __launch_bounds__(1024) k_bp_scan_top(BatchArgs A)
{
    __shared__ uint32_t ws[33];
    dev_scan_top(A.cb.block_sums, A.ntiles_scan, A.cb.cell_start + A.cb.ncells, ws);
}
__global__ void k_bp_scan_apply(BatchArgs A)
{
    __shared__ uint32_t ws[33];
    bp_scan_apply(A, ws);
}
__global__ void __launch_bounds__(256) k_bp_scatter(BatchArgs A)
{
    bp_scatter(A);
}
template <int D, typename T>
__global__ void __launch_bounds__(256) k_bp_gather(BatchArgs A)
{
    bp_gather<D, T>(A);
}
template <int D, typename T, int K>
__global__ void __launch_bounds__(kPhasedBlock, sizeof(T) == 4 ? (D == 2 ? 12 : 9) : 4) k_bp_density(BatchArgs A)
{
    bp_density<D, T, K>(A);
}
template <int D, typename T, int K>
__global__ void __launch_bounds__(kPhasedBlock, sizeof(T) == 4 ? (D == 2 ? 12 : 10) : 4) k_bp_force(BatchArgs A)
{
    bp_force<D, T, K>(A);
}
__global__ void __launch_bounds__(256) k_bp_cfl(BatchArgs A, int step)
{
    bp_cfl(A, step);
}

template <int D, typename T, int K>
static cudaError_t phased_steps(const BatchArgs &A, int scan_block, cudaStream_t st)
{
    const int g256 = (A.n + 255) / 256;
    const int tiles = (A.n + kPhasedBlock - 1) / kPhasedBlock;
    for (int step = 0; step < A.nsteps; ++step) {
        k_bp_hash<D><<<g256, 256, 0, st>>>(A);
        k_bp_scan_reduce<<<A.ntiles_scan, scan_block, 0, st>>>(A);
        k_bp_scan_top<<<1, 1024, 0, st>>>(A);
        k_bp_scan_apply<<<A.ntiles_scan, scan_block, 0, st>>>(A);
        k_bp_scatter<<<g256, 256, 0, st>>>(A);
        k_bp_gather<D, T><<<g256, 256, 0, st>>>(A);
        k_bp_density<D, T, K><<<tiles, kPhasedBlock, 0, st>>>(A);
        k_bp_force<D, T, K><<<tiles, kPhasedBlock, 0, st>>>(A);
        k_bp_cfl<<<1, 256, 0, st>>>(A, step);
    }
    return cudaGetLastError();
}

template <int K>
static cudaError_t launch_phased_k(int dim, bool f32, const BatchArgs &A, int scan_block, cudaStream_t st)
{
    if (dim == 2)
        return f32 ? phased_steps<2, float, K>(A, scan_block, st) : phased_steps<2, double, K>(A, scan_block, st);
    return f32 ? phased_steps<3, float, K>(A, scan_block, st) : phased_steps<3, double, K>(A, scan_block, st);
}

static cudaError_t launch_phased(int dim, bool f32, int K, const BatchArgs &A, int scan_block, cudaStream_t st)
{
    return K == 2 ? launch_phased_k<2>(dim, f32, A, scan_block, st) : launch_phased_k<1>(dim, f32, A, scan_block, st);
}

}  // namespace sph

// ---------------------------------------------------------------------------
// host side

struct sph_batch {
    int ncases = 0, dim = 0, n = 0;
    int K = 1;  // stencil radius in cells, shared by every case
    bool f32 = true;
    std::vector<int> off, cnt;
    std::vector<DevParams> hp;
    DevParams *cp = nullptr;
    uint16_t *case_of = nullptr;
    CellBufs cb{};
    SortedBufs sb{};
    std::vector<void *> owned;
    unsigned long long *vmax2 = nullptr, *amax2 = nullptr, *n_pairs = nullptr;
    DiagDev *diag = nullptr;
    uint32_t *status = nullptr;
    BarrierState *bar = nullptr;
    int block = 128, grid = 0, blocks_per_sm = 0;
    int form = SPH_BATCH_PERSISTENT;
    long long spin_limit = 0;
    size_t smem = 0;
    size_t count_bytes = 0;
    // graphs keyed by (nsteps, state pointers)
    std::map<std::string, cudaGraphExec_t> graphs;
    int graph_used = -1;
    std::string err;
};

static std::string g_batch_create_error;

static int bfail(sph_batch *b, int code, const std::string &m)
{
    if (b) b->err = m;
    else g_batch_create_error = m;
    return code;
}


template <int D, typename T>
static void *batch_kernel_ptr(int K)
{
    return K == 2 ? (void *)k_batch<D, T, 2> : (void *)k_batch<D, T, 1>;
}

static void *batch_kernel(int dim, bool f32, int K)
{
    if (dim == 2 && f32) return K == 2 ? (void *)k_batch_2f<2> : (void *)k_batch_2f<1>;
    if (dim == 2) return batch_kernel_ptr<2, double>(K);
    return f32 ? batch_kernel_ptr<3, float>(K) : batch_kernel_ptr<3, double>(K);
}

extern "C" {

const char *sph_batch_last_error(const sph_batch *b)
{
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

int sph_batch_destroy(sph_batch *b)
{
    if (!b) return SPH_OK;
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    for (void *p : b->owned)
        if (p) cudaFree(p);
    delete b;
    return SPH_OK;
}

int sph_batch_create(const sph_case_desc *cases, int ncases, const sph_tune *tune, sph_batch **out)
{
    if (!out) return bfail(nullptr, SPH_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!cases || ncases < 1 || ncases > 65535) return bfail(nullptr, SPH_ERR_INVALID, "bad case list");
    sph_batch *b = new (std::nothrow) sph_batch();
    if (!b) return bfail(nullptr, SPH_ERR_INVALID, "out of host memory");
    b->ncases = ncases;
    b->dim = cases[0].params.dim;
    b->f32 = cases[0].params.precision == SPH_PREC_F32;
    long long ntot = 0, ncells = 0;
    b->hp.resize(ncases);
    std::vector<double> rho_ref(ncases);
    for (int c = 0; c < ncases; ++c) {
        const sph_params &p = cases[c].params;
        if (p.dim != b->dim || (p.precision == SPH_PREC_F32) != b->f32) {
            sph_batch_destroy(b);
            return bfail(nullptr, SPH_ERR_INVALID, "all cases must share dim and precision");
        }
        if (cases[c].n < 0) {
            sph_batch_destroy(b);
            return bfail(nullptr, SPH_ERR_INVALID, "negative case size");
        }
        std::string why;
        if (!make_dev_params(&p, &b->hp[c], &rho_ref[c], why)) {
            sph_batch_destroy(b);
            return bfail(nullptr, SPH_ERR_INVALID, std::string("case ") + std::to_string(c) + ": " + why);
        }
        if (p.model != SPH_MODEL_WCSPH) {
            sph_batch_destroy(b);
            return bfail(nullptr, SPH_ERR_INVALID,
                         std::string("case ") + std::to_string(c) + ": the batched form runs SPH_MODEL_WCSPH only");
        }
        if (p.dt_mode != SPH_DT_FIXED) {
            sph_batch_destroy(b);
            return bfail(nullptr, SPH_ERR_INVALID,
                         std::string("case ") + std::to_string(c) + ": the batched form takes a fixed dt");
        }
        if (c == 0) b->K = b->hp[0].K;
        if (b->hp[c].K != b->K) {
            sph_batch_destroy(b);
            return bfail(nullptr, SPH_ERR_INVALID,
                         "all cases must share the cell size class (cs >= 2h, or h <= cs < 2h)");
        }
        b->off.push_back((int)ntot);
        b->cnt.push_back(cases[c].n);
        ntot += cases[c].n;
        long long nc = 1;
        for (int k = 0; k < b->dim; ++k) nc *= p.ncell[k];
        b->hp[c].cell_off = (uint32_t)ncells;
        ncells += nc;
    }
    if (ntot > (1 << 30) || ncells > 2000000000LL) {
        sph_batch_destroy(b);
        return bfail(nullptr, SPH_ERR_INVALID, "batch too large");
    }
    b->n = (int)ntot;
    // tuning
    b->form = tune ? tune->form : SPH_BATCH_PERSISTENT;
    if (b->form != SPH_BATCH_PERSISTENT && b->form != SPH_BATCH_PHASED) {
        sph_batch_destroy(b);
        return bfail(nullptr, SPH_ERR_INVALID, "tune.form must be SPH_BATCH_PERSISTENT or SPH_BATCH_PHASED");
    }
    b->block = tune && tune->block ? tune->block : 128;
    if (b->block != 64 && b->block != 128 && b->block != 256) {
        sph_batch_destroy(b);
        return bfail(nullptr, SPH_ERR_INVALID, "tune.block must be 64, 128 or 256");
    }
    if (b->form == SPH_BATCH_PHASED && b->block != kPhasedBlock) {
        sph_batch_destroy(b);
        return bfail(nullptr, SPH_ERR_INVALID, "the phased form runs blocks of 128 threads");
    }
    b->spin_limit = tune && tune->spin_limit > 0 ? tune->spin_limit : (1LL << 24);
    const int NC = b->dim == 3 ? 27 : 9;
    b->smem = 33 * sizeof(uint32_t);
    void *kfn = batch_kernel(b->dim, b->f32, b->K);
    int dev = 0, nsm = 0, occ = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (b->form == SPH_BATCH_PERSISTENT) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, b->block, b->smem);
        if (e != cudaSuccess || occ < 1) {
            sph_batch_destroy(b);
            return bfail(nullptr, SPH_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e));
        }
        b->blocks_per_sm =
            tune && tune->blocks_per_sm > 0 ? (tune->blocks_per_sm < occ ? tune->blocks_per_sm : occ) : occ;
        b->grid = b->blocks_per_sm * nsm;
    } else {
        if (e != cudaSuccess) {
            sph_batch_destroy(b);
            return bfail(nullptr, SPH_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
        }
        // (the pair phases' grid: one block per tile of 128 particles)
        b->blocks_per_sm = 0;
        b->grid = (int)((ntot + kPhasedBlock - 1) / kPhasedBlock);
    }
    // buffers
    const size_t n = (size_t)(ntot > 0 ? ntot : 1);
    const size_t tsz = b->f32 ? 4 : 8;
    b->cb.ncells = ncells;
    const int min_tile = 64 * 8;
    b->cb.scan_blocks = (int)((ncells + min_tile - 1) / min_tile);
    const size_t padded = ((size_t)ncells + 2048) / 2048 * 2048 + 2048;
    b->count_bytes = padded * 4;
    auto AL = [&](void **ptr, size_t bytes) {
        if (e != cudaSuccess) return;
        e = cudaMalloc(ptr, bytes ? bytes : 16);
        if (e == cudaSuccess) b->owned.push_back(*ptr);
        else *ptr = nullptr;
    };
    AL((void **)&b->cb.key, n * 4);
    AL((void **)&b->cb.rank, n * 4);
    AL((void **)&b->cb.tmp, n * 4);
    AL((void **)&b->cb.cell_count, padded * 4);
    AL((void **)&b->cb.cell_start, ((size_t)ncells + 1) * 4);
    AL((void **)&b->cb.block_sums, ((size_t)b->cb.scan_blocks + 1) * 4);
    AL(&b->sb.pos, n * 4 * tsz);
    AL(&b->sb.vel, n * 4 * tsz);
    AL(&b->sb.phat, n * tsz);
    for (int k = 0; k < b->dim; ++k) AL((void **)&b->sb.rs[k], n * 8);
    AL((void **)&b->sb.cell_s, n * 4);
    AL((void **)&b->sb.id_s, n * 4);
    AL((void **)&b->sb.kind_s, n);
    AL((void **)&b->sb.mask, (n + 256) * NC * 4);
    AL((void **)&b->sb.ovf, n);
    AL((void **)&b->sb.src, n * 4);
    AL((void **)&b->sb.nnb, n * 2);
    AL((void **)&b->case_of, n * 2);
    AL((void **)&b->cp, sizeof(DevParams) * ncases);
    AL((void **)&b->vmax2, 8 * (size_t)ncases);
    AL((void **)&b->amax2, 8 * (size_t)ncases);
    AL((void **)&b->diag, sizeof(DiagDev) * ncases);
    AL((void **)&b->n_pairs, 8);
    AL((void **)&b->status, 4);
    AL((void **)&b->bar, sizeof(BarrierState));
    // per-case cell base tables
    std::vector<double *> bv;
    std::vector<long long *> bk;
    for (int c = 0; c < ncases && e == cudaSuccess; ++c) {
        StencilEntry *sh = nullptr;
        AL((void **)&sh, 27 * sizeof(StencilEntry));
        if (e == cudaSuccess) {
            StencilEntry hsh[27];
            stencil_table(b->dim, cases[c].params.cs, b->hp[c].nc, hsh, b->hp[c].K);
            e = cudaMemcpy(sh, hsh, sizeof(hsh), cudaMemcpyHostToDevice);
            b->hp[c].stab = sh;
        }
        for (int k = 0; k < b->dim; ++k) {
            double *v = nullptr;
            long long *kk = nullptr;
            AL((void **)&v, ((size_t)cases[c].params.ncell[k] + 1) * 8);
            AL((void **)&kk, ((size_t)cases[c].params.ncell[k] + 1) * 8);
            b->hp[c].bval[k] = v;
            b->hp[c].bkey[k] = kk;
            bv.push_back(v);
            bk.push_back(kk);
        }
        if (e == cudaSuccess) {
            double *vv[3] = {(double *)b->hp[c].bval[0], (double *)b->hp[c].bval[1],
                             b->dim == 3 ? (double *)b->hp[c].bval[2] : nullptr};
            long long *kk[3] = {(long long *)b->hp[c].bkey[0], (long long *)b->hp[c].bkey[1],
                                b->dim == 3 ? (long long *)b->hp[c].bkey[2] : nullptr};
            e = launch_base_tables(b->hp[c], vv, kk, 0);
        }
    }
    std::vector<uint16_t> co(n, 0);
    for (int c = 0; c < ncases; ++c)
        for (int i = 0; i < b->cnt[c]; ++i) co[(size_t)b->off[c] + i] = (uint16_t)c;
    if (e == cudaSuccess) e = cudaMemcpy(b->case_of, co.data(), n * 2, cudaMemcpyHostToDevice);
    for (int c = 0; c < ncases; ++c) {  // used by bounds-checked builds only
        b->hp[c].chk_status = b->status;
        b->hp[c].chk_cap = (uint32_t)n;
    }
    if (e == cudaSuccess) e = cudaMemcpy(b->cp, b->hp.data(), sizeof(DevParams) * ncases, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->cb.cell_count, 0, padded * 4);
    if (e == cudaSuccess) e = cudaMemset(b->cb.cell_start, 0, ((size_t)ncells + 1) * 4);
    if (e == cudaSuccess) e = cudaMemset(b->vmax2, 0, 8 * (size_t)ncases);
    if (e == cudaSuccess) e = cudaMemset(b->amax2, 0, 8 * (size_t)ncases);
    if (e == cudaSuccess) e = cudaMemset(b->diag, 0, sizeof(DiagDev) * ncases);
    if (e == cudaSuccess) e = cudaMemset(b->n_pairs, 0, 8);
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, 4);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        std::string m = std::string("sph_batch_create: ") + cudaGetErrorString(e);
        sph_batch_destroy(b);
        return bfail(nullptr, SPH_ERR_CUDA, m);
    }
    *out = b;
    return SPH_OK;
}

static cudaError_t batch_launch(sph_batch *b, const BatchArgs &args, cudaStream_t st)
{
    // barrier state and the count table start at zero in every launch (a
    // launch that aborted at a barrier may have left counts behind)
    cudaError_t e = cudaMemsetAsync(b->bar, 0, sizeof(BarrierState), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->cb.cell_count, 0, b->count_bytes, st);
    if (e != cudaSuccess) return e;
    if (b->form == SPH_BATCH_PHASED) return launch_phased(b->dim, b->f32, b->K, args, b->block, st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(b->block);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    void *fn = batch_kernel(b->dim, b->f32, b->K);
    void *kargs[] = {(void *)&args};
    return cudaLaunchKernelExC(&cfg, fn, kargs);
}

static BatchArgs make_args(sph_batch *b, const sph_state *s, int nsteps, int selftest)
{
    BatchArgs a{};
    a.n = b->n;
    a.ncases = b->ncases;
    a.cp = b->cp;
    a.case_of = b->case_of;
    a.s = *s;
    a.cb = b->cb;
    a.sb = b->sb;
    a.ntiles_scan = (int)((b->cb.ncells + (long long)b->block * 8 - 1) / ((long long)b->block * 8));
    a.vmax2 = b->vmax2;
    a.amax2 = b->amax2;
    a.diag = b->diag;
    a.n_pairs = b->n_pairs;
    a.status = b->status;
    a.bar = b->bar;
    a.spin_limit = b->spin_limit;
    a.nsteps = nsteps;
    a.selftest = selftest;
    return a;
}

int sph_batch_step(sph_batch *b, sph_state *s, int nsteps, sph_stream_t stream)
{
    if (!b) return SPH_ERR_INVALID;
    if (!s || s->n != b->n) return bfail(b, SPH_ERR_INVALID, "packed state size differs from the batch");
    if (nsteps < 0) return bfail(b, SPH_ERR_INVALID, "negative nsteps");
    if (nsteps == 0 || b->n == 0) return SPH_OK;
    for (int k = 0; k < b->dim; ++k)
        if (!s->r[k] || !s->v[k]) return bfail(b, SPH_ERR_INVALID, "NULL r or v component");
    if (!s->id || !s->kind || !s->rho || !s->p) return bfail(b, SPH_ERR_INVALID, "NULL state array");
    cudaStream_t st = (cudaStream_t)stream;
    const BatchArgs args = make_args(b, s, nsteps, 0);
    char key[256];
    snprintf(key, sizeof(key), "%d:%p:%p:%p:%p:%p:%p:%p:%p:%p:%p", nsteps, (void *)s->r[0], (void *)s->r[1],
             (void *)s->r[2], s->v[0], s->v[1], s->v[2], s->rho, s->p, (void *)s->id, (void *)s->kind);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end() && b->graph_used != 0) {
        // capture the resets + the cooperative launch (or the phased form's
        // nsteps x 9 launches) once per (nsteps, state buffers); replay the
        // graph afterwards
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t el = batch_launch(b, args, st);
            e = cudaStreamEndCapture(st, &g);
            if (el != cudaSuccess) e = el;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e == cudaSuccess) {
            it = b->graphs.emplace(key, ge).first;
            b->graph_used = 1;
        } else {
            cudaGetLastError();  // clear; fall back to direct launches
            b->graph_used = 0;
        }
    }
    cudaError_t e;
    if (it != b->graphs.end()) e = cudaGraphLaunch(it->second, st);
    else e = batch_launch(b, args, st);
    if (e != cudaSuccess) return bfail(b, SPH_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
    return SPH_OK;
}

int sph_batch_get_status(sph_batch *b, uint32_t *out, int sync, sph_stream_t stream)
{
    if (!b || !out) return SPH_ERR_INVALID;
    if (sync) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) return bfail(b, SPH_ERR_CUDA, cudaGetErrorString(e));
    }
    uint32_t v = 0;
    cudaError_t e = cudaMemcpy(&v, b->status, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->status, 0, 4);
    if (e != cudaSuccess) return bfail(b, SPH_ERR_CUDA, cudaGetErrorString(e));
    *out = v;
    return SPH_OK;
}

int sph_batch_diag(sph_batch *b, sph_diag *per_case, int64_t *n_pairs_total)
{
    if (!b) return SPH_ERR_INVALID;
    std::vector<DiagDev> d(b->ncases);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(d.data(), b->diag, sizeof(DiagDev) * b->ncases, cudaMemcpyDeviceToHost);
    unsigned long long np = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&np, b->n_pairs, 8, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bfail(b, SPH_ERR_CUDA, cudaGetErrorString(e));
    if (per_case)
        for (int c = 0; c < b->ncases; ++c) {
            per_case[c].n_pairs = 0;
            per_case[c].n_pairs_fluid = 0;
            per_case[c].vmax = d[c].vmax;
            per_case[c].amax = d[c].amax;
            per_case[c].dt_cfl = d[c].dt_cfl;
            per_case[c].status = 0;
        }
    if (n_pairs_total) *n_pairs_total = (int64_t)np;
    return SPH_OK;
}

int sph_batch_info(const sph_batch *b, int *block, int *grid, int *graph_used, int *n_total)
{
    if (!b) return SPH_ERR_INVALID;
    if (block) *block = b->block;
    if (grid) *grid = b->grid;
    if (graph_used) *graph_used = b->graph_used;
    if (n_total) *n_total = b->n;
    return SPH_OK;
}

int sph_batch_selftest_barrier(sph_batch *b, const sph_state *s, long long spin_limit, uint32_t *status_out,
                               sph_stream_t stream)
{
    if (!b || !s || !status_out || spin_limit < 1) return SPH_ERR_INVALID;
    if (s->n != b->n) return bfail(b, SPH_ERR_INVALID, "packed state size differs from the batch");
    if (b->form != SPH_BATCH_PERSISTENT) return bfail(b, SPH_ERR_INVALID, "the phased form has no grid barrier");
    cudaStream_t st = (cudaStream_t)stream;
    BatchArgs args = make_args(b, s, 1, 1);
    args.spin_limit = spin_limit;
    cudaError_t e = batch_launch(b, args, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bfail(b, SPH_ERR_CUDA, cudaGetErrorString(e));
    return sph_batch_get_status(b, status_out, 0, stream);
}

}  // extern "C"
