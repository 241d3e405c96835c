// sph_pairs.cu -- the pair sums of one WCSPH step and the integration.
//
// Paper (arXiv:1710.08259): Section 2.1 Eq. (interaction_formula), a pair sum
// over neighbours within the influence radius; Section 5.1, the SPH
// interpolant (summation density) and Eq. (diffop1) (symmetric pressure
// gradient); Section 5.1.1, the Wendland kernel, the artificial viscosity
// Pi_ij and the semi-implicit Euler update (v first, then r with the new v).
//
// GB300 design.  The pair loop is gather-only (no atomics in the numerics,
// deterministic): one thread per particle i of the canonical order walks the
// 3^D cells around its own; the particles of a cell are contiguous, so each
// neighbour cell is one contiguous run of float4 loads that the warp's lanes
// (sitting in the same or adjacent cells) share through L1.  This is FP32 ALU
// work, not a dense contraction, so no tensor cores.
//
// Divergence.  Only ~17% of the candidates (3D, h = 1.3 dx, cell 2h) are
// neighbours; with one lane per particle some lane of a warp hits on almost
// every candidate, so a pair body inside the candidate loop runs for the
// whole warp nearly every iteration.  The density pass therefore splits the
// work: loop 1 only tests candidates and records one bit per candidate in a
// 32-bit mask per neighbour cell (cells of <= 32 particles; larger cells take
// a slow path); loop 2 visits set bits only.  The masks go to global memory
// (block-major, coalesced) and the force pass reuses them: it never tests a
// candidate again.
//
// FP32 form: positions enter the pair loop as cell-relative float offsets.
// For a neighbour cell at offset (dx, dy, dz) cells, lane i shifts its own
// offset once, s = o_i - d * cs (exact product), and each candidate costs
// x_ij = s - o_j per axis.  The neighbour predicate d2 < R2 uses
// d2 = fma(z, z, fma(y, y, x * x)) with explicit round-to-nearest
// intrinsics, so it is bit-identical to the CPU oracle's emulation.
//
// Cells of edge h (K = 2, the default of the dam breaks): the neighbours lie
// in the 5^D cells around i's own, walked as 5^(D-1) rows of five
// consecutive cells (one contiguous run each, trimmed by the gap test; the
// x frame per candidate from the cell index in pos.w).  Half of these
// candidates are hits, so the density pass sums the kernel inside the
// candidate loop (plain per-row partial sums, Kahan-compensated across
// rows) and records one mask word per row for the force pass.
#include <cuda_runtime.h>

#include "sph_internal.cuh"
#include "sph_nbr.cuh"
#include "sph_phases.cuh"

namespace sph {

// Resident blocks per SM the FP32 pair kernels are compiled for: 9 blocks of
// 128 threads cap them at 56 registers (the 3D density pass spills one word)
// and hide more of the neighbour-load latency than 8 (4 % per 3D step); the
// 2D passes need fewer registers and run best at 12 (the batched 2D
// workload: 1.21 -> 1.10 ms per step).
constexpr int kPairMinBlocksF32 = 9;
constexpr int kPairMinBlocksF32_2D = 12;
template <int D, typename T> constexpr int pair_min_blocks()
{
    return sizeof(T) == 4 ? (D == 2 ? kPairMinBlocksF32_2D : kPairMinBlocksF32) : 4;
}
// The 3D force pass (54 registers at 9 blocks) fits 10 blocks of 128 without
// spilling and hides more of its neighbour-load latency there (100^3, cells of
// edge h: 0.355 -> 0.329 ms); at 12 it spills and takes 0.66 ms.
constexpr int kForceMinBlocksF32_3D = 10;
template <int D, typename T> constexpr int force_min_blocks()
{
    return (sizeof(T) == 4 && D == 3) ? kForceMinBlocksF32_3D : pair_min_blocks<D, T>();
}

// ---- density + equation of state ----------------------------------------

template <int D, typename T, int K>
__global__ void __launch_bounds__(kBlock, pair_min_blocks<D, T>()) k_density(
    DevParams P, int n, const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ cell_s,
    const uint32_t *__restrict__ start, vec4_t<T> *vel, T *phat, T *rho_out, T *p_out, Accum *acc, uint32_t *gmask,
    uint8_t *ovf, uint16_t *nnb)
{
    constexpr int NC = Sten<D, K>::NC;
    const int tid = threadIdx.x;
    const int i = blockIdx.x * blockDim.x + tid;
    unsigned long long pairs = 0;
    if (i < n)
        pairs = dev_density<D, T, K>(P, i, pos, cell_s, start, vel, phat, rho_out, p_out,
                                  gmask + (size_t)blockIdx.x * NC * kBlock + tid, kBlock, ovf, nnb);
    pairs = warp_sum(pairs);
    __shared__ unsigned long long ws[kBlock / 32];
    if ((tid & 31) == 0) ws[tid >> 5] = pairs;
    __syncthreads();
    if (tid == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        if (t) atomicAdd(&acc->n_pairs, t);
    }
}

// The density pass with TEAM lanes per particle (cells of edge h, small
// cases: see dev_density_team); the masks keep the one-lane layout.
template <int D, typename T, int TEAM>
__global__ void __launch_bounds__(kBlock, pair_min_blocks<D, T>()) k_density_team(
    DevParams P, int n, const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ cell_s,
    const uint32_t *__restrict__ start, vec4_t<T> *vel, T *phat, T *rho_out, T *p_out, Accum *acc, uint32_t *gmask,
    uint8_t *ovf, uint16_t *nnb)
{
    constexpr int NC = Sten<D, 2>::NC;
    const int tid = threadIdx.x;
    const int g = blockIdx.x * blockDim.x + tid;
    const int i = g / TEAM, tl = g % TEAM;
    unsigned long long pairs = dev_density_team<D, T, TEAM>(
        P, i, i < n, tl, pos, cell_s, start, vel, phat, rho_out, p_out,
        gmask + (size_t)(i / kBlock) * NC * kBlock + (i % kBlock), kBlock, ovf, nnb);
    pairs = warp_sum(pairs);
    __shared__ unsigned long long ws[kBlock / 32];
    if ((tid & 31) == 0) ws[tid >> 5] = pairs;
    __syncthreads();
    if (tid == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        if (t) atomicAdd(&acc->n_pairs, t);
    }
}

// ---- accelerations (+ integration) ---------------------------------------

template <int D, typename T, bool INTEGRATE, int K>
__global__ void __launch_bounds__(kBlock, force_min_blocks<D, T>()) k_force(
    DevParams P, int n, const vec4_t<T> *__restrict__ pos, const vec4_t<T> *__restrict__ vel,
    const T *__restrict__ phat, const uint32_t *__restrict__ cell_s, const uint32_t *__restrict__ start,
    const uint32_t *__restrict__ gmask, const uint8_t *__restrict__ ovf, SortedBufs sb, sph_state s, T *a0, T *a1,
    T *a2, Accum *acc, uint32_t *status)
{
    constexpr int NC = Sten<D, K>::NC;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    ForceOut<T> o{(T)0, (T)0, 0u, false};
    if (i < n)
        o = dev_force<D, T, INTEGRATE, K>(P, i, pos, vel, phat, cell_s, start,
                                       gmask + (size_t)blockIdx.x * NC * kBlock + threadIdx.x, kBlock, ovf, sb, s,
                                       a0, a1, a2);
    if (o.bad) atomicOr(status, SPH_STATUS_NAN);
    const T v2max = warp_max(o.v2);
    const T a2max = warp_max(o.a2);
    const unsigned long long fpairs = warp_sum((unsigned long long)o.pairs);
    __shared__ T wv[kBlock / 32], wa[kBlock / 32];
    __shared__ unsigned long long wp[kBlock / 32];
    if ((threadIdx.x & 31) == 0) {
        wv[threadIdx.x >> 5] = v2max;
        wa[threadIdx.x >> 5] = a2max;
        wp[threadIdx.x >> 5] = fpairs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T mv = (T)0, ma = (T)0;
        unsigned long long tp = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            mv = fmax(mv, wv[w]);
            ma = fmax(ma, wa[w]);
            tp += wp[w];
        }
        if (tp) atomicAdd(&acc->n_pairs_fluid, tp);
        raise_max(&acc->vmax2, (double)mv);
        raise_max(&acc->amax2, (double)ma);
    }
}

// The force pass (with integration) with TEAM lanes per particle (cells of
// edge h, small cases: see dev_force_team).
template <int D, typename T, int TEAM>
__global__ void __launch_bounds__(kBlock, force_min_blocks<D, T>()) k_force_team(
    DevParams P, int n, const vec4_t<T> *__restrict__ pos, const vec4_t<T> *__restrict__ vel,
    const T *__restrict__ phat, const uint32_t *__restrict__ cell_s, const uint32_t *__restrict__ start,
    const uint32_t *__restrict__ gmask, const uint8_t *__restrict__ ovf, SortedBufs sb, sph_state s, Accum *acc,
    uint32_t *status)
{
    constexpr int NC = Sten<D, 2>::NC;
    __shared__ vec4_t<T> tbuf[(kBlock / TEAM) * kTeamHits];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g / TEAM, tl = g % TEAM;
    const ForceOut<T> o = dev_force_team<D, T, true, TEAM>(
        P, i, i < n, tl, pos, vel, phat, cell_s, start, gmask + (size_t)(i / kBlock) * NC * kBlock + (i % kBlock),
        kBlock, ovf, sb, s, tbuf + (threadIdx.x / TEAM) * kTeamHits, nullptr, nullptr, nullptr);
    if (o.bad) atomicOr(status, SPH_STATUS_NAN);
    const T v2max = warp_max(o.v2);
    const T a2max = warp_max(o.a2);
    const unsigned long long fpairs = warp_sum((unsigned long long)o.pairs);
    __shared__ T wv[kBlock / 32], wa[kBlock / 32];
    __shared__ unsigned long long wp[kBlock / 32];
    if ((threadIdx.x & 31) == 0) {
        wv[threadIdx.x >> 5] = v2max;
        wa[threadIdx.x >> 5] = a2max;
        wp[threadIdx.x >> 5] = fpairs;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T mv = (T)0, ma = (T)0;
        unsigned long long tp = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            mv = fmax(mv, wv[w]);
            ma = fmax(ma, wa[w]);
            tp += wp[w];
        }
        if (tp) atomicAdd(&acc->n_pairs_fluid, tp);
        raise_max(&acc->vmax2, (double)mv);
        raise_max(&acc->amax2, (double)ma);
    }
}

// The force pass's teams also hold their terms in shared memory (kTeamHits
// per particle, at most 32 KB per block): 8 or 4 lanes in FP32, 8 in FP64.
static int force_team(int n, bool f32)
{
    const int t = pair_team(n);
    return t == 8 || (t == 4 && f32) ? t : 1;
}

// step: the pass ended a time step (the step size is recorded, the elapsed
// time advanced and, for SPH_DT_ADAPTIVE, the next step size set)
__global__ void k_finish(DevParams P, double h, double c0, Accum *acc, uint32_t *status, DiagDev *diag, int step)
{
    double vmax = sqrt(__longlong_as_double((long long)acc->vmax2));
    double amax = sqrt(__longlong_as_double((long long)acc->amax2));
    double t1 = 0.25 * h / (c0 + vmax);
    double t2 = amax > 0.0 ? 0.25 * sqrt(h / amax) : INFINITY;
    double dtc = fmin(t1, t2);
    const double dt_used = P.adaptive ? diag->dt_next : P.dt;
    // the SPH sound-speed bound means nothing for the DEM model
    if (P.model != SPH_MODEL_DEM && dt_used > dtc) atomicOr(status, SPH_STATUS_CFL);
    if (step) {
        diag->dt = dt_used;
        diag->time += dt_used;
        if (P.adaptive) diag->dt_next = fmin(P.dt, P.cfl * dtc);
    }
    diag->n_pairs = (long long)acc->n_pairs;
    diag->n_pairs_fluid = (long long)acc->n_pairs_fluid;
    diag->vmax = vmax;
    diag->amax = amax;
    diag->dt_cfl = dtc;
    diag->status = *status;
    acc->n_pairs = 0;
    acc->n_pairs_fluid = 0;
    acc->vmax2 = 0;
    acc->amax2 = 0;
}

// ---- neighbour queries (tests): the sets the density pass found -----------

template <int D, typename T, int K>
__global__ void __launch_bounds__(kBlock) k_nbr_list(DevParams P, int n, const vec4_t<T> *__restrict__ pos,
                                                     const uint32_t *__restrict__ cell_s,
                                                     const uint32_t *__restrict__ start,
                                                     const uint32_t *__restrict__ gmask,
                                                     const uint8_t *__restrict__ ovf,
                                                     const uint32_t *__restrict__ id_s,
                                                     const int64_t *__restrict__ offsets, uint32_t *counts,
                                                     uint32_t *ids, uint8_t *images)
{
    constexpr int NC = Sten<D, K>::NC;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t *out = ids ? ids + offsets[i] : nullptr;
    uint32_t cnt = 0;
    auto body = [&](uint32_t j, T, T, T, T) {
        if (j == (uint32_t)i) return;
        if (out) out[cnt] = id_s[j];
        ++cnt;
    };
    if (!ovf[i])
        nbr_masked<D, T, K>(P, pos[i], cell_s[i], pos, start, [&](int idx) { return gmask[mask_index(NC, idx)]; },
                            body);
    else
        nbr_scan<D, T, K>(P, pos[i], cell_s[i], pos, start, body);
    if (counts) counts[i] = cnt;
    if (!out) return;
    if (images)
        for (uint32_t a = 0; a < cnt; ++a) images[offsets[i] + a] = 0;  // (no images: cut-off faces)
    // ascending ids (insertion sort; lists hold ~20-80 entries)
    for (uint32_t a = 1; a < cnt; ++a) {
        uint32_t v = out[a];
        uint32_t b = a;
        while (b > 0 && out[b - 1] > v) {
            out[b] = out[b - 1];
            --b;
        }
        out[b] = v;
    }
}

// ---- launchers --------------------------------------------------------------

static inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

// Threads per block of the team kernels: a small case's grid covers few
// blocks per SM, so in FP64, where the narrow FP64 pipe bounds each SM, blocks
// of 64 spread the work more evenly (2D 64 x 64: 318 blocks of 128 put 3 on
// some SMs and 2 on most; FP64 step 0.089 -> 0.084 ms).  FP32 keeps 128
// (0.031 against 0.032 ms with 64).
template <typename T> constexpr int team_block() { return sizeof(T) == 8 ? 64 : kBlock; }

template <int D, typename T>
static void density_impl(const DevParams &P, int n, const CellBufs &cb, const SortedBufs &sb,
                         void *rho_out, void *p_out, Accum *acc, cudaStream_t st)
{
    using V4 = vec4_t<T>;
    const int team = P.K == 2 ? pair_team(n) : 1;
    if (team > 1) {
        auto kt = team == 8 ? k_density_team<D, T, 8> : (team == 4 ? k_density_team<D, T, 4> : k_density_team<D, T, 2>);
        kt<<<blocks_for((int)((long long)n * team), team_block<T>()), team_block<T>(), 0, st>>>(
            P, n, static_cast<const V4 *>(sb.pos), sb.cell_s, cb.cell_start, static_cast<V4 *>(sb.vel),
            static_cast<T *>(sb.phat), static_cast<T *>(rho_out), static_cast<T *>(p_out), acc, sb.mask, sb.ovf,
            sb.nnb);
        return;
    }
    auto kern = P.K == 2 ? k_density<D, T, 2> : k_density<D, T, 1>;
    kern<<<blocks_for(n, kBlock), kBlock, 0, st>>>(
        P, n, static_cast<const V4 *>(sb.pos), sb.cell_s, cb.cell_start, static_cast<V4 *>(sb.vel),
        static_cast<T *>(sb.phat), static_cast<T *>(rho_out), static_cast<T *>(p_out), acc, sb.mask, sb.ovf, sb.nnb);
}

cudaError_t launch_density(const DevParams &P, bool f32, int n, const CellBufs &cb,
                           const SortedBufs &sb, void *rho_out, void *p_out, Accum *acc,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (P.dim == 2) {
        if (f32) density_impl<2, float>(P, n, cb, sb, rho_out, p_out, acc, st);
        else density_impl<2, double>(P, n, cb, sb, rho_out, p_out, acc, st);
    } else {
        if (f32) density_impl<3, float>(P, n, cb, sb, rho_out, p_out, acc, st);
        else density_impl<3, double>(P, n, cb, sb, rho_out, p_out, acc, st);
    }
    return cudaGetLastError();
}

template <int D, typename T>
static void force_impl(const DevParams &P, int n, const CellBufs &cb, const SortedBufs &sb,
                       const sph_state &s, void *const *a_out, Accum *acc, uint32_t *status,
                       cudaStream_t st)
{
    using V4 = vec4_t<T>;
    const V4 *pos = static_cast<const V4 *>(sb.pos);
    const V4 *vel = static_cast<const V4 *>(sb.vel);
    const T *ph = static_cast<const T *>(sb.phat);
    if (a_out) {
        auto kern = P.K == 2 ? k_force<D, T, false, 2> : k_force<D, T, false, 1>;
        kern<<<blocks_for(n, kBlock), kBlock, 0, st>>>(
            P, n, pos, vel, ph, sb.cell_s, cb.cell_start, sb.mask, sb.ovf, sb, s, static_cast<T *>(a_out[0]),
            static_cast<T *>(a_out[1]), D == 3 ? static_cast<T *>(a_out[2]) : nullptr, acc, status);
    } else if (P.K == 2 && force_team(n, sizeof(T) == 4) > 1) {
        const int team = force_team(n, sizeof(T) == 4);
        auto kt = k_force_team<D, T, 8>;
        if constexpr (sizeof(T) == 4)
            if (team == 4) kt = k_force_team<D, T, 4>;
        kt<<<blocks_for((int)((long long)n * team), team_block<T>()), team_block<T>(), 0, st>>>(
            P, n, pos, vel, ph, sb.cell_s, cb.cell_start, sb.mask, sb.ovf, sb, s, acc, status);
    } else {
        auto kern = P.K == 2 ? k_force<D, T, true, 2> : k_force<D, T, true, 1>;
        kern<<<blocks_for(n, kBlock), kBlock, 0, st>>>(
            P, n, pos, vel, ph, sb.cell_s, cb.cell_start, sb.mask, sb.ovf, sb, s, nullptr, nullptr, nullptr, acc,
            status);
    }
}

cudaError_t launch_force(const DevParams &P, bool f32, int n, const CellBufs &cb,
                         const SortedBufs &sb, const sph_state &s, void *const *a_out, Accum *acc,
                         uint32_t *status, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (P.dim == 2) {
        if (f32) force_impl<2, float>(P, n, cb, sb, s, a_out, acc, status, st);
        else force_impl<2, double>(P, n, cb, sb, s, a_out, acc, status, st);
    } else {
        if (f32) force_impl<3, float>(P, n, cb, sb, s, a_out, acc, status, st);
        else force_impl<3, double>(P, n, cb, sb, s, a_out, acc, status, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_finish(const DevParams &P, double h, double c0, Accum *acc, uint32_t *status,
                          DiagDev *diag, int step, cudaStream_t st)
{
    k_finish<<<1, 1, 0, st>>>(P, h, c0, acc, status, diag, step);
    return cudaGetLastError();
}

template <int D, typename T>
static void nbr_impl(const DevParams &P, int n, const CellBufs &cb, const SortedBufs &sb,
                     uint32_t *counts, const int64_t *offsets, uint32_t *ids, uint8_t *images, cudaStream_t st)
{
    using V4 = vec4_t<T>;
    auto kern = P.K == 2 ? k_nbr_list<D, T, 2> : k_nbr_list<D, T, 1>;
    kern<<<blocks_for(n, kBlock), kBlock, 0, st>>>(P, n, static_cast<const V4 *>(sb.pos), sb.cell_s, cb.cell_start,
                                                   sb.mask, sb.ovf, sb.id_s, offsets, counts, ids, images);
}

cudaError_t launch_nbr(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                       uint32_t *counts, const int64_t *offsets, uint32_t *ids, cudaStream_t st, uint8_t *images)
{
    if (n <= 0) return cudaSuccess;
    if (P.dim == 2) {
        if (f32) nbr_impl<2, float>(P, n, cb, sb, counts, offsets, ids, images, st);
        else nbr_impl<2, double>(P, n, cb, sb, counts, offsets, ids, images, st);
    } else {
        if (f32) nbr_impl<3, float>(P, n, cb, sb, counts, offsets, ids, images, st);
        else nbr_impl<3, double>(P, n, cb, sb, counts, offsets, ids, images, st);
    }
    return cudaGetLastError();
}

}  // namespace sph
