// sph_phases.cuh -- the per-particle (or per-tile) bodies of every phase of
// one WCSPH step, shared by the one-kernel-per-phase path (sph_cells.cu,
// sph_pairs.cu) and the persistent batched kernel (sph_batch.cu), so that both
// run the same arithmetic.
//
// Phases (arXiv:1710.08259, Section 3.2.1 cell grid; Section 5.1 / 5.1.1 SPH
// operators, EOS, viscosity, semi-implicit Euler):
//   hash      : cell of each particle, warp-aggregated counting per cell
//   scan      : exclusive prefix sum of the cell counts -> cell start table
//   scatter   : particle index -> start[cell] + arrival slot
//   gather    : rank inside the cell by persistent id, reorder the state
//   density   : candidate tests -> neighbour masks, Kahan density, Tait EOS
//   force     : pressure + viscosity accelerations over the masks, update
//
// DevParams.cell_off is the offset of a case's cells in a shared cell table
// (0 for a single case): keys and cell_s hold global cell indices.
#pragma once

#include <cuda_runtime.h>

#include "sph_internal.cuh"
#include "sph_nbr.cuh"

namespace sph {

__device__ __forceinline__ double cell_base(double lo, double cs, int c)
{
    return __dadd_rn(lo, __dmul_rn((double)c, cs));
}

// Order-preserving signed key of a double (-0 taken as +0): key(a) < key(b)
// iff a < b for non-NaN a, b.  NaNs land outside every finite range.
__device__ __forceinline__ long long okey(double x)
{
    long long b = __double_as_longlong(x);
    if (b == (long long)0x8000000000000000ULL) b = 0;
    return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

// Largest c with base(c) <= x (base in double RN, no contraction), from a
// float estimate corrected by integer compares against the base table (no
// FP64 arithmetic: the FP64 pipe of this GPU is narrow).  Outside the grid
// (or NaN) sets bad and returns the nearest valid cell so that the build stays
// memory-safe; the status word reports the error.
__device__ __forceinline__ int cell_axis(const DevParams &P, int k, double x, bool &bad)
{
    const long long *kb = P.bkey[k];
    const int nc = P.nc[k];
    const long long kx = okey(x);
    if (!(kx >= kb[0])) {
        bad = true;
        return 0;
    }
    if (!(kx < kb[nc])) {
        bad = true;
        return nc - 1;
    }
    float est = floorf((__double2float_rn(x) - P.lof[k]) * P.inv_csf);
    est = fminf(fmaxf(est, 0.0f), (float)(nc - 1));
    int c = (int)est;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        if (c > 0 && kb[c] > kx) --c;
        if (c + 1 < nc && kb[c + 1] <= kx) ++c;
    }
    if (!(kb[c] <= kx && kx < kb[c + 1])) {
        // the float estimate was far off (huge domain): bisect the table
        int lo = 0, hi = nc;  // kb[lo] <= kx < kb[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (kb[mid] <= kx) lo = mid;
            else hi = mid;
        }
        c = lo;
    }
    return c;
}

// ---- hash + count --------------------------------------------------------
// Every lane of the warp calls this (active = false past the end).  The
// input is nearly sorted (the previous step left it in canonical order), so
// lanes holding the same cell mostly sit side by side: each run of equal
// cells in adjacent active lanes is counted by one atomicAdd of its first
// lane, and a lane's arrival slot is the run's base plus its place in the
// run.  A cell split over several runs takes one atomic per run; any such
// grouping gives the cell's particles distinct slots, and the gather then
// orders every cell by persistent id.  (Grouping the warp's lanes of each
// cell with __match_any_sync took 0.98 against 0.91 ms per 256^3 build.)
template <int D>
__device__ __forceinline__ void dev_hash(const DevParams &P, int k, bool active, const sph_state &s,
                                         uint32_t *key, uint32_t *rank, uint32_t *cell_count, uint32_t *status)
{
    const int lane = threadIdx.x & 31;
    bool bad = false;
    uint32_t c = 0;
    if (active) {
        const int cx = cell_axis(P, 0, s.r[0][k], bad);
        const int cy = cell_axis(P, 1, s.r[1][k], bad);
        int cz = 0;
        if (D == 3) cz = cell_axis(P, 2, s.r[2][k], bad);
        c = P.cell_off + (uint32_t)cx + (uint32_t)P.nc[0] * ((uint32_t)cy + (uint32_t)P.nc[1] * (uint32_t)cz);
    }
    const unsigned act = __ballot_sync(0xffffffffu, active);
    const uint32_t cprev = __shfl_up_sync(0xffffffffu, c, 1);
    const bool prev_act = lane > 0 && ((act >> (lane - 1)) & 1u);
    // run heads: active lanes whose left neighbour is inactive or holds
    // another cell; a run ends at the next head or inactive lane
    const unsigned heads = __ballot_sync(0xffffffffu, active && (!prev_act || cprev != c));
    const unsigned le = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;  // lanes <= this one
    const int lead = 31 - __clz(heads & le);
    const unsigned brk = (heads | ~act) & ~le;
    const int end = brk ? __ffs(brk) - 1 : 32;
    uint32_t base = 0;
    if (active && lane == lead) base = atomicAdd(&cell_count[c], (uint32_t)(end - lane));
    base = __shfl_sync(0xffffffffu, base, lead & 31);
    if (active) {
        rank[k] = base + (uint32_t)(lane - lead);
        key[k] = c;
        if (bad) atomicOr(status, SPH_STATUS_OUT_OF_DOMAIN);
    }
}

// ---- exclusive scan of the cell counts ------------------------------------
// A tile is blockDim.x * 8 cells; every thread of the block takes part.
// ws: shared scratch of >= 33 words.

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ void dev_scan_reduce(const uint32_t *__restrict__ cnt, uint32_t *block_sums, int tile,
                                                uint32_t *ws)
{
    const uint4 *c4 = reinterpret_cast<const uint4 *>(cnt + (size_t)tile * blockDim.x * 8) + threadIdx.x * 2;
    const uint4 a = c4[0], b = c4[1];
    uint32_t s = a.x + a.y + a.z + a.w + b.x + b.y + b.z + b.w;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        block_sums[tile] = t;
    }
    __syncthreads();
}

// One block: exclusive scan of nb block sums in place; total -> *total.
__device__ __forceinline__ void dev_scan_top(uint32_t *block_sums, int nb, uint32_t *total, uint32_t *ws)
{
    uint32_t &carry = ws[32];
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    for (int base = 0; base < nb; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t v = i < nb ? block_sums[i] : 0u;
        const uint32_t inc = warp_incl_scan(v);
        if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = inc;
        __syncthreads();
        if (threadIdx.x < 32) {
            const uint32_t w = threadIdx.x < nw ? ws[threadIdx.x] : 0u;
            const uint32_t e = warp_incl_scan(w) - w;
            if (threadIdx.x < nw) ws[threadIdx.x] = e;
        }
        __syncthreads();
        const uint32_t excl = carry + ws[threadIdx.x >> 5] + inc - v;
        if (i < nb) block_sums[i] = excl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
    __syncthreads();
}

__device__ __forceinline__ void dev_scan_apply(uint32_t *cnt, const uint32_t *__restrict__ block_sums,
                                               uint32_t *start, int64_t ncells, int tile, uint32_t *ws)
{
    uint4 *c4 = reinterpret_cast<uint4 *>(cnt + (size_t)tile * blockDim.x * 8) + threadIdx.x * 2;
    const uint4 a = c4[0], b = c4[1];
    const uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t tsum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) tsum += v[q];
    const uint32_t inc = warp_incl_scan(tsum);
    const int nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
        const uint32_t w = threadIdx.x < nw ? ws[threadIdx.x] : 0u;
        const uint32_t e = warp_incl_scan(w) - w;
        if (threadIdx.x < nw) ws[threadIdx.x] = e;
    }
    __syncthreads();
    uint32_t run = block_sums[tile] + ws[threadIdx.x >> 5] + inc - tsum;
    const int64_t c0 = (int64_t)tile * blockDim.x * 8 + (int64_t)threadIdx.x * 8;
    // (two 16-byte stores per thread: a warp writes 1 KB contiguously;
    // eight scalar stores ran the 70 M-cell table at 2.7 TB/s)
    if (c0 + 8 <= ncells) {
        uint32_t o[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            o[q] = run;
            run += v[q];
        }
        uint4 *s4 = reinterpret_cast<uint4 *>(start + c0);
        s4[0] = make_uint4(o[0], o[1], o[2], o[3]);
        s4[1] = make_uint4(o[4], o[5], o[6], o[7]);
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (c0 + q < ncells) start[c0 + q] = run;
            run += v[q];
        }
    }
    // counts are consumed: zero them for the next build
    c4[0] = make_uint4(0, 0, 0, 0);
    c4[1] = make_uint4(0, 0, 0, 0);
    __syncthreads();
}

__device__ __forceinline__ void dev_scatter(int k, const uint32_t *__restrict__ key,
                                            const uint32_t *__restrict__ rank, const uint32_t *__restrict__ start,
                                            uint32_t *tmp)
{
    tmp[start[key[k]] + rank[k]] = (uint32_t)k;
}

// ---- rank inside the cell by id, gather the state into its canonical slot ---
template <int D, typename T>
__device__ __forceinline__ uint32_t dev_order_gather(const DevParams &P, int t, const sph_state &s,
                                                 const uint32_t *__restrict__ key,
                                                 const uint32_t *__restrict__ start,
                                                 const uint32_t *__restrict__ tmp, const SortedBufs &sb,
                                                 uint32_t *status)
{
    const uint32_t k = tmp[t];
    const uint32_t c = key[k];
    const uint32_t s0 = start[c], s1 = start[c + 1];
    const uint32_t myid = s.id[k];
    uint32_t pos;
    if (s1 - s0 > (uint32_t)SPH_MAX_CELL) {
        atomicOr(status, SPH_STATUS_CELL_OVERFLOW);
        pos = (uint32_t)t;
    } else {
        uint32_t below = 0, same = 0;
        for (uint32_t q = s0; q < s1; ++q) {
            const uint32_t o = s.id[tmp[q]];
            below += (o < myid);
            same += (o == myid);
        }
        if (same != 1) atomicOr(status, SPH_STATUS_DUPLICATE_ID);
        pos = s0 + below;
    }
    if (!SPH_IN_BOUNDS(P, pos < P.chk_cap && s0 <= s1)) return 0xFFFFFFFFu;
    const T *vx = static_cast<const T *>(s.v[0]);
    const T *vy = static_cast<const T *>(s.v[1]);
    const T *vz = static_cast<const T *>(s.v[2]);
    const double x = s.r[0][k], y = s.r[1][k], z = D == 3 ? s.r[2][k] : 0.0;
    using V4 = vec4_t<T>;
    V4 pv;
    const CellXYZ cc = decode_cell(P, c);
    if (sizeof(T) == 4) {
        // cell-relative float offsets: o = (float)(x - base(c))
        pv.x = (T)__double2float_rn(__dsub_rn(x, P.bval[0][cc.x]));
        pv.y = (T)__double2float_rn(__dsub_rn(y, P.bval[1][cc.y]));
        pv.z = D == 3 ? (T)__double2float_rn(__dsub_rn(z, P.bval[2][cc.z])) : (T)0;
    } else {
        pv.x = (T)x;
        pv.y = (T)y;
        pv.z = (T)z;
    }
    // w: the radius of a sphere (SPH_MODEL_DEM); the cell's x index where the
    // stencil is walked as rows (K = 2: the x frame of a candidate); else unused
    pv.w = (P.model == SPH_MODEL_DEM && s.radius) ? static_cast<const T *>(s.radius)[k]
           : P.K == 2                             ? (T)cc.x
                                                  : (T)0;
    V4 vv;
    // (no velocity in the state of the field model: zeros)
    vv.x = vx ? vx[k] : (T)0;
    vv.y = vy ? vy[k] : (T)0;
    vv.z = (D == 3 && vz) ? vz[k] : (T)0;
    // w: the density when the model carries it as a field (continuity
    // equation), the mass of a sphere (DEM), otherwise filled by the
    // density pass
    vv.w = (P.model == SPH_MODEL_EXAMPLE_1A && s.rho)   ? static_cast<const T *>(s.rho)[k]
           : (P.model == SPH_MODEL_DEM && s.mass) ? static_cast<const T *>(s.mass)[k]
                                                    : (T)0;
    static_cast<V4 *>(sb.pos)[pos] = pv;
    static_cast<V4 *>(sb.vel)[pos] = vv;
    sb.rs[0][pos] = x;
    sb.rs[1][pos] = y;
    if (D == 3) sb.rs[2][pos] = z;
    sb.cell_s[pos] = c;
    sb.id_s[pos] = myid;
    sb.src[pos] = k;
    sb.kind_s[pos] = s.kind[k];
    return pos;
}

// One hit of the density sum into a row's plain partial sum:
// w(q) = (1 - q/2)^4 (2q + 1) with hih = 1 / (2h).
template <typename T>
__device__ __forceinline__ void density_hit(T d2, T hih, T &sr)
{
    const T u = Ar<T>::dist_ftz(d2) * hih;  // q / 2
    const T t = (T)1 - u;
    const T t2 = t * t;
    sr += t2 * t2 * ((T)4 * u + (T)1);
}

// S += y, Kahan-compensated (comp carries the lost low part).
template <typename T>
__device__ __forceinline__ void kahan_add(T &S, T &comp, T y0)
{
    const T y = y0 - comp;
    const T s2 = S + y;
    comp = (s2 - S) - y;
    S = s2;
}

// The density pass's per-particle tail: rho from the kernel sum S, the Tait
// pressure, P/rho^2, the outputs and the flags.
template <typename T>
__device__ __forceinline__ void density_finish(const DevParams &P, int i, T S, int total, bool over, vec4_t<T> *vel,
                                               T *phat, T *rho_out, T *p_out, uint8_t *ovf, uint16_t *nnb)
{
    nnb[i] = (uint16_t)total;
    const T rho = (T)P.mAlpha * S;
    // (rho/rho_ref)^gamma - 1 = (1+d)^gamma - 1 with d = S/S_ref - 1, as
    // d * polynomial(d): no cancellation near rest.
    const T d = (S - (T)P.S_ref) * (T)P.inv_S_ref;
    T poly = (T)P.binom[P.gamma - 1];
    for (int k = P.gamma - 2; k >= 0; --k) poly = poly * d + (T)P.binom[k];
    T p = (T)P.B * d * poly;
    if (P.clamp && p < (T)0) p = (T)0;
    vel[i].w = rho;
    phat[i] = p / (rho * rho);
    if (rho_out) rho_out[i] = rho;
    if (p_out) p_out[i] = p;
    ovf[i] = over ? 1 : 0;
}

// ---- density + equation of state ------------------------------------------
// mbase: this particle's mask words at mbase[idx * mstride] (global; the
// force and adjoint passes reuse them).  Returns the number of neighbours
// (self excluded).
template <int D, typename T, int K = 1>
__device__ __forceinline__ uint32_t dev_density(const DevParams &P, int i, const vec4_t<T> *__restrict__ pos,
                                                const uint32_t *__restrict__ cell_s,
                                                const uint32_t *__restrict__ start, vec4_t<T> *vel, T *phat,
                                                T *rho_out, T *p_out, uint32_t *mbase, int mstride, uint8_t *ovf,
                                                uint16_t *nnb)
{
    const vec4_t<T> pi = pos[i];
    const uint32_t c = cell_s[i];
    const T cs = cell_edge<T>(P), R2 = radius2<T>(P);
    // a neighbour cell whose box lies beyond the support radius cannot hold a
    // neighbour: skip its candidates (F32 form, cell-relative offsets; the
    // margin keeps the test conservative against rounding).  Squared gaps to
    // the lower / upper neighbour cell per axis:
    const T R2cull = R2 * (T)1.0001;
    const T glx = pi.x * pi.x, gux = (cs - pi.x) * (cs - pi.x);
    const T gly = pi.y * pi.y, guy = (cs - pi.y) * (cs - pi.y);
    const T glz = D == 3 ? pi.z * pi.z : (T)0, guz = D == 3 ? (cs - pi.z) * (cs - pi.z) : (T)0;
    // loop 1: candidate tests, one bit per candidate (and, for the row
    // stencil, the kernel sum of the hits)
    bool over = false;
    int total = 0;
    const T hih = (T)P.half_inv_h;
    T S = (T)0, comp = (T)0;
    uint32_t cnt = 0;
    // one hit of the kernel sum, Kahan-compensated: S = sum of
    // w(q) = (1 - q/2)^4 (2q + 1) (self pair included: w(0) = 1)
    auto body = [&](uint32_t, T, T, T, T d2) {
        T w = (T)0;
        density_hit<T>(d2, hih, w);
        kahan_add<T>(S, comp, w);
        ++cnt;
    };
    if (K == 1) {
        for_stencil<D>(P, decode_cell(P, c), [&](int idx, int cell, int dx, int dy, int dz) {
            uint32_t a = 0, b = 0;
            if (cell >= 0) {
                a = start[cell];
                b = start[cell + 1];
                if (!SPH_IN_BOUNDS(P, a <= b && b <= P.chk_cap)) b = a;
            }
            if (b - a > 32u) {
                over = true;
                b = a;
            }
            if (sizeof(T) == 4) {
                const T g = (dx < 0 ? glx : (dx > 0 ? gux : (T)0)) + (dy < 0 ? gly : (dy > 0 ? guy : (T)0)) +
                            (dz < 0 ? glz : (dz > 0 ? guz : (T)0));
                if (g > R2cull) b = a;
            }
            const Frame<D, T> s(pi, cs, dx, dy, dz);
            uint32_t w = 0, bit = 1u;
#pragma unroll 4
            for (uint32_t j = a; j < b; ++j, bit <<= 1) {
                T rx, ry, rz;
                const T d2 = geometry<D, T>(s, pos[j], rx, ry, rz);
                if (d2 < R2) w |= bit;
            }
            mbase[idx * mstride] = w;
            total += __popc(w);
        });
    } else {
        // rows of five cells (edge cs in [h, 2h)); the F32 form trims each
        // row to the cells whose box comes within the support radius (the
        // same conservative squared-gap test), bits count from the row's
        // first (clipped, untrimmed) cell.  About half of these candidates
        // are neighbours, so the kernel sum runs inside the candidate loop
        // (a second walk over the masks, which re-reads every neighbour,
        // cost 22 % more at 100^3).  The few hits of a row (~3) add up in a
        // plain partial sum and the row sums in the compensated (Kahan) sum:
        // one addition per hit instead of four (100^3: 0.469 -> 0.448 ms).
        // With cells of 2h only one candidate in five is a neighbour and the
        // sum walks the masks, Kahan-compensated per hit.
        T sr = (T)0;
        total = row_candidates<D, T>(
            P, pi, c, pos, start, mbase, mstride, over,
            [&](uint32_t, T, T, T, T d2) { density_hit<T>(d2, hih, sr); },
            [&] {
                kahan_add<T>(S, comp, sr);
                sr = (T)0;
            });
        cnt = (uint32_t)total;
    }
    // loop 2 (3^D cells), or a row of more than 32 particles: the slow
    // path rescans every candidate from an empty sum
    if (over) {
        S = (T)0;
        comp = (T)0;
        cnt = 0;
        nbr_scan<D, T, K>(P, pi, c, pos, start, body);
    } else if (K == 1) {
        nbr_walk<D, T, K>(P, pi, c, pos, start, [&](int idx) { return mbase[idx * mstride]; }, total, body);
    }
    density_finish<T>(P, i, S, total, over, vel, phat, rho_out, p_out, ovf, nnb);
    return cnt - 1;  // the self pair is in the sum (W(0)) but not a neighbour
}

// ---- accelerations (+ integration) -----------------------------------------
// v2, a2: |v|^2 and |a|^2 of a fluid particle in the working precision (the
// maxima are taken in it and widened once per block: the FP64 pipe of this
// GPU is narrow)
template <typename T>
struct ForceOut {
    T v2, a2;
    uint32_t pairs;
    bool bad;
};

// The constants of the momentum equation in the working precision, converted
// once per particle (a conversion from double per pair would load GB300's
// narrow FP64 pipe): 1/(2h), m C_g, the viscosity numerator, eps h^2.
template <typename T>
struct ForceConst {
    T hih, mCg, vnum, eh2;
};
template <typename T>
__device__ __forceinline__ ForceConst<T> force_const(const DevParams &P)
{
    return ForceConst<T>{(T)P.half_inv_h, (T)P.mCg, (T)P.visc_num, (T)P.eps_h2};
}

// The coefficient of one pair term of the momentum equation (pressure and
// Monaghan viscosity): a_i += coef * r_ij for particle i (velocity vi,
// P_i/rho_i^2 = Pi, density rhoi) and neighbour j (velocity and density vj,
// P_j/rho_j^2 = Pj) at r_ij = (rx, ry, rz), |r_ij|^2 = d2.
template <int D, typename T>
__device__ __forceinline__ T force_coef(const ForceConst<T> &K, const vec4_t<T> &vi, T Pi, T rhoi,
                                        const vec4_t<T> &vj, T Pj, T rx, T ry, T rz, T d2)
{
    const T u = Ar<T>::dist(d2) * K.hih;
    const T t = (T)1 - u;
    const T t3 = t * t * t;
    T vr = (vi.x - vj.x) * rx + (vi.y - vj.y) * ry;
    if (D == 3) vr += (vi.z - vj.z) * rz;
    const T visc = vr < (T)0 ? Ar<T>::div_ftz(K.vnum * vr, (rhoi + vj.w) * (d2 + K.eh2)) : (T)0;
    return K.mCg * t3 * (Pi + Pj + visc);
}

// a += coef * r, one rounding per component (the order of the terms is the
// walk's: rows in order, bits from the lowest).
template <int D, typename T>
__device__ __forceinline__ void force_add(T coef, T rx, T ry, T rz, T &ax, T &ay, T &az)
{
    ax = Ar<T>::fma(coef, rx, ax);
    ay = Ar<T>::fma(coef, ry, ay);
    if (D == 3) az = Ar<T>::fma(coef, rz, az);
}

// The force pass's per-particle tail: INTEGRATE: the new state of slot i
// (fluid: v += dt a, r += dt v; other kinds stay) to s; otherwise the
// accelerations to a0..a2; |v|^2 and |a|^2 into out.
template <int D, typename T, bool INTEGRATE>
__device__ __forceinline__ void force_finish(const DevParams &P, int i, uint8_t kd, const vec4_t<T> &vi, T ax, T ay,
                                             T az, const SortedBufs &sb, const sph_state &s, T *a0, T *a1, T *a2,
                                             ForceOut<T> &out)
{
    if (INTEGRATE) {
        T *vx = static_cast<T *>(s.v[0]);
        T *vy = static_cast<T *>(s.v[1]);
        T *vz = static_cast<T *>(s.v[2]);
        if (kd == SPH_FLUID) {
            // (SPH_DT_ADAPTIVE: the step size the last step's CFL bound set)
            const double dtd = P.adaptive ? *P.dt_next : P.dt;
            const T dt = (T)dtd;
            const T nvx = vi.x + dt * ax, nvy = vi.y + dt * ay;
            const T nvz = D == 3 ? vi.z + dt * az : (T)0;
            s.r[0][i] = sb.rs[0][i] + dtd * (double)nvx;
            s.r[1][i] = sb.rs[1][i] + dtd * (double)nvy;
            vx[i] = nvx;
            vy[i] = nvy;
            if (D == 3) {
                s.r[2][i] = sb.rs[2][i] + dtd * (double)nvz;
                vz[i] = nvz;
            }
            const T v2 = nvx * nvx + nvy * nvy + nvz * nvz;
            const T a2 = ax * ax + ay * ay + az * az;
            out.v2 = v2;
            out.a2 = a2;
            out.bad = !isfinite(v2) || !isfinite(a2);
        } else {
            s.r[0][i] = sb.rs[0][i];
            s.r[1][i] = sb.rs[1][i];
            vx[i] = vi.x;
            vy[i] = vi.y;
            if (D == 3) {
                s.r[2][i] = sb.rs[2][i];
                vz[i] = vi.z;
            }
        }
        s.id[i] = sb.id_s[i];
        s.kind[i] = kd;
    } else {
        a0[i] = ax;
        a1[i] = ay;
        if (D == 3) a2[i] = az;
        if (kd == SPH_FLUID) {
            const T a2 = ax * ax + ay * ay + az * az;
            out.a2 = a2;
            out.bad = !isfinite(a2);
        }
    }
}

// mbase: mask words of particle i at mbase[idx * mstride].  INTEGRATE: write
// the new state of slot i to s; otherwise the accelerations to a0..a2.
template <int D, typename T, bool INTEGRATE, int K = 1>
__device__ __forceinline__ ForceOut<T> dev_force(const DevParams &P, int i, const vec4_t<T> *__restrict__ pos,
                                              const vec4_t<T> *__restrict__ vel, const T *__restrict__ phat,
                                              const uint32_t *__restrict__ cell_s,
                                              const uint32_t *__restrict__ start, const uint32_t *mbase,
                                              int mstride, const uint8_t *__restrict__ ovf, const SortedBufs &sb,
                                              const sph_state &s, T *a0, T *a1, T *a2)
{
    ForceOut<T> out{(T)0, (T)0, 0u, false};
    const uint8_t kd = sb.kind_s[i];
    const vec4_t<T> vi = vel[i];
    T ax = (T)0, ay = (T)0, az = (T)0;
    if (kd == SPH_FLUID) {
        const vec4_t<T> pi = pos[i];
        const T Pi = phat[i];
        const T rhoi = vi.w;
        const ForceConst<T> fc = force_const<T>(P);
        uint32_t cnt = 0;
        // a_i = sum_j m (P_i + P_j + Pi_ij) (5 alpha_D / h^2) t^3 r_ij,
        // i.e. -sum_j m (...) grad_i W_ij with grad_i W_ij = -(5 alpha_D/h^2) t^3 r_ij;
        // the self pair has r_ij = 0 and adds nothing.
        auto body = [&](uint32_t j, T rx, T ry, T rz, T d2) {
            const T coef = force_coef<D, T>(fc, vi, Pi, rhoi, vel[j], phat[j], rx, ry, rz, d2);
            force_add<D, T>(coef, rx, ry, rz, ax, ay, az);
        };
        const uint32_t c = cell_s[i];
        if (!ovf[i]) {
            // (the walk visits the density pass's hits: nnb of them)
            cnt = sb.nnb[i];
            nbr_walk<D, T, K>(P, pi, c, pos, start, [&](int idx) { return mbase[idx * mstride]; }, (int)cnt, body);
        } else {
            nbr_scan<D, T, K>(P, pi, c, pos, start, [&](uint32_t j, T rx, T ry, T rz, T d2) {
                body(j, rx, ry, rz, d2);
                ++cnt;
            });
        }
        out.pairs = cnt - 1;  // minus the self pair
        ax += (T)P.g[0];
        ay += (T)P.g[1];
        if (D == 3) az += (T)P.g[2];
    }
    force_finish<D, T, INTEGRATE>(P, i, kd, vi, ax, ay, az, sb, s, a0, a1, a2, out);
    if (out.bad) {
        out.v2 = (T)0;
        out.a2 = (T)0;
    }
    return out;
}

// ---- small cases: a team of lanes per particle (row stencil) ---------------
// With few particles the pair passes are bound by the length of one lane's
// walk, not by the SMs.  TEAM consecutive lanes of a warp then share particle
// i: the rows of its stencil are dealt to them round-robin (row r to lane
// r mod TEAM), each lane tests or walks its row, and the row sums join the
// particle's sums in the single lane's order (dev_density: the row partial
// sums into the compensated sum; dev_force: every hit's term, see below), so
// the results are the same bit for bit.  Every lane of the warp calls these
// (valid = false past the last particle): the shuffles need the whole warp.

template <int D, typename T, int TEAM>
__device__ __forceinline__ uint32_t dev_density_team(const DevParams &P, int i, bool valid, int tl,
                                                     const vec4_t<T> *__restrict__ pos,
                                                     const uint32_t *__restrict__ cell_s,
                                                     const uint32_t *__restrict__ start, vec4_t<T> *vel, T *phat,
                                                     T *rho_out, T *p_out, uint32_t *mbase, int mstride,
                                                     uint8_t *ovf, uint16_t *nnb)
{
    constexpr int NR = Sten<D, 2>::NR;
    vec4_t<T> pi;
    pi.x = pi.y = pi.z = pi.w = (T)0;
    uint32_t c = P.cell_off;
    if (valid) {
        pi = pos[i];
        c = cell_s[i];
    }
    const CellXYZ cc = decode_cell(P, c);
    const RowTrim tr = row_trim<D, T>(P, pi, cc);
    const T hih = (T)P.half_inv_h;
    T S = (T)0, comp = (T)0;
    int total = 0;
    uint32_t rows = 0;
    bool over = false;
#pragma unroll 1
    for (int r0 = 0; r0 < NR; r0 += TEAM) {
        const int idx = r0 + tl;
        T sr = (T)0;
        uint32_t w = 0;
        if (valid && idx < NR) {
            int row, lo, hi, dy, dz;
            row_at<D>(P, cc, idx, row, lo, hi, dy, dz);
            w = row_test<D, T>(P, pi, row, lo, hi, dy, dz, tr, pos, start, over,
                               [&](uint32_t, T, T, T, T d2) { density_hit<T>(d2, hih, sr); });
            mbase[idx * mstride] = w;
        }
#pragma unroll
        for (int t = 0; t < TEAM; ++t) {
            const T y = __shfl_sync(0xffffffffu, sr, t, TEAM);
            const uint32_t wt = __shfl_sync(0xffffffffu, w, t, TEAM);
            if (r0 + t < NR) {
                kahan_add<T>(S, comp, y);
                total += __popc(wt);
                rows |= (wt != 0u ? 1u : 0u) << (r0 + t);
            }
        }
    }
    int ov = over ? 1 : 0;
#pragma unroll
    for (int o = 1; o < TEAM; o <<= 1) ov |= __shfl_xor_sync(0xffffffffu, ov, o, TEAM);
    if (!valid || tl != 0) return 0;
    mbase[NR * mstride] = rows;
    uint32_t cnt = (uint32_t)total;
    if (ov) {
        // a row of more than 32 particles: every candidate again, one lane
        S = (T)0;
        comp = (T)0;
        cnt = 0;
        nbr_scan<D, T, 2>(P, pi, c, pos, start, [&](uint32_t, T, T, T, T d2) {
            T w = (T)0;
            density_hit<T>(d2, hih, w);
            kahan_add<T>(S, comp, w);
            ++cnt;
        });
    }
    density_finish<T>(P, i, S, total, ov != 0, vel, phat, rho_out, p_out, ovf, nnb);
    return cnt - 1;
}

// The force pass: the terms of a particle's hits are computed by its team
// (row r by lane r mod TEAM) into buf, at the positions of the one-lane walk
// (rows in order, bits from the lowest), and the team's first lane adds them
// in that order, one fused multiply-add per component as the walk does.
// buf: kTeamHits entries (coef, x, y, z) per particle and round of rows; a
// round with more hits sends the particle to the one-lane walk.
constexpr int kTeamHits = 64;

template <int D, typename T, bool INTEGRATE, int TEAM>
__device__ __forceinline__ ForceOut<T> dev_force_team(const DevParams &P, int i, bool valid, int tl,
                                                      const vec4_t<T> *__restrict__ pos,
                                                      const vec4_t<T> *__restrict__ vel, const T *__restrict__ phat,
                                                      const uint32_t *__restrict__ cell_s,
                                                      const uint32_t *__restrict__ start, const uint32_t *mbase,
                                                      int mstride, const uint8_t *__restrict__ ovf,
                                                      const SortedBufs &sb, const sph_state &s, vec4_t<T> *buf,
                                                      T *a0, T *a1, T *a2)
{
    constexpr int NR = Sten<D, 2>::NR;
    ForceOut<T> out{(T)0, (T)0, 0u, false};
    uint8_t kd = 0;
    vec4_t<T> pi, vi;
    pi.x = pi.y = pi.z = pi.w = (T)0;
    vi = pi;
    T Pi = (T)0;
    uint32_t c = P.cell_off;
    bool walk = false;
    if (valid) {
        kd = sb.kind_s[i];
        vi = vel[i];
        if (kd == SPH_FLUID) {
            pi = pos[i];
            Pi = phat[i];
            c = cell_s[i];
            walk = !ovf[i];
        }
    }
    const T rhoi = vi.w;
    const ForceConst<T> fc = force_const<T>(P);
    const T cs = cell_edge<T>(P);
    const int cb = (int)c + max(-2, -(int)pi.w);
    const uint32_t rows = walk ? mbase[NR * mstride] : 0u;
    T ax = (T)0, ay = (T)0, az = (T)0;
    bool spill = false;  // (team-uniform) a round held more than kTeamHits hits
#pragma unroll 1
    for (int r0 = 0; r0 < NR; r0 += TEAM) {
        const int idx = r0 + tl;
        const bool mine = idx < NR && ((rows >> idx) & 1u);
        uint32_t w = mine ? mbase[idx * mstride] : 0u;
        const int n = __popc(w);
        int incl = n;
#pragma unroll
        for (int o = 1; o < TEAM; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o, TEAM);
            if (tl >= o) incl += t;
        }
        const int rtotal = __shfl_sync(0xffffffffu, incl, TEAM - 1, TEAM);
        spill = spill || rtotal > kTeamHits;
        if (!spill && n) {
            int q = incl - n;
            const StencilEntry e = P.stab[idx];
            const uint32_t a = start[cb + e.dcell];
            T fy = pi.y, fz = pi.z;
            if (sizeof(T) == 4) {
                fy = Ar<T>::sub(pi.y, (T)e.sy);
                if (D == 3) fz = Ar<T>::sub(pi.z, (T)e.sz);
            }
            while (w) {
                const uint32_t j = a + (uint32_t)(__ffs(w) - 1);
                w &= w - 1u;
                if (!SPH_IN_BOUNDS(P, j < P.chk_cap)) break;
                const vec4_t<T> pj = pos[j];
                const T rx = row_dx<T>(pi, pj, cs);
                const T ry = Ar<T>::sub(fy, pj.y);
                T d2 = Ar<T>::mul(rx, rx);
                d2 = Ar<T>::fma(ry, ry, d2);
                T rz = (T)0;
                if (D == 3) {
                    rz = Ar<T>::sub(fz, pj.z);
                    d2 = Ar<T>::fma(rz, rz, d2);
                }
                vec4_t<T> term;
                term.x = force_coef<D, T>(fc, vi, Pi, rhoi, vel[j], phat[j], rx, ry, rz, d2);
                term.y = rx;
                term.z = ry;
                term.w = rz;
                buf[q++] = term;
            }
        }
        __syncwarp();
        if (tl == 0 && !spill) {
            for (int q = 0; q < rtotal; ++q) {
                const vec4_t<T> term = buf[q];
                force_add<D, T>(term.x, term.y, term.z, term.w, ax, ay, az);
            }
        }
        __syncwarp();
    }
    if (!valid || tl != 0) return out;
    if (kd == SPH_FLUID) {
        uint32_t cnt = 0;
        auto body = [&](uint32_t j, T rx, T ry, T rz, T d2) {
            const T coef = force_coef<D, T>(fc, vi, Pi, rhoi, vel[j], phat[j], rx, ry, rz, d2);
            force_add<D, T>(coef, rx, ry, rz, ax, ay, az);
        };
        if (walk) {
            cnt = sb.nnb[i];
            if (spill) {
                // the one-lane walk over every hit
                ax = ay = az = (T)0;
                walk_rows<D, T>(P, pi, c, pos, start, [&](int q) { return mbase[q * mstride]; }, (int)cnt, body);
            }
        } else {
            // a row of more than 32 particles: every candidate, one lane
            nbr_scan<D, T, 2>(P, pi, c, pos, start, [&](uint32_t j, T rx, T ry, T rz, T d2) {
                body(j, rx, ry, rz, d2);
                ++cnt;
            });
        }
        out.pairs = cnt - 1;
        ax += (T)P.g[0];
        ay += (T)P.g[1];
        if (D == 3) az += (T)P.g[2];
    }
    force_finish<D, T, INTEGRATE>(P, i, kd, vi, ax, ay, az, sb, s, a0, a1, a2, out);
    if (out.bad) {
        out.v2 = (T)0;
        out.a2 = (T)0;
    }
    return out;
}

template <typename V>
__device__ __forceinline__ V warp_max(V v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Raise *addr (the bit pattern of a non-negative double; such doubles order
// like their bit patterns) to v.  A block issues the atomic only when its
// value exceeds the one already recorded: the recorded value only grows
// during a kernel, so a stale read costs at most an extra atomic, and the
// thousands of blocks of a launch no longer serialise on one address.
__device__ __forceinline__ void raise_max(unsigned long long *addr, double v)
{
    if (!(v > 0.0)) return;
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    if (b > __ldcg(addr)) atomicMax(addr, b);
}

}  // namespace sph
