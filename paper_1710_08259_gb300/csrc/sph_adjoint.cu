// sph_adjoint.cu -- reverse mode of one WCSPH step (sph_step_adjoint).
//
// The step differentiated is the forward step of sph_pairs.cu: summation
// density (Section 5.1 SPH interpolant with A = rho), Tait EOS with the
// negative-pressure clamp, the symmetric pressure term of Eq. (diffop1) with
// the artificial viscosity of Section 5.1.1, then v' = v + dt a, r' = r + dt v'
// on fluid particles.  Neighbour sets are frozen at the step's input (W, W'
// and W'' vanish at the support radius, so set changes carry no derivative).
//
// Notation: r_ij = r_i - r_j, d = |r_ij|, t = 1 - d/(2h), F_ij = m C t^3 with
// C = 5 alpha_D / h^2 (so m grad_i W_ij = -F_ij r_ij), P_i = p_i / rho_i^2,
// s_ij = P_i + P_j + Pi_ij, and for fluid i a_i = g + sum_j s_ij F_ij r_ij.
// With abar the acceleration adjoint (zero on boundary particles) and
// dA = abar_i - abar_j, one unordered pair contributes
//   sigma_ij = F (r_ij . dA)                    to Pbar_i, Pbar_j and Pibar_ij,
//   s_ij [F dA + (r_ij . dA) F'(d) r_ij / d]    to rbar_i (minus to rbar_j),
// plus the partials of Pi_ij in v_ij . r_ij, d^2, rho_i, rho_j and alpha, and
// the density adjoint -(rhobar_i + rhobar_j) F r_ij to rbar_i.  Every
// expression is symmetric in (i, j) up to the sign of r_ij / v_ij, so each
// particle GATHERS its own share over its neighbours: no atomics, the result
// is deterministic.
//
// Kernels per reverse step (after the forward build and density pass that
// recreate the step's neighbour masks, densities and pressures):
//   k_adj_prep : vtilde = vbar' + dt rbar', abar = dt vtilde (fluid)
//   k_adj_rho  : Pbar_i = sum_j sigma_ij, rhobar_i = Pbar_i dP/drho + Pi terms,
//                per-block partial sums of alphabar, which the last block to
//                finish adds up in block order (deterministic)
//   k_adj_rv   : rbar_i, vbar_i, written to the caller's order
#include <cuda_runtime.h>

#include "sph_internal.cuh"
#include "sph_nbr.cuh"

namespace sph {

template <int D, typename T>
__global__ void __launch_bounds__(kBlock) k_adj_prep(DevParams P, int n, const uint8_t *__restrict__ kind_s,
                                                     sph_grad g1, vec4_t<T> *abar, vec4_t<T> *vt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T *vb0 = static_cast<const T *>(g1.v_bar[0]);
    const T *vb1 = static_cast<const T *>(g1.v_bar[1]);
    const T *vb2 = static_cast<const T *>(g1.v_bar[2]);
    vec4_t<T> w, a;
    w.x = vb0[i];
    w.y = vb1[i];
    w.z = D == 3 ? vb2[i] : (T)0;
    w.w = (T)0;
    a.x = a.y = a.z = a.w = (T)0;
    if (kind_s[i] == SPH_FLUID) {
        w.x += (T)(P.dt * g1.r_bar[0][i]);
        w.y += (T)(P.dt * g1.r_bar[1][i]);
        if (D == 3) w.z += (T)(P.dt * g1.r_bar[2][i]);
        a.x = (T)P.dt * w.x;
        a.y = (T)P.dt * w.y;
        a.z = (T)P.dt * w.z;
    }
    vt[i] = w;
    abar[i] = a;
}

// dP/drho for P = p / rho^2 with the (clamped) Tait law.  The clamp's
// branch is the one the forward step took: clamped iff its p (in
// Phat = p / rho^2) is not positive.  (Deciding again from rho / rho_ref < 1
// would disagree with the forward step for particles within rounding of the
// kink p = 0, and give them the other side's derivative.)
template <typename T>
__device__ __forceinline__ T dP_drho(const DevParams &P, T rho, T Phat)
{
    const T x = rho * (T)P.inv_rho_ref;
    T dp = (T)0;
    if (!(P.clamp && !(Phat > (T)0))) {
        T xg = (T)1;
        for (int k = 0; k < P.gamma - 1; ++k) xg *= x;
        dp = (T)P.Bg_rho_ref * xg;  // B gamma / rho_ref (rho/rho_ref)^(gamma-1)
    }
    return (dp - (T)2 * Phat * rho) / (rho * rho);
}

// TEAM > 1 (cells of edge h, small cases): TEAM lanes per particle, the
// stencil rows dealt to them round-robin, their sums joined by team_sum.
template <int D, typename T, int K, int TEAM>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 8 : 4) k_adj_rho(DevParams P, int n, const vec4_t<T> *__restrict__ pos,
                                                    const vec4_t<T> *__restrict__ vel,
                                                    const T *__restrict__ phat,
                                                    const uint32_t *__restrict__ cell_s,
                                                    const uint32_t *__restrict__ start,
                                                    const uint32_t *__restrict__ gmask,
                                                    const uint8_t *__restrict__ ovf,
                                                    const vec4_t<T> *__restrict__ abar, T *rhobar,
                                                    double *alpha_part, unsigned int *ticket,
                                                    double *alpha_bar)
{
    constexpr int NC = Sten<D, K>::NC;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g / TEAM, tl = g % TEAM;
    double ab = 0.0;
    if (TEAM > 1 || i < n) {
        const bool valid = i < n;
        vec4_t<T> pi, vi, ai;
        pi.x = pi.y = pi.z = pi.w = (T)0;
        vi = ai = pi;
        if (valid) {
            pi = pos[i];
            vi = vel[i];
            ai = abar[i];
        }
        const T rhoi = vi.w;
        const T hih = (T)P.half_inv_h, mCg = (T)P.mCg, eh2 = (T)P.eps_h2, vnum1 = (T)P.visc_num1,
                alpha = (T)P.alpha;
        T Pbar = (T)0, rb = (T)0, abl = (T)0;
        auto body = [&](uint32_t j, T rx, T ry, T rz, T d2) {
            if (j == (uint32_t)i) return;
            const T u = Ar<T>::dist_ftz(d2) * hih;
            const T t = (T)1 - u;
            const T F = mCg * t * t * t;
            const vec4_t<T> aj = abar[j];
            T rdA = rx * (ai.x - aj.x) + ry * (ai.y - aj.y);
            if (D == 3) rdA += rz * (ai.z - aj.z);
            const T sigma = F * rdA;
            Pbar += sigma;
            const vec4_t<T> vj = vel[j];
            T vr = (vi.x - vj.x) * rx + (vi.y - vj.y) * ry;
            if (D == 3) vr += (vi.z - vj.z) * rz;
            if (vr < (T)0) {
                const T rs = rhoi + vj.w;
                const T Pi1 = Ar<T>::div_ftz(vnum1 * vr, rs * (d2 + eh2));  // Pi per unit alpha
                rb -= sigma * alpha * Pi1 / rs;
                abl += sigma * Pi1;
            }
        };
        if (TEAM == 1) {
            const uint32_t c = cell_s[i];
            if (!ovf[i])
                nbr_masked<D, T, K>(P, pi, c, pos, start, [&](int idx) { return gmask[mask_index(NC, idx)]; },
                                    body);
            else
                nbr_scan<D, T, K>(P, pi, c, pos, start, body);
        } else {
            constexpr int NR = Sten<D, 2>::NR;
            const uint32_t c = valid ? cell_s[i] : P.cell_off;
            const CellXYZ cc = decode_cell(P, c);
            const bool walk = valid && !ovf[i];
            const uint32_t *mb = gmask + (size_t)(i / kBlock) * NC * kBlock + (i % kBlock);
#pragma unroll 1
            for (int r0 = 0; r0 < NR; r0 += TEAM) {
                const int idx = r0 + tl;
                if (walk && idx < NR) masked_row<D, T>(P, pi, cc, idx, mb[idx * kBlock], pos, start, body);
            }
            Pbar = team_sum<TEAM>(Pbar);
            rb = team_sum<TEAM>(rb);
            abl = team_sum<TEAM>(abl);
            if (valid && tl == 0 && !walk) {
                Pbar = rb = abl = (T)0;
                nbr_scan<D, T, K>(P, pi, c, pos, start, body);
            }
        }
        if (valid && tl == 0) {
            rhobar[i] = Pbar * dP_drho<T>(P, rhoi, phat[i]) + rb;
            ab = 0.5 * (double)abl;  // each unordered pair is met from both ends
        }
    }
    ab = warp_sum(ab);
    __shared__ double ws[kBlock / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = ab;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tsum = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) tsum += ws[w];
        alpha_part[blockIdx.x] = tsum;
    }
    if (!alpha_bar) return;
    // the last block to finish adds the partials in block order (so the sum
    // does not depend on which block finishes last) and resets the ticket
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += 32) s += __ldcg(&alpha_part[b]);
    s = warp_sum(s);
    if (threadIdx.x == 0) {
        *alpha_bar += s;
        *ticket = 0u;
    }
}

template <int D, typename T, int K, int TEAM>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 6 : 3) k_adj_rv(DevParams P, int n, const vec4_t<T> *__restrict__ pos,
                                                   const vec4_t<T> *__restrict__ vel,
                                                   const T *__restrict__ phat,
                                                   const uint32_t *__restrict__ cell_s,
                                                   const uint32_t *__restrict__ start,
                                                   const uint32_t *__restrict__ gmask,
                                                   const uint8_t *__restrict__ ovf,
                                                   const vec4_t<T> *__restrict__ abar,
                                                   const vec4_t<T> *__restrict__ vt,
                                                   const T *__restrict__ rhobar, const uint32_t *__restrict__ src,
                                                   sph_grad g1, sph_grad g0)
{
    constexpr int NC = Sten<D, K>::NC;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g / TEAM, tl = g % TEAM;
    const bool valid = i < n;
    if (TEAM == 1 && !valid) return;
    vec4_t<T> pi, vi, ai;
    pi.x = pi.y = pi.z = pi.w = (T)0;
    vi = ai = pi;
    T Pi_i = (T)0, rbi = (T)0;
    if (valid) {
        pi = pos[i];
        vi = vel[i];
        ai = abar[i];
        Pi_i = phat[i];
        rbi = rhobar[i];
    }
    const T rhoi = vi.w;
    const T hih = (T)P.half_inv_h, mCg = (T)P.mCg, eh2 = (T)P.eps_h2, vnum = (T)P.visc_num;
    const T dG = (T)(-1.5) * (T)P.mCg * (T)(1.0 / P.h);  // dF/dd = dG t^2
    T gx = (T)0, gy = (T)0, gz = (T)0, hx = (T)0, hy = (T)0, hz = (T)0;
    auto body = [&](uint32_t j, T rx, T ry, T rz, T d2) {
        if (j == (uint32_t)i) return;
        const T d = Ar<T>::dist_ftz(d2);
        const T t = (T)1 - d * hih;
        const T F = mCg * t * t * t;
        const vec4_t<T> aj = abar[j], vj = vel[j];
        const T dAx = ai.x - aj.x, dAy = ai.y - aj.y, dAz = D == 3 ? ai.z - aj.z : (T)0;
        T rdA = rx * dAx + ry * dAy;
        if (D == 3) rdA += rz * dAz;
        const T sigma = F * rdA;
        const T vx = vi.x - vj.x, vy = vi.y - vj.y, vz = D == 3 ? vi.z - vj.z : (T)0;
        T vr = vx * rx + vy * ry;
        if (D == 3) vr += vz * rz;
        T visc = (T)0, Pvr = (T)0, Pd2 = (T)0;
        if (vr < (T)0) {
            const T den = (rhoi + vj.w) * (d2 + eh2);
            Pvr = Ar<T>::div_ftz(vnum, den);
            visc = Pvr * vr;
            Pd2 = -visc / (d2 + eh2);
        }
        const T s = Pi_i + phat[j] + visc;
        // force term: s [F dA + (r . dA) F'(d) r / d]
        const T G = d > (T)0 ? dG * t * t * rdA / d : (T)0;
        // viscosity: sigma (Pvr v + 2 Pd2 r); density: -(rhobar_i + rhobar_j) F r
        const T cr = s * G + (T)2 * sigma * Pd2 - (rbi + rhobar[j]) * F;
        const T cv = sigma * Pvr;
        gx += s * F * dAx + cr * rx + cv * vx;
        gy += s * F * dAy + cr * ry + cv * vy;
        if (D == 3) gz += s * F * dAz + cr * rz + cv * vz;
        hx += cv * rx;
        hy += cv * ry;
        if (D == 3) hz += cv * rz;
    };
    if (TEAM == 1) {
        const uint32_t c = cell_s[i];
        if (!ovf[i])
            nbr_masked<D, T, K>(P, pi, c, pos, start, [&](int idx) { return gmask[mask_index(NC, idx)]; }, body);
        else
            nbr_scan<D, T, K>(P, pi, c, pos, start, body);
    } else {
        constexpr int NR = Sten<D, 2>::NR;
        const uint32_t c = valid ? cell_s[i] : P.cell_off;
        const CellXYZ cc = decode_cell(P, c);
        const bool walk = valid && !ovf[i];
        const uint32_t *mb = gmask + (size_t)(i / kBlock) * NC * kBlock + (i % kBlock);
#pragma unroll 1
        for (int r0 = 0; r0 < NR; r0 += TEAM) {
            const int idx = r0 + tl;
            if (walk && idx < NR) masked_row<D, T>(P, pi, cc, idx, mb[idx * kBlock], pos, start, body);
        }
        gx = team_sum<TEAM>(gx);
        gy = team_sum<TEAM>(gy);
        hx = team_sum<TEAM>(hx);
        hy = team_sum<TEAM>(hy);
        if (D == 3) {
            gz = team_sum<TEAM>(gz);
            hz = team_sum<TEAM>(hz);
        }
        if (!valid || tl != 0) return;
        if (!walk) {
            gx = gy = gz = hx = hy = hz = (T)0;
            nbr_scan<D, T, K>(P, pi, c, pos, start, body);
        }
    }
    const vec4_t<T> w = vt[i];
    const uint32_t k = src[i];
    g0.r_bar[0][k] = g1.r_bar[0][i] + (double)gx;
    g0.r_bar[1][k] = g1.r_bar[1][i] + (double)gy;
    static_cast<T *>(g0.v_bar[0])[k] = w.x + hx;
    static_cast<T *>(g0.v_bar[1])[k] = w.y + hy;
    if (D == 3) {
        g0.r_bar[2][k] = g1.r_bar[2][i] + (double)gz;
        static_cast<T *>(g0.v_bar[2])[k] = w.z + hz;
    }
}

static inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

template <int D, typename T>
static void adjoint_impl(const DevParams &P, int n, const CellBufs &cb, const SortedBufs &sb, const AdjBufs &ab,
                         const sph_grad &g1, const sph_grad &g0, double *alpha_bar, cudaStream_t st)
{
    using V4 = vec4_t<T>;
    const int nb = blocks_for(n, kBlock);
    const V4 *pos = static_cast<const V4 *>(sb.pos);
    const V4 *vel = static_cast<const V4 *>(sb.vel);
    const T *ph = static_cast<const T *>(sb.phat);
    V4 *abar = static_cast<V4 *>(ab.abar);
    V4 *vt = static_cast<V4 *>(ab.vt);
    T *rhobar = static_cast<T *>(ab.rhobar);
    k_adj_prep<D, T><<<nb, kBlock, 0, st>>>(P, n, sb.kind_s, g1, abar, vt);
    const int team = P.K == 2 ? pair_team(n) : 1;
    auto krho = P.K == 2 ? k_adj_rho<D, T, 2, 1> : k_adj_rho<D, T, 1, 1>;
    auto krv = P.K == 2 ? k_adj_rv<D, T, 2, 1> : k_adj_rv<D, T, 1, 1>;
    if (team == 8) {
        krho = k_adj_rho<D, T, 2, 8>;
        krv = k_adj_rv<D, T, 2, 8>;
    } else if (team == 4) {
        krho = k_adj_rho<D, T, 2, 4>;
        krv = k_adj_rv<D, T, 2, 4>;
    } else if (team == 2) {
        krho = k_adj_rho<D, T, 2, 2>;
        krv = k_adj_rv<D, T, 2, 2>;
    }
    const int nbt = blocks_for((int)((long long)n * team), kBlock);
    krho<<<nbt, kBlock, 0, st>>>(P, n, pos, vel, ph, sb.cell_s, cb.cell_start, sb.mask, sb.ovf, abar, rhobar,
                                 ab.alpha_part, ab.alpha_ticket, alpha_bar);
    krv<<<nbt, kBlock, 0, st>>>(P, n, pos, vel, ph, sb.cell_s, cb.cell_start, sb.mask, sb.ovf, abar, vt, rhobar,
                                sb.src, g1, g0);
}

cudaError_t launch_adjoint(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                           const AdjBufs &ab, const sph_grad &g1, const sph_grad &g0, double *alpha_bar,
                           cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (P.dim == 2) {
        if (f32) adjoint_impl<2, float>(P, n, cb, sb, ab, g1, g0, alpha_bar, st);
        else adjoint_impl<2, double>(P, n, cb, sb, ab, g1, g0, alpha_bar, st);
    } else {
        if (f32) adjoint_impl<3, float>(P, n, cb, sb, ab, g1, g0, alpha_bar, st);
        else adjoint_impl<3, double>(P, n, cb, sb, ab, g1, g0, alpha_bar, st);
    }
    return cudaGetLastError();
}

}  // namespace sph
