// sph_model.cu -- the faces of the computational domain (Section 3.2.1:
// cut-off, symmetric and periodic) as neighbour images; the Example 1a step
// in the paper's own form (Section 5.1.1, Eq. SPH_fluid_continuity to
// Eq. SPH_fluid_momentum, in the equation order of Appendix A); the SPH
// sampling operator of the performance benchmark (Section 6).
//
// Same GB300 design as sph_pairs.cu: gather-only pair loops (no atomics in
// the numerics), one thread per particle of the canonical order, FP32 pair
// arithmetic from cell-relative float offsets, candidate tests recorded as
// 32-bit hit masks by the first pass and walked by the second.  What differs
// is the stencil: a stencil cell outside the grid is not dropped but mapped
// to the cell that holds its images:
//   periodic face : the cell on the other side of the grid; the frame shift
//                   stays the unwrapped offset d * cs (F32; the offsets are
//                   cell-relative) or becomes -+L (F64, absolute positions);
//   symmetric face: the particle's own cell, reflected: x_ij = (p_i - S) +
//                   p_j with S = 0 or 2 cs (F32), 2 w (F64, w the face), and
//                   the image's velocity component along that axis negated;
//   cut-off face  : nothing.
// (sph_images.cuh).
#include <cuda_runtime.h>

#include "sph_images.cuh"
#include "sph_internal.cuh"
#include "sph_nbr.cuh"
#include "sph_phases.cuh"

namespace sph {
namespace {

template <typename V>
__device__ __forceinline__ void block_add(V v, unsigned long long *dst)
{
    __shared__ unsigned long long ws[kBlock / 32];
    unsigned long long x = warp_sum((unsigned long long)v);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kBlock / 32; ++w) t += ws[w];
        if (t) atomicAdd(dst, t);
    }
}

// ---- continuity + linear EOS (eq1, eq2, eq3) ------------------------------
// rho_i' = rho_i - dt rho_i m (5 alpha_D / h^2) sum_j t^3 (v_ij . r_ij) / rho_j
// (grad_i W_ij = -(5 alpha_D / h^2) t^3 r_ij, t = 1 - q/2), p' = c^2 (rho' -
// rho0); the sum runs over the neighbour images (the self pair adds 0).

template <int D, typename T>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? (D == 2 ? 12 : 8) : 4)
    k_cont(DevParams P, int n, const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ cell_s,
           const uint32_t *__restrict__ start, const vec4_t<T> *__restrict__ vel, T *phat, T *rho1, T *p1,
           Accum *acc, uint32_t *gmask, uint8_t *ovf, uint16_t *nnb)
{
    constexpr int NC = Stencil<D>::NC;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long pairs = 0;
    if (i < n) {
        const vec4_t<T> pi = pos[i];
        const vec4_t<T> vi = vel[i];
        const uint32_t clin = cell_s[i];
        const CellXYZ cc = decode_cell(P, clin);
        uint32_t *mbase = gmask + (size_t)blockIdx.x * NC * kBlock + threadIdx.x;
        bool over;
        const int total = image_masks<D, T>(P, pi, cc, clin, pos, start, mbase, over);
        const T hih = (T)P.half_inv_h;
        T sum = (T)0;
        uint32_t cnt = 0;
        auto body = [&](uint32_t j, T rx, T ry, T rz, T d2, const ImageCell<T> &ic) {
            const T u = Ar<T>::dist_ftz(d2) * hih;
            const T t = (T)1 - u;
            const T t3 = t * t * t;
            const vec4_t<T> vj = vel[j];
            // v_ij . r_ij = (s v_i - v_j) . x'
            T vr = (ic.s[0] * vi.x - vj.x) * rx + (ic.s[1] * vi.y - vj.y) * ry;
            if (D == 3) vr += (ic.s[2] * vi.z - vj.z) * rz;
            sum += t3 * Ar<T>::div_ftz(vr, vj.w);
            ++cnt;
        };
        if (!over)
            walk_images<D, T>(P, pi, cc, clin, pos, start, [&](int idx) { return mbase[idx * kBlock]; }, total,
                              body);
        else
            scan_images<D, T>(P, pi, cc, clin, pos, start, body);
        nnb[i] = (uint16_t)total;
        ovf[i] = over ? 1 : 0;
        const T rho = vi.w;
        const T rn = rho - ((T)P.dt * rho) * ((T)P.mCg * sum);
        const T p = (T)P.c2 * (rn - (T)P.rho0);
        phat[i] = p / (rn * rn);
        if (rho1) rho1[i] = rn;
        if (p1) p1[i] = p;
        pairs = cnt - 1;  // the self pair is visited but is not a neighbour
    }
    block_add(pairs, &acc->n_pairs);
}

// ---- momentum (eq4, eq5) and integration (eq6, eq7) ------------------------
// a_i = sum_j m (5 alpha_D / h^2) t^3 (P_i + P_j + Pi_ij) r_ij + g, P = p'/rho'^2,
// Pi_ij = -alpha c h (v_ij . r_ij) / (rho_i' |r_ij|^2) when v_ij . r_ij < 0.

template <int D, typename T, bool INTEGRATE>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? (D == 2 ? 12 : 8) : 4)
    k_mom(DevParams P, int n, const vec4_t<T> *__restrict__ pos, const vec4_t<T> *__restrict__ vel,
          const T *__restrict__ phat, const T *__restrict__ rho1, const uint32_t *__restrict__ cell_s,
          const uint32_t *__restrict__ start, const uint32_t *__restrict__ gmask, const uint8_t *__restrict__ ovf,
          SortedBufs sb, sph_state s, T *a0, T *a1, T *a2, Accum *acc, uint32_t *status)
{
    constexpr int NC = Stencil<D>::NC;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // squares for the diagnostics in the working precision (narrow FP64 pipe)
    T v2 = (T)0, a2m = (T)0;
    unsigned long long pairs = 0;
    bool bad = false;
    if (i < n) {
        const uint8_t kd = sb.kind_s[i];
        const vec4_t<T> vi = vel[i];
        T ax = (T)0, ay = (T)0, az = (T)0;
        if (kd == SPH_FLUID) {
            const vec4_t<T> pi = pos[i];
            const uint32_t clin = cell_s[i];
            const CellXYZ cc = decode_cell(P, clin);
            const uint32_t *mbase = gmask + (size_t)blockIdx.x * NC * kBlock + threadIdx.x;
            const T Pi = phat[i];
            const T rhoi = rho1[i];
            const T hih = (T)P.half_inv_h, mCg = (T)P.mCg, vnum = (T)P.visc1a;
            uint32_t cnt = 0;
            auto body = [&](uint32_t j, T rx, T ry, T rz, T d2, const ImageCell<T> &ic) {
                const T u = Ar<T>::dist_ftz(d2) * hih;
                const T t = (T)1 - u;
                const T t3 = t * t * t;
                const vec4_t<T> vj = vel[j];
                T vr = (ic.s[0] * vi.x - vj.x) * rx + (ic.s[1] * vi.y - vj.y) * ry;
                if (D == 3) vr += (ic.s[2] * vi.z - vj.z) * rz;
                const T visc = vr < (T)0 ? Ar<T>::div_ftz(vnum * vr, rhoi * d2) : (T)0;
                const T coef = mCg * t3 * (Pi + phat[j] + visc);
                ax += coef * ic.s[0] * rx;
                ay += coef * ic.s[1] * ry;
                if (D == 3) az += coef * ic.s[2] * rz;
                ++cnt;
            };
            if (!ovf[i])
                walk_images<D, T>(P, pi, cc, clin, pos, start, [&](int idx) { return mbase[idx * kBlock]; },
                                  (int)sb.nnb[i], body);
            else
                scan_images<D, T>(P, pi, cc, clin, pos, start, body);
            pairs = cnt - 1;
            ax += (T)P.g[0];
            ay += (T)P.g[1];
            if (D == 3) az += (T)P.g[2];
        }
        if (INTEGRATE) {
            T *vx = static_cast<T *>(s.v[0]);
            T *vy = static_cast<T *>(s.v[1]);
            T *vz = static_cast<T *>(s.v[2]);
            if (kd == SPH_FLUID) {
                const T dt = (T)P.dt;
                const T nv[3] = {vi.x + dt * ax, vi.y + dt * ay, D == 3 ? vi.z + dt * az : (T)0};
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    double x = sb.rs[k][i] + P.dt * (double)nv[k];
                    if (P.bc[k] == SPH_BC_PERIODIC) {
                        if (x < P.dom_min[k]) x = x + P.per[k];
                        else if (x >= P.hi[k]) x = x - P.per[k];
                    }
                    s.r[k][i] = x;
                }
                vx[i] = nv[0];
                vy[i] = nv[1];
                if (D == 3) vz[i] = nv[2];
                v2 = nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2];
                a2m = ax * ax + ay * ay + az * az;
                bad = !isfinite(v2) || !isfinite(a2m);
            } else {
#pragma unroll
                for (int k = 0; k < D; ++k) s.r[k][i] = sb.rs[k][i];
                vx[i] = vi.x;
                vy[i] = vi.y;
                if (D == 3) vz[i] = vi.z;
            }
            s.id[i] = sb.id_s[i];
            s.kind[i] = kd;
        } else {
            a0[i] = ax;
            a1[i] = ay;
            if (D == 3) a2[i] = az;
            if (kd == SPH_FLUID) {
                a2m = ax * ax + ay * ay + az * az;
                bad = !isfinite(a2m);
            }
        }
        if (bad) {
            v2 = (T)0;
            a2m = (T)0;
        }
    }
    if (bad) atomicOr(status, SPH_STATUS_NAN);
    const T v2max = warp_max(v2);
    const T a2max = warp_max(a2m);
    const unsigned long long fp = warp_sum(pairs);
    __shared__ T wv[kBlock / 32], wa[kBlock / 32];
    __shared__ unsigned long long wp[kBlock / 32];
    if ((threadIdx.x & 31) == 0) {
        wv[threadIdx.x >> 5] = v2max;
        wa[threadIdx.x >> 5] = a2max;
        wp[threadIdx.x >> 5] = fp;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T mv = (T)0, ma = (T)0;
        unsigned long long tp = 0;
        for (int w = 0; w < kBlock / 32; ++w) {
            mv = fmax(mv, wv[w]);
            ma = fmax(ma, wa[w]);
            tp += wp[w];
        }
        if (tp) atomicAdd(&acc->n_pairs_fluid, tp);
        raise_max(&acc->vmax2, (double)mv);
        raise_max(&acc->amax2, (double)ma);
    }
}

// ---- neighbour images (tests) ----------------------------------------------

template <int D, typename T>
__global__ void __launch_bounds__(kBlock)
    k_nbr_img(DevParams P, int n, const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ cell_s,
              const uint32_t *__restrict__ start, const uint32_t *__restrict__ gmask, const uint8_t *__restrict__ ovf,
              const uint16_t *__restrict__ nnb, const uint32_t *__restrict__ id_s, const int64_t *__restrict__ offsets,
              uint32_t *counts, uint32_t *ids, uint8_t *img)
{
    constexpr int NC = Stencil<D>::NC;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t *out = ids ? ids + offsets[i] : nullptr;
    uint8_t *oc = img ? img + offsets[i] : nullptr;
    uint32_t cnt = 0;
    auto body = [&](uint32_t j, T, T, T, T, const ImageCell<T> &ic) {
        if (j == (uint32_t)i && ic.code == 0) return;
        if (out) out[cnt] = id_s[j];
        if (oc) oc[cnt] = (uint8_t)ic.code;
        ++cnt;
    };
    const uint32_t clin = cell_s[i];
    const CellXYZ cc = decode_cell(P, clin);
    if (!ovf[i]) {
        const uint32_t *mbase = gmask + (size_t)blockIdx.x * NC * kBlock + threadIdx.x;
        walk_images<D, T>(P, pos[i], cc, clin, pos, start, [&](int idx) { return mbase[idx * kBlock]; },
                          (int)nnb[i], body);
    } else {
        scan_images<D, T>(P, pos[i], cc, clin, pos, start, body);
    }
    if (counts) counts[i] = cnt;
    if (!out) return;
    // ascending (id, code); lists hold ~10-80 entries
    for (uint32_t a = 1; a < cnt; ++a) {
        const uint32_t v = out[a];
        const uint8_t cv = oc ? oc[a] : 0;
        uint32_t b = a;
        while (b > 0 && (out[b - 1] > v || (out[b - 1] == v && oc && oc[b - 1] > cv))) {
            out[b] = out[b - 1];
            if (oc) oc[b] = oc[b - 1];
            --b;
        }
        out[b] = v;
        if (oc) oc[b] = cv;
    }
}

// ---- sampling operator (Section 6) -----------------------------------------
// S_i = alpha_D sum_j q_j w(|x_ij|/h), q_j = A_j m_j / rho_j (stored in
// pos[j].w by k_sample_prep), w(q) = (1 - q/2)^4 (2q + 1), self included.

template <typename T>
__global__ void __launch_bounds__(kBlock)
    k_sample_prep(int n, vec4_t<T> *pos, const T *__restrict__ A, const T *__restrict__ m, const T *__restrict__ rho)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pos[i].w = A[i] * m[i] / rho[i];
}

// G lanes per particle (G a power of two <= 32): lane g of a particle's group
// takes the stencil cells g, g + G, ...; the group's partial sums meet by
// warp shuffles in a fixed order.  G = 1 for large inputs (one lane per
// particle, enough warps to hide latency); small inputs take G > 1, since
// one lane walking all ~290 candidates is a serial chain of cache hits that
// too few warps cannot hide.  The candidate loop is fused with the kernel
// sum: the body is short, and unrolled candidates keep several loads in
// flight per lane.
template <int D, typename T, int G>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 8 : 4)
    k_sample(DevParams P, int n, const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ cell_s,
             const uint32_t *__restrict__ start, T *S)
{
    constexpr int NC = Stencil<D>::NC;
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = (int)(t / G);
    const int g = (int)(t % G);
    T sum = (T)0;
    if (i < n) {
        const vec4_t<T> pi = pos[i];
        const uint32_t clin = cell_s[i];
        const CellXYZ cc = decode_cell(P, clin);
        const bool inner = interior_cell<D>(P, cc);
        const T cs = cell_edge<T>(P), R2 = radius2<T>(P);
        const T R2cull = R2 * (T)1.0001;
        const T hih = (T)P.half_inv_h;
        const Gaps<D, T> gap(pi, cs);
#pragma unroll 1
        for (int idx = g; idx < NC; idx += G) {
            int dx, dy, dz;
            stencil_offsets<D>(idx, dx, dy, dz);
            if (sizeof(T) == 4 && gap(dx, dy, dz) > R2cull) continue;
            ImageCell<T> ic;
            if (!image_cell_at<D, T>(P, cc, clin, inner, idx, dx, dy, dz, ic)) continue;
            const ImgFrame<D, T> fr(pi, ic);
            const uint32_t a = start[ic.cell];
            uint32_t b = start[ic.cell + 1];
            if (!SPH_IN_BOUNDS(P, a <= b && b <= P.chk_cap)) b = a;
#pragma unroll 4
            for (uint32_t j = a; j < b; ++j) {
                const vec4_t<T> pj = pos[j];
                T rx, ry, rz;
                const T d2 = img_geometry<D, T>(fr, pj, rx, ry, rz);
                if (d2 < R2) {
                    const T u = Ar<T>::dist_ftz(d2) * hih;
                    const T w = (T)1 - u;
                    const T w2 = w * w;
                    sum += pj.w * (w2 * w2 * ((T)4 * u + (T)1));
                }
            }
        }
    }
    if (G > 1) {
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    }
    if (i < n && g == 0) S[i] = (T)P.alphaD * sum;
}

// Lanes per particle for n particles: enough threads to fill the GPU at about
// half occupancy (152 SMs x 1024), at most 32.
inline int sample_group(int n)
{
    const long long want = 152LL * 1024;
    int G = 1;
    while (G < 32 && (long long)n * G < want) G <<= 1;
    return G;
}

inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

}  // namespace

// ---- launchers ----------------------------------------------------------------

#define SPH_DISPATCH(P, f32, CALL)                          \
    do {                                                    \
        if ((P).dim == 2) {                                 \
            if (f32) { constexpr int D = 2; using T = float; CALL; }  \
            else { constexpr int D = 2; using T = double; CALL; }     \
        } else {                                            \
            if (f32) { constexpr int D = 3; using T = float; CALL; }  \
            else { constexpr int D = 3; using T = double; CALL; }     \
        }                                                   \
    } while (0)

cudaError_t launch_cont(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                        void *rho1, void *p1, Accum *acc, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    SPH_DISPATCH(P, f32, (k_cont<D, T><<<blocks_for(n, kBlock), kBlock, 0, st>>>(
                              P, n, static_cast<const vec4_t<T> *>(sb.pos), sb.cell_s, cb.cell_start,
                              static_cast<const vec4_t<T> *>(sb.vel), static_cast<T *>(sb.phat),
                              static_cast<T *>(rho1), static_cast<T *>(p1), acc, sb.mask, sb.ovf, sb.nnb)));
    return cudaGetLastError();
}

cudaError_t launch_mom(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                       const sph_state &s, const void *rho1, void *const *a_out, Accum *acc, uint32_t *status,
                       cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (a_out) {
        SPH_DISPATCH(P, f32, (k_mom<D, T, false><<<blocks_for(n, kBlock), kBlock, 0, st>>>(
                                  P, n, static_cast<const vec4_t<T> *>(sb.pos),
                                  static_cast<const vec4_t<T> *>(sb.vel), static_cast<const T *>(sb.phat),
                                  static_cast<const T *>(rho1), sb.cell_s, cb.cell_start, sb.mask, sb.ovf, sb, s,
                                  static_cast<T *>(a_out[0]), static_cast<T *>(a_out[1]),
                                  D == 3 ? static_cast<T *>(a_out[2]) : nullptr, acc, status)));
    } else {
        SPH_DISPATCH(P, f32, (k_mom<D, T, true><<<blocks_for(n, kBlock), kBlock, 0, st>>>(
                                  P, n, static_cast<const vec4_t<T> *>(sb.pos),
                                  static_cast<const vec4_t<T> *>(sb.vel), static_cast<const T *>(sb.phat),
                                  static_cast<const T *>(rho1), sb.cell_s, cb.cell_start, sb.mask, sb.ovf, sb, s,
                                  nullptr, nullptr, nullptr, acc, status)));
    }
    return cudaGetLastError();
}

cudaError_t launch_nbr_img(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                           uint32_t *counts, const int64_t *offsets, uint32_t *ids, uint8_t *img, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    SPH_DISPATCH(P, f32, (k_nbr_img<D, T><<<blocks_for(n, kBlock), kBlock, 0, st>>>(
                              P, n, static_cast<const vec4_t<T> *>(sb.pos), sb.cell_s, cb.cell_start, sb.mask,
                              sb.ovf, sb.nnb, sb.id_s, offsets, counts, ids, img)));
    return cudaGetLastError();
}

cudaError_t launch_sample(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                          const void *A, const void *m, const void *rho, void *S, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int G = sample_group(n);
    const long long threads = (long long)n * G;
    const int nb = (int)((threads + kBlock - 1) / kBlock);
#define SPH_SAMPLE_G(GG)                                                                                     \
    SPH_DISPATCH(P, f32, (k_sample<D, T, GG><<<nb, kBlock, 0, st>>>(P, n, static_cast<const vec4_t<T> *>(sb.pos), \
                                                                 sb.cell_s, cb.cell_start, static_cast<T *>(S))))
    SPH_DISPATCH(P, f32, (k_sample_prep<T><<<blocks_for(n, kBlock), kBlock, 0, st>>>(
                              n, static_cast<vec4_t<T> *>(sb.pos), static_cast<const T *>(A),
                              static_cast<const T *>(m), static_cast<const T *>(rho))));
    switch (G) {
    case 1: SPH_SAMPLE_G(1); break;
    case 2: SPH_SAMPLE_G(2); break;
    case 4: SPH_SAMPLE_G(4); break;
    case 8: SPH_SAMPLE_G(8); break;
    case 16: SPH_SAMPLE_G(16); break;
    default: SPH_SAMPLE_G(32); break;
    }
#undef SPH_SAMPLE_G
    return cudaGetLastError();
}

#undef SPH_DISPATCH

}  // namespace sph
