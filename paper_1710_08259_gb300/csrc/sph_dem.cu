// sph_dem.cu -- the DEM particle damper of Example 2 (Section 5.2): Hertzian
// contact with the damping and Coulomb friction of Eq. DEM_force and the
// effective quantities of Eq. effective_quantities, the tank walls as the
// symmetric faces of the domain (their images, sph_images.cuh), and the tank
// oscillator of Eq. tank_ode driven by the wall force of Eq. boundary_force.
//
// One step: the cell build, then
//   k_dem_force     one lane per sphere walks the image stencil (an interior
//                   cell's stencil as 3^(D-1) runs of consecutive cells),
//                   tests the candidates within 2h (h the largest radius),
//                   queues the overlaps and applies the contact law to them;
//                   the forces from mirror images (the walls) are reduced
//                   per warp in double, in a fixed order, into one partial
//                   per warp;
//   k_dem_tank      one block sums the partials in a fixed order (so the
//                   step is deterministic), computes Zddot and advances the
//                   tank (symplectic Euler);
//   k_dem_integrate a = F/m + g - Zddot e_z (the tank's frame), v += dt a,
//                   r += dt v, periodic shift, state written in canonical
//                   order with the radius and mass that moved with it.
// The radius is carried in the w component of the sorted position, the mass
// in that of the sorted velocity.
#include <cuda_runtime.h>

#include "sph_images.cuh"
#include "sph_internal.cuh"
#include "sph_nbr.cuh"
#include "sph_phases.cuh"

namespace sph {
namespace {

// contacts queued per lane before the contact law runs over them
constexpr int kQueue = 16;

template <int D, typename T>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 8 : 4)
    k_dem_force(DevParams P, int n, const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ cell_s,
                const uint32_t *__restrict__ start, const vec4_t<T> *__restrict__ vel, vec4_t<T> *F, double *fbp,
                Accum *acc)
{
    constexpr int NC = Stencil<D>::NC;
    __shared__ uint32_t qj[kQueue][kBlock];
    __shared__ uint8_t qidx[kQueue][kBlock];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long contacts = 0;
    // a sphere's wall force in the working precision (it touches at most a
    // few wall images), widened once for the block sum in double
    T wbt[3] = {(T)0, (T)0, (T)0};
    double wb[3] = {0.0, 0.0, 0.0};
    if (i < n) {
        const vec4_t<T> pi = pos[i];
        const vec4_t<T> vi = vel[i];
        const T Ri = pi.w, mi = vi.w;
        const uint32_t clin = cell_s[i];
        const CellXYZ cc = decode_cell(P, clin);
        const bool inner = interior_cell<D>(P, cc);
        const T cs = cell_edge<T>(P), R2 = radius2<T>(P);
        const T R2cull = R2 * (T)1.0001;
        const Gaps<D, T> gap(pi, cs);
        const T Ep = (T)P.demEp, cf = (T)P.demCf;
        T f[3] = {(T)0, (T)0, (T)0};
        // the contact law with sphere j seen in the frame fr of its image
        // cell (x' = s x_ij; s = -1 on a mirrored axis, wall: any mirror)
        auto contact = [&](uint32_t j, ImgFrame<D, T> fr, T sx, T sy, T sz, bool wall) {
            const T sg[3] = {sx, sy, sz};
            const vec4_t<T> pj = pos[j];
            T x[3];
            const T d2 = img_geometry<D, T>(fr, pj, x[0], x[1], x[2]);
            if (!(d2 < R2)) return;
            const T d = Ar<T>::dist_ftz(d2);
            const T delta = (Ri + pj.w) - d;
            if (!(delta > (T)0) || !(d > (T)0)) return;
            // frame space: x' = s x_ij, w = s (v_i - v_j^t) = s v_i - v_j
            const vec4_t<T> vj = vel[j];
            // FP32: reciprocal square roots (one MUFU op each) for 1/d,
            // sqrt(R'), sqrt(m' k), delta^(1/2) and delta^(1/4): the IEEE
            // square roots and division took most of the law's issue slots;
            // FP64 keeps the correctly rounded forms
            const bool f32 = sizeof(T) == 4;
            const T inv_d = f32 ? (T)rsqrtf((float)d2) : (T)1 / d;
            const T w[3] = {sg[0] * vi.x - vj.x, sg[1] * vi.y - vj.y, D == 3 ? sg[2] * vi.z - vj.z : (T)0};
            T vn = w[0] * x[0] + w[1] * x[1];
            if (D == 3) vn += w[2] * x[2];
            vn *= inv_d;  // v_ij . n
            const T Rp = Ar<T>::div_ftz(Ri * pj.w, Ri + pj.w);
            const T mp = Ar<T>::div_ftz(mi * vj.w, mi + vj.w);
            const T kh = (T)(4.0 / 3.0) * (f32 ? Rp * (T)Ar<float>::rsqrt_ftz((float)Rp) : sqrt(Rp)) * Ep;
            const T mk = mp * kh;
            const T ch = (f32 ? mk * (T)Ar<float>::rsqrt_ftz((float)mk) : sqrt(mk)) * (T)0.125;
            const T sd = f32 ? delta * (T)Ar<float>::rsqrt_ftz((float)delta) : sqrt(delta);  // delta^(1/2)
            const T qd = f32 ? sd * (T)Ar<float>::rsqrt_ftz((float)sd) : sqrt(sd);            // delta^(1/4)
            const T fn = kh * delta * sd - ch * qd * vn;
            T vt[3], vt2 = (T)0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                vt[k] = k < D ? -w[k] + vn * x[k] * inv_d : (T)0;
                vt2 += vt[k] * vt[k];
            }
            // no sliding (|v_t| <= 1e-5 |v_ij|): no direction, no friction;
            // rounding would otherwise turn a head-on impact (or a sphere
            // against its own wall image) into a full Coulomb force
            const T vij2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
            const T ft = vt2 > (T)1e-10 * vij2
                             ? (f32 ? cf * fabs(fn) * (T)rsqrtf((float)vt2) : Ar<T>::div(cf * fabs(fn), sqrt(vt2)))
                             : (T)0;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const T fk = sg[k] * (fn * x[k] * inv_d + ft * vt[k]);
                f[k] += fk;
                if (wall) wbt[k] += fk;
            }
            ++contacts;
        };
        // Contacts are queued (sphere, stencil index) in shared memory by a
        // cheap test and the law runs over the queue: a lane then evaluates
        // the law only for its own contacts (~6 of ~30 candidates) instead
        // of idling through every other lane's.  The queue is worked off in
        // order whenever it fills and at the end, so the contacts add up in
        // candidate order, as an inline evaluation would.
        int nq = 0;
        auto drain = [&]() {
            for (int q = 0; q < nq; ++q) {
                const uint32_t j = qj[q][threadIdx.x];
                const int idx = qidx[q][threadIdx.x];
                int dx, dy, dz;
                stencil_offsets<D>(idx, dx, dy, dz);
                ImageCell<T> ic;
                image_cell_at<D, T>(P, cc, clin, inner, idx, dx, dy, dz, ic);
                const bool wall = ic.s[0] < (T)0 || ic.s[1] < (T)0 || ic.s[2] < (T)0;
                contact(j, ImgFrame<D, T>(pi, ic), ic.s[0], ic.s[1], ic.s[2], wall);
            }
            nq = 0;
        };
        auto test = [&](uint32_t j, const ImgFrame<D, T> &fr, int idx) {
            const vec4_t<T> pj = pos[j];
            T x[3];
            const T d2 = img_geometry<D, T>(fr, pj, x[0], x[1], x[2]);
            if (!(d2 < R2)) return;
            const T d = Ar<T>::dist_ftz(d2);
            const T delta = (Ri + pj.w) - d;
            if (!(delta > (T)0) || !(d > (T)0)) return;
            qj[nq][threadIdx.x] = j;
            qidx[nq][threadIdx.x] = (uint8_t)idx;
            if (++nq == kQueue) drain();
        };
        if (inner) {
            // no image anywhere in the stencil: the three cells of a stencil
            // row (dy, dz) are consecutive in the cell table, so their
            // spheres are one run of the sorted order, walked with the frame
            // of each sphere's cell; cells beyond the support are trimmed
            // from the run's ends exactly as they are skipped below, so the
            // candidates, their order and every result are the same
            constexpr int NR = D == 3 ? 9 : 3;
#pragma unroll 1
            for (int row = 0; row < NR; ++row) {
                const int dy = row % 3 - 1, dz = D == 3 ? row / 3 - 1 : 0;
                const bool use_l = !(sizeof(T) == 4 && gap(-1, dy, dz) > R2cull);
                const bool use_m = !(sizeof(T) == 4 && gap(0, dy, dz) > R2cull);
                const bool use_r = !(sizeof(T) == 4 && gap(1, dy, dz) > R2cull);
                if (!use_m) continue;  // (the middle cell is the nearest of the row)
                ImageCell<T> icl, icm, icr;
                image_cell_at<D, T>(P, cc, clin, true, 3 * row, -1, dy, dz, icl);
                image_cell_at<D, T>(P, cc, clin, true, 3 * row + 1, 0, dy, dz, icm);
                image_cell_at<D, T>(P, cc, clin, true, 3 * row + 2, 1, dy, dz, icr);
                const uint32_t s0 = start[icm.cell - 1], s1 = start[icm.cell], s2 = start[icm.cell + 1],
                               s3 = start[icm.cell + 2];
                if (!SPH_IN_BOUNDS(P, s0 <= s1 && s1 <= s2 && s2 <= s3 && s3 <= P.chk_cap)) continue;
                const ImgFrame<D, T> fl(pi, icl), fm(pi, icm), fr(pi, icr);
                const uint32_t jlo = use_l ? s0 : s1, jhi = use_r ? s3 : s2;
#pragma unroll 2
                for (uint32_t j = jlo; j < jhi; ++j) {
                    ImgFrame<D, T> f = fm;
                    f.x = j < s1 ? fl.x : (j < s2 ? fm.x : fr.x);
                    test(j, f, 3 * row + (j < s1 ? 0 : (j < s2 ? 1 : 2)));
                }
            }
        } else {
#pragma unroll 1
            for (int idx = 0; idx < NC; ++idx) {
                int dx, dy, dz;
                stencil_offsets<D>(idx, dx, dy, dz);
                if (sizeof(T) == 4 && gap(dx, dy, dz) > R2cull) continue;
                ImageCell<T> ic;
                if (!image_cell_at<D, T>(P, cc, clin, inner, idx, dx, dy, dz, ic)) continue;
                const ImgFrame<D, T> fr(pi, ic);
                const uint32_t a = start[ic.cell];
                uint32_t b = start[ic.cell + 1];
                if (!SPH_IN_BOUNDS(P, a <= b && b <= P.chk_cap)) b = a;
#pragma unroll 2
                for (uint32_t j = a; j < b; ++j) test(j, fr, idx);
            }
        }
        drain();
        vec4_t<T> out;
        out.x = f[0];
        out.y = f[1];
        out.z = f[2];
        out.w = (T)0;
        F[i] = out;
    }
    // contacts and the wall-force partial of the warp (fixed order); no
    // block barrier, so a warp that is done leaves at once
    const unsigned long long c = warp_sum(contacts);
    double s3[3] = {0.0, 0.0, 0.0};
    // (double arithmetic is scarce on this GPU: only the warps that touched
    // a wall reduce; the others' partial is exactly zero)
#pragma unroll
    for (int k = 0; k < 3; ++k) wb[k] = (double)wbt[k];
    if (__any_sync(0xffffffffu, wb[0] != 0.0 || wb[1] != 0.0 || wb[2] != 0.0)) {
#pragma unroll
        for (int k = 0; k < 3; ++k) s3[k] = warp_sum(wb[k]);
    }
    if ((threadIdx.x & 31) == 0) {
        if (c) atomicAdd(&acc->n_pairs, c);
        const size_t w = (size_t)blockIdx.x * (kBlock / 32) + (threadIdx.x >> 5);
        for (int k = 0; k < 3; ++k) fbp[w * 3 + k] = s3[k];
    }
}

// The wall force: the warps' partials are summed by kWallBlocks blocks, each
// over its contiguous slice in a fixed order, and the last block to finish
// adds the blocks' sums in block order and advances the tank, so the sum is
// deterministic and the double additions are spread over many SMs (double
// arithmetic is scarce on this GPU).  The blocks' sums sit at the front of
// the partials buffer.
constexpr int kWallBlocks = 64;
constexpr int kWallThreads = 256;

// Sum of red[0..m) for each component in a fixed tree order (m a power of
// two, every thread of the block calls it).
__device__ __forceinline__ void tree3(double (*red)[kWallThreads], int m)
{
    for (int h = m / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h) {
            red[0][threadIdx.x] += red[0][threadIdx.x + h];
            red[1][threadIdx.x] += red[1][threadIdx.x + h];
            red[2][threadIdx.x] += red[2][threadIdx.x + h];
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kWallThreads)
    k_dem_tank(DevParams P, int nparts, const double *__restrict__ wp, double *bsum, TankDev *tank, int advance)
{
    static_assert(kWallBlocks <= kWallThreads, "one thread per block sum");
    __shared__ double red[3][kWallThreads];
    __shared__ int last;
    const int per = (nparts + kWallBlocks - 1) / kWallBlocks;
    const int lo = blockIdx.x * per, hi = min(nparts, lo + per);
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int q = lo + threadIdx.x; q < hi; q += kWallThreads) {
        s0 += wp[(size_t)q * 3];
        s1 += wp[(size_t)q * 3 + 1];
        s2 += wp[(size_t)q * 3 + 2];
    }
    red[0][threadIdx.x] = s0;
    red[1][threadIdx.x] = s1;
    red[2][threadIdx.x] = s2;
    __syncthreads();
    tree3(red, kWallThreads);
    if (threadIdx.x == 0) {
        bsum[blockIdx.x * 3] = red[0][0];
        bsum[blockIdx.x * 3 + 1] = red[1][0];
        bsum[blockIdx.x * 3 + 2] = red[2][0];
        __threadfence();
        last = atomicAdd(&tank->done, 1u) == kWallBlocks - 1;
    }
    __syncthreads();
    if (!last) return;
    // the last block: the blocks' sums, again in a fixed tree order
    __threadfence();
    const int t = threadIdx.x;
    red[0][t] = t < kWallBlocks ? __ldcg(bsum + t * 3) : 0.0;
    red[1][t] = t < kWallBlocks ? __ldcg(bsum + t * 3 + 1) : 0.0;
    red[2][t] = t < kWallBlocks ? __ldcg(bsum + t * 3 + 2) : 0.0;
    __syncthreads();
    tree3(red, kWallBlocks);
    if (t != 0) return;
    tank->done = 0;
    const double Fz = P.dim == 3 ? red[2][0] : red[1][0];
    const double Zdd = P.tankM > 0.0 ? (-P.tankS * tank->Z - Fz) / P.tankM : 0.0;
    tank->Zddot = Zdd;
    tank->Fb[0] = red[0][0];
    tank->Fb[1] = red[1][0];
    tank->Fb[2] = red[2][0];
    if (advance) {
        tank->Zdot = tank->Zdot + P.dt * Zdd;
        tank->Z = tank->Z + P.dt * tank->Zdot;
    }
}

template <int D, typename T, bool INTEGRATE>
__global__ void __launch_bounds__(kBlock)
    k_dem_integrate(DevParams P, int n, SortedBufs sb, const vec4_t<T> *__restrict__ F,
                    const TankDev *__restrict__ tank, sph_state s, T *a0, T *a1, T *a2, Accum *acc,
                    uint32_t *status)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    // |v|^2, |a|^2 for the diagnostics in the working precision: only the
    // block maximum is widened (the FP64 pipe of this GPU is narrow)
    T v2 = (T)0, a2m = (T)0;
    bool bad = false;
    if (i < n) {
        const uint8_t kd = sb.kind_s[i];
        const vec4_t<T> vi = static_cast<const vec4_t<T> *>(sb.vel)[i];
        const vec4_t<T> fi = F[i];
        const T m = vi.w;
        const T Zdd = (T)tank->Zddot;
        const T fa[3] = {fi.x, fi.y, fi.z};
        const T va[3] = {vi.x, vi.y, vi.z};
        T a[3] = {(T)0, (T)0, (T)0};
        if (kd == SPH_FLUID) {
#pragma unroll
            for (int k = 0; k < D; ++k) a[k] = Ar<T>::div(fa[k], m) + (T)P.g[k] - (k == D - 1 ? Zdd : (T)0);
        }
        if (INTEGRATE) {
            T nv[3] = {va[0], va[1], va[2]};
#pragma unroll
            for (int k = 0; k < D; ++k) {
                double x = sb.rs[k][i];
                if (kd == SPH_FLUID) {
                    nv[k] = va[k] + (T)P.dt * a[k];
                    x = x + P.dt * (double)nv[k];
                    if (P.bc[k] == SPH_BC_PERIODIC) {
                        if (x < P.dom_min[k]) x = x + P.per[k];
                        else if (x >= P.hi[k]) x = x - P.per[k];
                    }
                }
                s.r[k][i] = x;
                static_cast<T *>(s.v[k])[i] = nv[k];
            }
            static_cast<T *>(s.radius)[i] = static_cast<const vec4_t<T> *>(sb.pos)[i].w;
            static_cast<T *>(s.mass)[i] = m;
            s.id[i] = sb.id_s[i];
            s.kind[i] = kd;
            if (kd == SPH_FLUID) {
                v2 = nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2];
                a2m = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
                bad = !isfinite(v2) || !isfinite(a2m);
            }
        } else {
            a0[i] = a[0];
            a1[i] = a[1];
            if (D == 3) a2[i] = a[2];
            if (kd == SPH_FLUID) {
                a2m = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
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
    __shared__ T wv[kBlock / 32], wa[kBlock / 32];
    if ((threadIdx.x & 31) == 0) {
        wv[threadIdx.x >> 5] = v2max;
        wa[threadIdx.x >> 5] = a2max;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        T mv = (T)0, ma = (T)0;
        for (int w = 0; w < kBlock / 32; ++w) {
            mv = fmax(mv, wv[w]);
            ma = fmax(ma, wa[w]);
        }
        raise_max(&acc->vmax2, (double)mv);
        raise_max(&acc->amax2, (double)ma);
    }
}

inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

}  // namespace

#define SPH_DISPATCH(P, f32, CALL)                                   \
    do {                                                             \
        if ((P).dim == 2) {                                          \
            if (f32) { constexpr int D = 2; using T = float; CALL; }  \
            else { constexpr int D = 2; using T = double; CALL; }     \
        } else {                                                     \
            if (f32) { constexpr int D = 3; using T = float; CALL; }  \
            else { constexpr int D = 3; using T = double; CALL; }     \
        }                                                            \
    } while (0)

cudaError_t launch_dem_force(const DevParams &P, bool f32, int n, const CellBufs &cb, const SortedBufs &sb,
                             void *F, double *fbp, Accum *acc, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    // (the warps' partials follow the wall blocks' sums)
    SPH_DISPATCH(P, f32, (k_dem_force<D, T><<<blocks_for(n, kBlock), kBlock, 0, st>>>(
                              P, n, static_cast<const vec4_t<T> *>(sb.pos), sb.cell_s, cb.cell_start,
                              static_cast<const vec4_t<T> *>(sb.vel), static_cast<vec4_t<T> *>(F),
                              fbp + 3 * kWallBlocks, acc)));
    return cudaGetLastError();
}

cudaError_t launch_dem_tank(const DevParams &P, int n, double *fbp, TankDev *tank, int advance, cudaStream_t st)
{
    k_dem_tank<<<kWallBlocks, kWallThreads, 0, st>>>(P, n > 0 ? blocks_for(n, kBlock) * (kBlock / 32) : 0,
                                                     fbp + 3 * kWallBlocks, fbp, tank, advance);
    return cudaGetLastError();
}

size_t dem_partials_bytes(int n)
{
    return (size_t)(3 * kWallBlocks + ((n + kBlock - 1) / kBlock + 1) * (kBlock / 32) * 3) * sizeof(double);
}

cudaError_t launch_dem_integrate(const DevParams &P, bool f32, int n, const SortedBufs &sb, const void *F,
                                 const TankDev *tank, const sph_state &s, void *const *a_out, Accum *acc,
                                 uint32_t *status, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (a_out) {
        SPH_DISPATCH(P, f32, (k_dem_integrate<D, T, false><<<blocks_for(n, kBlock), kBlock, 0, st>>>(
                                  P, n, sb, static_cast<const vec4_t<T> *>(F), tank, s, static_cast<T *>(a_out[0]),
                                  static_cast<T *>(a_out[1]), D == 3 ? static_cast<T *>(a_out[2]) : nullptr, acc,
                                  status)));
    } else {
        SPH_DISPATCH(P, f32, (k_dem_integrate<D, T, true><<<blocks_for(n, kBlock), kBlock, 0, st>>>(
                                  P, n, sb, static_cast<const vec4_t<T> *>(F), tank, s, nullptr, nullptr, nullptr,
                                  acc, status)));
    }
    return cudaGetLastError();
}

#undef SPH_DISPATCH

}  // namespace sph
