// sph_dem.cu -- the DEM particle damper of Example 2 (Section 5.2): Hertzian
// contact with the damping and Coulomb friction of Eq. DEM_force and the
// effective quantities of Eq. effective_quantities, the tank walls as the
// symmetric faces of the domain (their images, sph_images.cuh), and the tank
// oscillator of Eq. tank_ode driven by the wall force of Eq. boundary_force.
//
// One step: the cell build, then
//   k_dem_force     one lane per sphere walks the image stencil, tests the
//                   candidates within 2h (h the largest radius) and applies
//                   the contact law to every overlap; the forces from mirror
//                   images (the walls) are reduced per block in double, in a
//                   fixed order, into one partial per block;
//   k_dem_tank      one block sums the partials in a fixed order (so the
//                   step is deterministic), computes Zddot and advances the
//                   tank (symplectic Euler);
//   k_dem_integrate a = F/m + g - Zddot e_z (the tank's frame), v += dt a,
//                   r += dt v, periodic shift, state written in canonical
//                   order with the radius and mass that moved with it.
// Contacts are few (a sphere touches ~6-12 others among ~30 candidates), so
// the contact body sits inside the candidate loop.  The radius is carried in
// the w component of the sorted position, the mass in that of the sorted
// velocity.
#include <cuda_runtime.h>

#include "sph_images.cuh"
#include "sph_internal.cuh"
#include "sph_nbr.cuh"
#include "sph_phases.cuh"

namespace sph {
namespace {

template <int D, typename T>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 8 : 4)
    k_dem_force(DevParams P, int n, const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ cell_s,
                const uint32_t *__restrict__ start, const vec4_t<T> *__restrict__ vel, vec4_t<T> *F, double *fbp,
                Accum *acc)
{
    constexpr int NC = Stencil<D>::NC;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long contacts = 0;
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
#pragma unroll 1
        for (int idx = 0; idx < NC; ++idx) {
            int dx, dy, dz;
            stencil_offsets<D>(idx, dx, dy, dz);
            if (sizeof(T) == 4 && gap(dx, dy, dz) > R2cull) continue;
            ImageCell<T> ic;
            if (!image_cell_at<D, T>(P, cc, clin, inner, idx, dx, dy, dz, ic)) continue;
            const ImgFrame<D, T> fr(pi, ic);
            const bool wall = ic.s[0] < (T)0 || ic.s[1] < (T)0 || ic.s[2] < (T)0;
            const uint32_t a = start[ic.cell];
            uint32_t b = start[ic.cell + 1];
            if (!SPH_IN_BOUNDS(P, a <= b && b <= P.chk_cap)) b = a;
#pragma unroll 2
            for (uint32_t j = a; j < b; ++j) {
                const vec4_t<T> pj = pos[j];
                T x[3];
                const T d2 = img_geometry<D, T>(fr, pj, x[0], x[1], x[2]);
                if (!(d2 < R2)) continue;
                const T d = Ar<T>::dist(d2);
                const T delta = (Ri + pj.w) - d;
                if (!(delta > (T)0) || !(d > (T)0)) continue;
                // frame space: x' = s x_ij, w = s (v_i - v_j^t) = s v_i - v_j
                const vec4_t<T> vj = vel[j];
                const T inv_d = (T)1 / d;
                const T w[3] = {ic.s[0] * vi.x - vj.x, ic.s[1] * vi.y - vj.y, D == 3 ? ic.s[2] * vi.z - vj.z : (T)0};
                T vn = w[0] * x[0] + w[1] * x[1];
                if (D == 3) vn += w[2] * x[2];
                vn *= inv_d;  // v_ij . n
                const T Rp = Ar<T>::div(Ri * pj.w, Ri + pj.w);
                const T mp = Ar<T>::div(mi * vj.w, mi + vj.w);
                const T kh = (T)(4.0 / 3.0) * sqrt(Rp) * Ep;
                const T ch = sqrt(mp * kh) * (T)0.125;
                const T sd = sqrt(delta);
                const T fn = kh * delta * sd - ch * sqrt(sd) * vn;
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
                const T ft = vt2 > (T)1e-10 * vij2 ? Ar<T>::div(cf * fabs(fn), sqrt(vt2)) : (T)0;
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    const T fk = ic.s[k] * (fn * x[k] * inv_d + ft * vt[k]);
                    f[k] += fk;
                    if (wall) wb[k] += (double)fk;
                }
                ++contacts;
            }
        }
        vec4_t<T> out;
        out.x = f[0];
        out.y = f[1];
        out.z = f[2];
        out.w = (T)0;
        F[i] = out;
    }
    // contacts and the wall-force partial of the block (fixed order)
    __shared__ unsigned long long wc[kBlock / 32];
    __shared__ double ww[3][kBlock / 32];
    const unsigned long long c = warp_sum(contacts);
    double s3[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) s3[k] = warp_sum(wb[k]);
    if ((threadIdx.x & 31) == 0) {
        wc[threadIdx.x >> 5] = c;
        for (int k = 0; k < 3; ++k) ww[k][threadIdx.x >> 5] = s3[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        double b3[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < kBlock / 32; ++q) {
            t += wc[q];
            for (int k = 0; k < 3; ++k) b3[k] += ww[k][q];
        }
        if (t) atomicAdd(&acc->n_pairs, t);
        for (int k = 0; k < 3; ++k) fbp[(size_t)blockIdx.x * 3 + k] = b3[k];
    }
}

constexpr int kTankThreads = 1024;

__global__ void __launch_bounds__(kTankThreads)
    k_dem_tank(DevParams P, int nblocks, const double *__restrict__ fbp, TankDev *tank, int advance)
{
    __shared__ double red[3][kTankThreads];
    double s[3] = {0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += kTankThreads)
        for (int k = 0; k < 3; ++k) s[k] += fbp[(size_t)b * 3 + k];
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int h = kTankThreads / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int ax = P.dim - 1;
        double Fb[3] = {red[0][0], red[1][0], red[2][0]};
        const double Zdd = P.tankM > 0.0 ? (-P.tankS * tank->Z - Fb[ax]) / P.tankM : 0.0;
        tank->Zddot = Zdd;
        for (int k = 0; k < 3; ++k) tank->Fb[k] = Fb[k];
        if (advance) {
            tank->Zdot = tank->Zdot + P.dt * Zdd;
            tank->Z = tank->Z + P.dt * tank->Zdot;
        }
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
    const double v2max = (double)warp_max(v2);
    const double a2max = (double)warp_max(a2m);
    __shared__ double wv[kBlock / 32], wa[kBlock / 32];
    if ((threadIdx.x & 31) == 0) {
        wv[threadIdx.x >> 5] = v2max;
        wa[threadIdx.x >> 5] = a2max;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double mv = 0.0, ma = 0.0;
        for (int w = 0; w < kBlock / 32; ++w) {
            mv = fmax(mv, wv[w]);
            ma = fmax(ma, wa[w]);
        }
        raise_max(&acc->vmax2, mv);
        raise_max(&acc->amax2, ma);
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
    SPH_DISPATCH(P, f32, (k_dem_force<D, T><<<blocks_for(n, kBlock), kBlock, 0, st>>>(
                              P, n, static_cast<const vec4_t<T> *>(sb.pos), sb.cell_s, cb.cell_start,
                              static_cast<const vec4_t<T> *>(sb.vel), static_cast<vec4_t<T> *>(F), fbp, acc)));
    return cudaGetLastError();
}

cudaError_t launch_dem_tank(const DevParams &P, int n, const double *fbp, TankDev *tank, int advance,
                            cudaStream_t st)
{
    k_dem_tank<<<1, kTankThreads, 0, st>>>(P, n > 0 ? blocks_for(n, kBlock) : 0, fbp, tank, advance);
    return cudaGetLastError();
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
