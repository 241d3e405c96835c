// sph_images.cuh -- the stencil of a particle's cell with the faces of the
// domain (Section 3.2.1): a stencil cell outside the grid is mapped to the
// cell that holds its images (periodic: the cell on the other side; symmetric:
// the particle's own cell, reflected; cut-off: none), with the frame shift and
// sign that give the relative position of each image exactly as the CPU
// oracle defines it.  Shared by the Example 1a / sampling kernels
// (sph_model.cu) and the DEM kernels (sph_dem.cu).
//
// The reflection costs nothing per candidate: with the sign s = -1 of a
// mirrored axis, x_ij = (p_i - S) + p_j = s ((s (p_i - S)) - p_j) exactly
// (negation is exact in round-to-nearest), so the candidate loop runs the
// plain geometry on the frame s (p_i - S) and d2 is unchanged; a hit takes
// its true x_ij = s x' and v_ij . r_ij = (s v_i - v_j) . x'.
#pragma once

#include <cuda_runtime.h>

#include "sph_internal.cuh"
#include "sph_nbr.cuh"

namespace sph {


// One stencil cell seen from a particle's cell.
template <typename T>
struct ImageCell {
    int cell;  // global index of the cell that holds the candidates
    T S[3];    // frame shift of i's coordinates
    T s[3];    // +1, or -1 on a mirrored axis
    int code;  // image code t_x + 3 t_y + 9 t_z (t: 0 itself, 1 lower face, 2 upper face)
};

template <int D, typename T>
__device__ __forceinline__ bool image_cell(const DevParams &P, const CellXYZ &c, int dx, int dy, int dz,
                                           ImageCell<T> &o)
{
    constexpr bool F32 = sizeof(T) == 4;
    const int cc[3] = {c.x, c.y, c.z};
    const int dd[3] = {dx, dy, dz};
    int real[3] = {0, 0, 0};
    int code = 0, mul = 1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        o.S[k] = (T)0;
        o.s[k] = (T)1;
        if (k >= D) continue;
        const int u = cc[k] + dd[k];
        const int nc = P.nc[k];
        T S = F32 ? (T)((float)dd[k] * P.csf) : (T)0;
        int t = 0;
        if (u >= 0 && u < nc) {
            real[k] = u;
        } else {
            const int b = P.bc[k];
            if (b == SPH_BC_CUTOFF) return false;
            t = u < 0 ? 1 : 2;
            if (b == SPH_BC_PERIODIC) {
                real[k] = u < 0 ? u + nc : u - nc;
                if (!F32) S = (T)(u < 0 ? -P.per[k] : P.per[k]);
            } else {
                real[k] = cc[k];
                o.s[k] = (T)-1;
                if (F32) S = u < 0 ? (T)0 : (T)(2.0f * P.csf);
                else S = (T)(2.0 * (u < 0 ? P.dom_min[k] : P.hi[k]));
            }
        }
        o.S[k] = S;
        code += t * mul;
        mul *= 3;
    }
    o.cell = (int)P.cell_off + real[0] + P.nc[0] * (real[1] + P.nc[1] * real[2]);
    o.code = code;
    return true;
}

// A cell at least one cell away from every face: its stencil needs no image
// mapping.
template <int D>
__device__ __forceinline__ bool interior_cell(const DevParams &P, const CellXYZ &c)
{
    bool in = c.x >= 1 && c.x <= P.nc[0] - 2 && c.y >= 1 && c.y <= P.nc[1] - 2;
    if (D == 3) in = in && c.z >= 1 && c.z <= P.nc[2] - 2;
    return in;
}

// image_cell with a fast path for interior cells: the stencil table of the
// context gives the cell index delta and the FP32 frame shift (float)d * cs,
// the same values image_cell computes for in-grid cells.  clin: the global
// index of the particle's cell; idx: the stencil index of (dx, dy, dz).
template <int D, typename T>
__device__ __forceinline__ bool image_cell_at(const DevParams &P, const CellXYZ &c, uint32_t clin, bool inner,
                                              int idx, int dx, int dy, int dz, ImageCell<T> &o)
{
    if (inner) {
        const StencilEntry e = P.stab[idx];
        o.cell = (int)clin + e.dcell;
        o.S[0] = sizeof(T) == 4 ? (T)e.sx : (T)0;
        o.S[1] = sizeof(T) == 4 ? (T)e.sy : (T)0;
        o.S[2] = sizeof(T) == 4 && D == 3 ? (T)e.sz : (T)0;
        o.s[0] = o.s[1] = o.s[2] = (T)1;
        o.code = 0;
        return true;
    }
    return image_cell<D, T>(P, c, dx, dy, dz, o);
}

// Stencil index -> offsets (the order of for_stencil: dz, dy, dx).
template <int D>
__device__ __forceinline__ void stencil_offsets(int idx, int &dx, int &dy, int &dz)
{
    dx = idx % 3 - 1;
    dy = (idx / 3) % 3 - 1;
    dz = D == 3 ? idx / 9 - 1 : 0;
}

// Frame of i for one image cell: s (p_i - S) per axis.
template <int D, typename T>
struct ImgFrame {
    T x, y, z;
    __device__ __forceinline__ ImgFrame(const vec4_t<T> &pi, const ImageCell<T> &ic)
    {
        x = ic.s[0] * Ar<T>::sub(pi.x, ic.S[0]);
        y = ic.s[1] * Ar<T>::sub(pi.y, ic.S[1]);
        z = D == 3 ? ic.s[2] * Ar<T>::sub(pi.z, ic.S[2]) : (T)0;
    }
};

// x' = frame - p_j and d2, exactly the oracle's predicate (x_ij = s x').
template <int D, typename T>
__device__ __forceinline__ T img_geometry(const ImgFrame<D, T> &f, const vec4_t<T> &pj, T &rx, T &ry, T &rz)
{
    rx = Ar<T>::sub(f.x, pj.x);
    ry = Ar<T>::sub(f.y, pj.y);
    T d2 = Ar<T>::mul(rx, rx);
    d2 = Ar<T>::fma(ry, ry, d2);
    rz = (T)0;
    if (D == 3) {
        rz = Ar<T>::sub(f.z, pj.z);
        d2 = Ar<T>::fma(rz, rz, d2);
    }
    return d2;
}

// Squared distance from i's offsets to the box of the (unwrapped) stencil
// cell (dx, dy, dz): F32 form only; a cell beyond the support holds no
// neighbour.  Images lie in the unwrapped cell's box, so the test holds for
// every face treatment.
template <int D, typename T>
struct Gaps {
    T lx, ux, ly, uy, lz, uz;
    __device__ __forceinline__ Gaps(const vec4_t<T> &pi, T cs)
    {
        lx = pi.x * pi.x;
        ux = (cs - pi.x) * (cs - pi.x);
        ly = pi.y * pi.y;
        uy = (cs - pi.y) * (cs - pi.y);
        lz = D == 3 ? pi.z * pi.z : (T)0;
        uz = D == 3 ? (cs - pi.z) * (cs - pi.z) : (T)0;
    }
    __device__ __forceinline__ T operator()(int dx, int dy, int dz) const
    {
        return (dx < 0 ? lx : (dx > 0 ? ux : (T)0)) + (dy < 0 ? ly : (dy > 0 ? uy : (T)0)) +
               (dz < 0 ? lz : (dz > 0 ? uz : (T)0));
    }
};

// Every candidate of every image cell: f(j, x', d2, image cell) on hits.
template <int D, typename T, typename F>
__device__ __forceinline__ void scan_images(const DevParams &P, const vec4_t<T> &pi, const CellXYZ &cc,
                                            uint32_t clin, const vec4_t<T> *__restrict__ pos,
                                            const uint32_t *__restrict__ start, F &&f)
{
    const bool inner = interior_cell<D>(P, cc);
    const T R2 = radius2<T>(P);
    constexpr int NC = Stencil<D>::NC;
#pragma unroll 1
    for (int idx = 0; idx < NC; ++idx) {
        int dx, dy, dz;
        stencil_offsets<D>(idx, dx, dy, dz);
        ImageCell<T> ic;
        if (!image_cell_at<D, T>(P, cc, clin, inner, idx, dx, dy, dz, ic)) continue;
        const ImgFrame<D, T> fr(pi, ic);
        const uint32_t a = start[ic.cell];
        uint32_t b = start[ic.cell + 1];
        if (!SPH_IN_BOUNDS(P, a <= b && b <= P.chk_cap)) b = a;
        for (uint32_t j = a; j < b; ++j) {
            T rx, ry, rz;
            const T d2 = img_geometry<D, T>(fr, pos[j], rx, ry, rz);
            if (d2 < R2) f(j, rx, ry, rz, d2, ic);
        }
    }
}

// Flattened walk over the hit masks (one iteration per neighbour image, self
// included), as walk_masks in sph_nbr.cuh but with the image cell of each
// stencil cell.  f(j, x', d2, image cell).
template <int D, typename T, typename M, typename F>
__device__ __forceinline__ void walk_images(const DevParams &P, const vec4_t<T> &pi, const CellXYZ &cc,
                                            uint32_t clin, const vec4_t<T> *__restrict__ pos,
                                            const uint32_t *__restrict__ start, M &&mask, int total, F &&f)
{
    const bool inner = interior_cell<D>(P, cc);
    constexpr int NC = Stencil<D>::NC;
    int idx = -1;
    uint32_t w = 0, a = 0;
    ImageCell<T> ic{0, {(T)0, (T)0, (T)0}, {(T)1, (T)1, (T)1}, 0};
    ImgFrame<D, T> fr(pi, ic);
    for (int n = 0; n < total; ++n) {
        if (w == 0) {
            do {
                ++idx;
                w = mask(idx);
            } while (w == 0 && idx < NC - 1);
            if (w == 0) break;  // inconsistent total: never walk past the stencil
            int dx, dy, dz;
            stencil_offsets<D>(idx, dx, dy, dz);
            if (!image_cell_at<D, T>(P, cc, clin, inner, idx, dx, dy, dz, ic)) break;  // never marked
            a = start[ic.cell];
            fr = ImgFrame<D, T>(pi, ic);
        }
        const uint32_t j = a + (uint32_t)(__ffs(w) - 1);
        w &= w - 1u;
        if (!SPH_IN_BOUNDS(P, j < P.chk_cap)) break;
        T rx, ry, rz;
        const T d2 = img_geometry<D, T>(fr, pos[j], rx, ry, rz);
        f(j, rx, ry, rz, d2, ic);
    }
}

// Candidate tests of one particle over its image cells: masks at
// mbase[idx * kBlock], returns the hit count (self included); over = a cell
// held more than 32 particles (no masks; the slow path rescans).
template <int D, typename T>
__device__ __forceinline__ int image_masks(const DevParams &P, const vec4_t<T> &pi, const CellXYZ &cc,
                                           uint32_t clin, const vec4_t<T> *__restrict__ pos,
                                           const uint32_t *__restrict__ start, uint32_t *mbase, bool &over)
{
    const bool inner = interior_cell<D>(P, cc);
    constexpr int NC = Stencil<D>::NC;
    const T cs = cell_edge<T>(P), R2 = radius2<T>(P);
    const T R2cull = R2 * (T)1.0001;
    const Gaps<D, T> gap(pi, cs);
    int total = 0;
    over = false;
#pragma unroll 1
    for (int idx = 0; idx < NC; ++idx) {
        int dx, dy, dz;
        stencil_offsets<D>(idx, dx, dy, dz);
        ImageCell<T> ic;
        uint32_t a = 0, b = 0;
        if (image_cell_at<D, T>(P, cc, clin, inner, idx, dx, dy, dz, ic)) {
            a = start[ic.cell];
            b = start[ic.cell + 1];
            if (!SPH_IN_BOUNDS(P, a <= b && b <= P.chk_cap)) b = a;
        }
        if (b - a > 32u) {
            over = true;
            b = a;
        }
        if (sizeof(T) == 4 && gap(dx, dy, dz) > R2cull) b = a;
        uint32_t wbits = 0;
        if (b > a) {
            const ImgFrame<D, T> fr(pi, ic);
            uint32_t bit = 1u;
#pragma unroll 4
            for (uint32_t j = a; j < b; ++j, bit <<= 1) {
                T rx, ry, rz;
                const T d2 = img_geometry<D, T>(fr, pos[j], rx, ry, rz);
                if (d2 < R2) wbits |= bit;
            }
        }
        mbase[idx * kBlock] = wbits;
        total += __popc(wbits);
    }
    return total;
}

// ---- the row stencil behind the image-walk interface ---------------------
// A domain whose faces are all cut-off has no images; with cells of edge cs
// in [h, 2h) its neighbours lie in the 5^D cells around a particle's own,
// walked as rows (sph_nbr.cuh).  These wrappers give that walk the
// interface of the image walks above, every neighbour seen as itself (image
// code 0, unit signs), for callers written against images (compiled
// interaction laws).

template <typename T>
__device__ __forceinline__ ImageCell<T> identity_image()
{
    return ImageCell<T>{0, {(T)0, (T)0, (T)0}, {(T)1, (T)1, (T)1}, 0};
}

// Candidate tests recorded as row masks at mbase[idx * kBlock]; returns the
// hit count (self included); over = a row held more than 32 particles.
template <int D, typename T>
__device__ __forceinline__ int row_image_masks(const DevParams &P, const vec4_t<T> &pi, uint32_t clin,
                                               const vec4_t<T> *__restrict__ pos,
                                               const uint32_t *__restrict__ start, uint32_t *mbase, bool &over)
{
    over = false;
    return row_candidates<D, T>(P, pi, clin, pos, start, mbase, kBlock, over, [](uint32_t, T, T, T, T) {},
                                [] {});
}

template <int D, typename T, typename M, typename F>
__device__ __forceinline__ void walk_row_images(const DevParams &P, const vec4_t<T> &pi, uint32_t clin,
                                                const vec4_t<T> *__restrict__ pos,
                                                const uint32_t *__restrict__ start, M &&mask, int total, F &&f)
{
    const ImageCell<T> ic = identity_image<T>();
    walk_rows<D, T>(P, pi, clin, pos, start, mask, total,
                    [&](uint32_t j, T x, T y, T z, T d2) { f(j, x, y, z, d2, ic); });
}

template <int D, typename T, typename F>
__device__ __forceinline__ void scan_row_images(const DevParams &P, const vec4_t<T> &pi, uint32_t clin,
                                                const vec4_t<T> *__restrict__ pos,
                                                const uint32_t *__restrict__ start, F &&f)
{
    const ImageCell<T> ic = identity_image<T>();
    for_neighbours_scan_rows<D, T>(P, pi, clin, pos, start,
                                   [&](uint32_t j, T x, T y, T z, T d2) { f(j, x, y, z, d2, ic); });
}

}  // namespace sph

