// sph_nbr.cuh -- device helpers of the pair loops: exact FP32/FP64 pair
// geometry (the neighbour predicate of the CPU oracle, bit for bit), the 3^D
// cell stencil, and neighbour iteration by candidate scan or by the hit masks
// the density pass records.
#pragma once

#include <cuda_runtime.h>

#include "sph_internal.cuh"

namespace sph {

template <typename T> struct Ar;
template <> struct Ar<float> {
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
    // |r| for the kernel value; d2 = 0 only for the self pair or coincident
    // particles, where the result must be 0 (not 0 * inf)
    static __device__ __forceinline__ float dist(float d2) { return d2 * rsqrtf(fmaxf(d2, 1e-30f)); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdividef(a, b); }
    // The flush-to-zero forms, which skip the handling of subnormal operands.
    // dist_ftz: the operand is clamped to >= 1e-30 and its reciprocal root is
    // <= 1e15, both normal, so the result is that of dist (3D density pass at
    // 256^3: 9 % fewer instructions, 5.90 -> 5.58 ms; sampling at 252^3
    // 5.11 -> 4.51 ms).  rsqrt_ftz: equal to
    // rsqrtf for a positive normal operand (the DEM law's R', m'k, delta and
    // delta^(1/2)).  div_ftz: equal to div while a, b and a / b are normal;
    // the viscosity quotients leave that range only when |a| < 2^-126, where
    // the term is below any other term's rounding.  (dist_ftz in the momentum
    // pass made it slower, 4.13 -> 4.32 ms at 256^3, so it keeps dist.)
    static __device__ __forceinline__ float dist_ftz(float d2)
    {
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fmaxf(d2, 1e-30f)));
        return d2 * r;
    }
    static __device__ __forceinline__ float rsqrt_ftz(float x)
    {
        float r;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    static __device__ __forceinline__ float div_ftz(float a, float b)
    {
        float r;
        asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
        return r;
    }
};
template <> struct Ar<double> {
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ double dist(double d2) { return sqrt(d2); }
    static __device__ __forceinline__ double div(double a, double b) { return a / b; }
    static __device__ __forceinline__ double dist_ftz(double d2) { return sqrt(d2); }
    static __device__ __forceinline__ double div_ftz(double a, double b) { return a / b; }
};

template <int D> struct Stencil { static constexpr int NC = D == 3 ? 27 : 9; };

struct CellXYZ {
    int x, y, z;
};

// Cell coordinates of a global cell index (c includes the case's cell_off).
__device__ __forceinline__ CellXYZ decode_cell(const DevParams &P, uint32_t c)
{
    c -= P.cell_off;
    CellXYZ r;
    r.x = (int)(c % (uint32_t)P.nc[0]);
    const uint32_t rest = c / (uint32_t)P.nc[0];
    r.y = (int)(rest % (uint32_t)P.nc[1]);
    r.z = (int)(rest / (uint32_t)P.nc[1]);
    return r;
}

// Visit the 3^D cells around (cx, cy, cz) in the fixed order (dz, dy, dx),
// calling f(idx, global cell index or -1 when outside the grid, dx, dy, dz).
template <int D, typename F>
__device__ __forceinline__ void for_stencil(const DevParams &P, const CellXYZ &c, F &&f)
{
    int idx = 0;
#pragma unroll 1
    for (int dz = (D == 3 ? -1 : 0); dz <= (D == 3 ? 1 : 0); ++dz) {
        const int z = c.z + dz;
        const bool zin = D == 2 || (z >= 0 && z < P.nc[2]);
#pragma unroll 1
        for (int dy = -1; dy <= 1; ++dy) {
            const int y = c.y + dy;
            const bool yin = zin && y >= 0 && y < P.nc[1];
            const int row = (int)P.cell_off + P.nc[0] * (y + P.nc[1] * (D == 3 ? z : 0));
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int x = c.x + dx;
                const bool in = yin && x >= 0 && x < P.nc[0];
                f(idx, in ? row + x : -1, dx, dy, dz);
                ++idx;
            }
        }
    }
}

// i's coordinates in the frame of the neighbour cell at offset (dx, dy, dz):
// F32: s = o_i - d * cs (the product is exact); F64: absolute, unchanged.
template <int D, typename T>
struct Frame {
    T x, y, z;
    __device__ __forceinline__ Frame(const vec4_t<T> &pi, T cs, int dx, int dy, int dz)
    {
        x = Ar<T>::sub(pi.x, (T)dx * cs);
        y = Ar<T>::sub(pi.y, (T)dy * cs);
        z = D == 3 ? Ar<T>::sub(pi.z, (T)dz * cs) : (T)0;
    }
};

// x_ij and d2 exactly as the neighbour predicate defines them.
template <int D, typename T>
__device__ __forceinline__ T geometry(const Frame<D, T> &s, const vec4_t<T> &pj, T &rx, T &ry, T &rz)
{
    rx = Ar<T>::sub(s.x, pj.x);
    ry = Ar<T>::sub(s.y, pj.y);
    T d2 = Ar<T>::mul(rx, rx);
    d2 = Ar<T>::fma(ry, ry, d2);
    rz = (T)0;
    if (D == 3) {
        rz = Ar<T>::sub(s.z, pj.z);
        d2 = Ar<T>::fma(rz, rz, d2);
    }
    return d2;
}

template <typename T> __device__ __forceinline__ T cell_edge(const DevParams &P)
{
    return sizeof(T) == 4 ? (T)P.csf : (T)0;
}
template <typename T> __device__ __forceinline__ T radius2(const DevParams &P)
{
    return sizeof(T) == 4 ? (T)P.R2f : (T)P.R2;
}

// Slow path: every candidate of the 3^D cells, f(j, x, y, z, d2) on hits.
template <int D, typename T, typename F>
__device__ __forceinline__ void for_neighbours_scan(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                                    const vec4_t<T> *__restrict__ pos,
                                                    const uint32_t *__restrict__ start, F &&f)
{
    const T cs = cell_edge<T>(P), R2 = radius2<T>(P);
    for_stencil<D>(P, decode_cell(P, c), [&](int, int cell, int dx, int dy, int dz) {
        if (cell < 0) return;
        const Frame<D, T> s(pi, cs, dx, dy, dz);
        const uint32_t a = start[cell];
        uint32_t b = start[cell + 1];
        if (!SPH_IN_BOUNDS(P, a <= b && b <= P.chk_cap)) b = a;
        for (uint32_t j = a; j < b; ++j) {
            T rx, ry, rz;
            const T d2 = geometry<D, T>(s, pos[j], rx, ry, rz);
            if (d2 < R2) f(j, rx, ry, rz, d2);
        }
    });
}

// Fast path: the set bits of the neighbour masks (word of neighbour cell idx
// read through mask(idx)), f(j, x, y, z, d2) for each.
template <int D, typename T, typename M, typename F>
__device__ __forceinline__ void for_neighbours_masked(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                                      const vec4_t<T> *__restrict__ pos,
                                                      const uint32_t *__restrict__ start, M &&mask, F &&f)
{
    const T cs = cell_edge<T>(P);
    for_stencil<D>(P, decode_cell(P, c), [&](int idx, int cell, int dx, int dy, int dz) {
        uint32_t w = mask(idx);
        if (!w) return;
        const Frame<D, T> s(pi, cs, dx, dy, dz);
        const uint32_t a = start[cell];
        do {
            const uint32_t j = a + (uint32_t)(__ffs(w) - 1);
            w &= w - 1u;
            if (!SPH_IN_BOUNDS(P, j < P.chk_cap)) break;
            T rx, ry, rz;
            const T d2 = geometry<D, T>(s, pos[j], rx, ry, rz);
            f(j, rx, ry, rz, d2);
        } while (w);
    });
}

// Flattened walk over the hit masks: one iteration per neighbour (self
// included), visiting cells in stencil order and bits from the lowest (the
// order of for_neighbours_masked).  mask(idx) gives the mask word of stencil
// cell idx; c is i's global cell; total = the sum of the popcounts.  A cell's
// first particle and frame shift come from the case's stencil table, so
// nothing is staged.  The lanes of a warp stay converged except at the short
// cell advances (a per-cell inner loop would run each cell for the lane with
// the most hits in it).
template <int D, typename T, typename M, typename F>
__device__ __forceinline__ void walk_masks(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                           const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ start,
                                           M &&mask, int total, F &&f)
{
    constexpr int NC = Stencil<D>::NC;
    int idx = -1;
    uint32_t w = 0, a = 0;
    T fx = pi.x, fy = pi.y, fz = pi.z;
    for (int n = 0; n < total; ++n) {
        if (w == 0) {
            do {
                ++idx;
                w = mask(idx);
            } while (w == 0 && idx < NC - 1);
            if (w == 0) break;  // inconsistent total: never walk past the stencil
            const StencilEntry e = P.stab[idx];
            a = start[(int)c + e.dcell];
            if (sizeof(T) == 4) {
                fx = Ar<T>::sub(pi.x, (T)e.sx);
                fy = Ar<T>::sub(pi.y, (T)e.sy);
                if (D == 3) fz = Ar<T>::sub(pi.z, (T)e.sz);
            }
        }
        const uint32_t j = a + (uint32_t)(__ffs(w) - 1);
        w &= w - 1u;
        if (!SPH_IN_BOUNDS(P, j < P.chk_cap)) break;
        const vec4_t<T> pj = pos[j];
        const T rx = Ar<T>::sub(fx, pj.x);
        const T ry = Ar<T>::sub(fy, pj.y);
        T d2 = Ar<T>::mul(rx, rx);
        d2 = Ar<T>::fma(ry, ry, d2);
        T rz = (T)0;
        if (D == 3) {
            rz = Ar<T>::sub(fz, pj.z);
            d2 = Ar<T>::fma(rz, rz, d2);
        }
        f(j, rx, ry, rz, d2);
    }
}

// ---- cells of edge cs in [h, 2h): the 5^D stencil walked as rows ---------
//
// With K = 2 cells per support radius, the neighbours of i lie in the 5^D
// cells around its own.  The five cells of a stencil row (fixed dy, dz) are
// consecutive in the canonical order, so a row is one contiguous run of the
// sorted copy: 5^(D-1) runs instead of 5^D cells.  One mask word per row
// holds the hits, bit b for the particle at the row's first cell start + b
// (the first cell is cx - 2, clipped to the grid); rows of more than 32
// particles take the slow path.  In the FP32 form the y and z frames are
// constant along a row, while the x frame changes from cell to cell: each
// particle carries its cell's x index in pos.w, and a candidate's x offset in
// i's frame is (o_i - (cx_j - cx_i) cs) - o_j, the same two rounded
// operations (the product exact for |cx_j - cx_i| <= 2) as the per-cell frame.

template <int D, int K> struct Sten;
template <int D> struct Sten<D, 1> { static constexpr int NC = D == 3 ? 27 : 9; };
// K = 2: the mask words of a particle are its 5^(D-1) rows' hit masks, then a
// bitmap of the rows that hold a hit (the force walk jumps from row to row by
// it instead of testing every mask word: 100^3 force pass 0.330 -> 0.279 ms)
template <int D> struct Sten<D, 2> {
    static constexpr int NR = D == 3 ? 25 : 5;  // rows
    static constexpr int NC = NR + 1;           // words per particle
};

// x offset of candidate j in the frame of i (F32; F64 positions are absolute)
template <typename T>
__device__ __forceinline__ T row_dx(const vec4_t<T> &pi, const vec4_t<T> &pj, T cs)
{
    if (sizeof(T) == 4) {
        const T d = Ar<T>::sub(pj.w, pi.w);  // cx_j - cx_i, exact
        return Ar<T>::sub(Ar<T>::fma(-d, cs, pi.x), pj.x);
    }
    return Ar<T>::sub(pi.x, pj.x);
}

// The row trimming's frame of particle i: its offsets in its cell in float
// (the FP32 form's stored offsets; in FP64 x - base(c), rounded once per
// particle: the squared-gap test keeps its 1e-4 margin against that
// rounding), the squared gaps to the cells at x offsets -2, -1, +1, +2, the
// cell edge and the culling radius.
struct RowTrim {
    float oy, oz, gx[4], cs, R2cull;
};

// Squared gap between i (offset o in its cell) and the cell at offset d
// along one axis (F32 cell-relative offsets).
template <typename T>
__device__ __forceinline__ T gap2(int d, T o, T cs)
{
    const T g = d < 0 ? o + (T)(-d - 1) * cs : (d > 0 ? (T)d * cs - o : (T)0);
    return g * g;
}

// Visit the rows of the 5^D stencil of cell c in row order (dz, dy), calling
// f(idx, row_first_cell or -1 when the row is outside the grid, lo, hi, dy,
// dz) with lo / hi the clipped x range [cx + lo, cx + hi] of the row.
template <int D, typename F>
__device__ __forceinline__ void for_rows(const DevParams &P, const CellXYZ &c, F &&f)
{
    const int lo = max(-2, -c.x), hi = min(2, P.nc[0] - 1 - c.x);
    int idx = 0;
#pragma unroll 1
    for (int dz = (D == 3 ? -2 : 0); dz <= (D == 3 ? 2 : 0); ++dz) {
        const int z = c.z + dz;
        const bool zin = D == 2 || (z >= 0 && z < P.nc[2]);
#pragma unroll 1
        for (int dy = -2; dy <= 2; ++dy) {
            const int y = c.y + dy;
            const bool in = zin && y >= 0 && y < P.nc[1];
            const int row = (int)P.cell_off + P.nc[0] * (y + P.nc[1] * (D == 3 ? z : 0)) + c.x;
            f(idx, in ? row : -1, lo, hi, dy, dz);
            ++idx;
        }
    }
}

// Row idx of the 5^D stencil of cell c (the order of for_rows): its first
// cell (or -1 outside the grid), the clipped x range [lo, hi] and (dy, dz).
template <int D>
__device__ __forceinline__ void row_at(const DevParams &P, const CellXYZ &c, int idx, int &row, int &lo, int &hi,
                                       int &dy, int &dz)
{
    const int q = D == 3 ? idx / 5 : 0;
    dz = D == 3 ? q - 2 : 0;
    dy = idx - 5 * q - 2;
    lo = max(-2, -c.x);
    hi = min(2, P.nc[0] - 1 - c.x);
    const int y = c.y + dy, z = c.z + dz;
    const bool in = (D == 2 || (z >= 0 && z < P.nc[2])) && y >= 0 && y < P.nc[1];
    row = in ? (int)P.cell_off + P.nc[0] * (y + P.nc[1] * (D == 3 ? z : 0)) + c.x : -1;
}

// The candidate tests of one stencil row: the row trimmed to the cells whose
// box comes within the support radius (the conservative squared-gap test on
// i's offsets in its cell, in float in both forms; the margin keeps it
// conservative against rounding), hit(j, x, y, z, d2) on every hit in row
// order; returns the row's mask word, bit b for the particle at the row's
// first (clipped, untrimmed) cell start + b.  over = the row holds more than
// 32 particles (its word is left empty: the caller takes the slow path).
// tr: i's trimming frame (row_trim).
template <int D, typename T, typename H>
__device__ __forceinline__ uint32_t row_test(const DevParams &P, const vec4_t<T> &pi, int row, int lo0, int hi0,
                                             int dy, int dz, const RowTrim &tr, const vec4_t<T> *__restrict__ pos,
                                             const uint32_t *__restrict__ start, bool &over, H &&hit)
{
    const T cs = cell_edge<T>(P);
    uint32_t a0 = 0, a = 0, b = 0;
    if (row >= 0) {
        int lo = lo0, hi = hi0;
        {
            const float gyz = gap2<float>(dy, tr.oy, tr.cs) + (D == 3 ? gap2<float>(dz, tr.oz, tr.cs) : 0.0f);
            if (lo == -2 && tr.gx[0] + gyz > tr.R2cull) lo = -1;
            if (lo == -1 && tr.gx[1] + gyz > tr.R2cull) lo = 0;
            if (lo == 0 && gyz > tr.R2cull) lo = 1;  // (the whole row is out of reach)
            if (hi == 2 && tr.gx[3] + gyz > tr.R2cull) hi = 1;
            if (hi == 1 && tr.gx[2] + gyz > tr.R2cull) hi = 0;
        }
        a0 = start[row + lo0];
        if (lo <= hi) {
            a = start[row + lo];
            b = start[row + hi + 1];
            if (!SPH_IN_BOUNDS(P, a0 <= a && a <= b && b <= P.chk_cap)) b = a;
            if (b - a0 > 32u) {
                over = true;
                b = a;
            }
        }
    }
    const T R2 = radius2<T>(P);
    const T fy = Ar<T>::sub(pi.y, (T)dy * cs);
    const T fz = D == 3 ? Ar<T>::sub(pi.z, (T)dz * cs) : (T)0;
    uint32_t w = 0;
    // (a running bit: one shift per candidate instead of a shift of j - a0
    // per hit, 0.453 -> 0.441 ms at 100^3)
    uint32_t bit = a < b ? 1u << (a - a0) : 0u;
#pragma unroll 4
    for (uint32_t j = a; j < b; ++j, bit <<= 1) {
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
        if (d2 < R2) {
            w |= bit;
            hit(j, rx, ry, rz, d2);
        }
    }
    return w;
}

template <int D, typename T>
__device__ __forceinline__ RowTrim row_trim(const DevParams &P, const vec4_t<T> &pi, const CellXYZ &cc)
{
    RowTrim tr;
    tr.cs = cell_edge<float>(P);
    tr.R2cull = radius2<float>(P) * 1.0001f;
    float ox;
    if (sizeof(T) == 4) {
        ox = (float)pi.x;
        tr.oy = (float)pi.y;
        tr.oz = (float)pi.z;
    } else {
        ox = __double2float_rn(__dsub_rn((double)pi.x, P.bval[0][cc.x]));
        tr.oy = __double2float_rn(__dsub_rn((double)pi.y, P.bval[1][cc.y]));
        tr.oz = D == 3 ? __double2float_rn(__dsub_rn((double)pi.z, P.bval[2][cc.z])) : 0.0f;
    }
    tr.gx[0] = gap2<float>(-2, ox, tr.cs);
    tr.gx[1] = gap2<float>(-1, ox, tr.cs);
    tr.gx[2] = gap2<float>(1, ox, tr.cs);
    tr.gx[3] = gap2<float>(2, ox, tr.cs);
    return tr;
}

// Candidate tests of the row stencil, row by row (row_test): one mask word
// per row at mbase[idx * mstride], hit(j, x, y, z, d2) on every hit in row
// order and row_end() after every row, the bitmap of the rows holding a hit
// after the rows' words.  Returns the number of hits (i itself included);
// over = a row held more than 32 particles.
template <int D, typename T, typename H, typename E>
__device__ __forceinline__ int row_candidates(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                              const vec4_t<T> *__restrict__ pos,
                                              const uint32_t *__restrict__ start, uint32_t *mbase, int mstride,
                                              bool &over, H &&hit, E &&row_end)
{
    const CellXYZ cc = decode_cell(P, c);
    const RowTrim tr = row_trim<D, T>(P, pi, cc);
    int total = 0;
    uint32_t rows = 0;  // the rows holding a hit
    for_rows<D>(P, cc, [&](int idx, int row, int lo0, int hi0, int dy, int dz) {
        const uint32_t w = row_test<D, T>(P, pi, row, lo0, hi0, dy, dz, tr, pos, start, over, hit);
        mbase[idx * mstride] = w;
        total += __popc(w);
        rows |= (w != 0u ? 1u : 0u) << idx;
        row_end();
    });
    mbase[Sten<D, 2>::NR * mstride] = rows;
    return total;
}

// Slow path of the row stencil: every candidate of the rows.
template <int D, typename T, typename F>
__device__ __forceinline__ void for_neighbours_scan_rows(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                                         const vec4_t<T> *__restrict__ pos,
                                                         const uint32_t *__restrict__ start, F &&f)
{
    const T cs = cell_edge<T>(P), R2 = radius2<T>(P);
    for_rows<D>(P, decode_cell(P, c), [&](int, int row, int lo, int hi, int dy, int dz) {
        if (row < 0) return;
        const T fy = Ar<T>::sub(pi.y, (T)dy * cs);
        const T fz = D == 3 ? Ar<T>::sub(pi.z, (T)dz * cs) : (T)0;
        const uint32_t a = start[row + lo];
        uint32_t b = start[row + hi + 1];
        if (!SPH_IN_BOUNDS(P, a <= b && b <= P.chk_cap)) b = a;
        for (uint32_t j = a; j < b; ++j) {
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
            if (d2 < R2) f(j, rx, ry, rz, d2);
        }
    });
}

// The set bits of the row masks, row by row (mask(idx): word of row idx).
template <int D, typename T, typename M, typename F>
__device__ __forceinline__ void for_neighbours_masked_rows(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                                           const vec4_t<T> *__restrict__ pos,
                                                           const uint32_t *__restrict__ start, M &&mask, F &&f)
{
    const T cs = cell_edge<T>(P);
    for_rows<D>(P, decode_cell(P, c), [&](int idx, int row, int lo, int, int dy, int dz) {
        uint32_t w = mask(idx);
        if (!w || row < 0) return;
        const T fy = Ar<T>::sub(pi.y, (T)dy * cs);
        const T fz = D == 3 ? Ar<T>::sub(pi.z, (T)dz * cs) : (T)0;
        const uint32_t a = start[row + lo];
        do {
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
            f(j, rx, ry, rz, d2);
        } while (w);
    });
}

// The set bits of one row's mask word w (row idx of cell c's stencil), bits
// from the lowest: one row of for_neighbours_masked_rows.
template <int D, typename T, typename F>
__device__ __forceinline__ void masked_row(const DevParams &P, const vec4_t<T> &pi, const CellXYZ &c, int idx,
                                           uint32_t w, const vec4_t<T> *__restrict__ pos,
                                           const uint32_t *__restrict__ start, F &&f)
{
    int row, lo, hi, dy, dz;
    row_at<D>(P, c, idx, row, lo, hi, dy, dz);
    if (!w || row < 0) return;
    const T cs = cell_edge<T>(P);
    const T fy = Ar<T>::sub(pi.y, (T)dy * cs);
    const T fz = D == 3 ? Ar<T>::sub(pi.z, (T)dz * cs) : (T)0;
    const uint32_t a = start[row + lo];
    do {
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
        f(j, rx, ry, rz, d2);
    } while (w);
}

// Sum over the TEAM lanes of a team (every lane gets the same value: each
// butterfly step adds the same two numbers on both lanes).
template <int TEAM, typename V>
__device__ __forceinline__ V team_sum(V v)
{
#pragma unroll
    for (int o = 1; o < TEAM; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o, TEAM);
    return v;
}

// Flattened walk over the row masks (as walk_masks): one iteration per hit,
// rows in order, bits from the lowest.  The bitmap of the rows in use (the
// word after the rows' masks) gives the next row at once, so its mask word,
// table entry and first particle are loaded together.  The row table
// P.stab gives each row's cell offset (dy, dz at dx = 0) and y / z frame
// shifts; cx_i comes from pi.w, so the row's first cell is
// c + dcell + max(-2, -cx_i).
template <int D, typename T, typename M, typename F>
__device__ __forceinline__ void walk_rows(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                          const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ start,
                                          M &&mask, int total, F &&f)
{
    constexpr int NR = Sten<D, 2>::NR;
    const T cs = cell_edge<T>(P);
    const int cb = (int)c + max(-2, -(int)pi.w);
    uint32_t rows = mask(NR);
    uint32_t w = 0, a = 0;
    T fy = pi.y, fz = pi.z;
    for (int n = 0; n < total; ++n) {
        if (w == 0) {
            if (rows == 0u) break;  // inconsistent total: never walk past the stencil
            const int idx = __ffs(rows) - 1;
            rows &= rows - 1u;
            // (the bitmap and the mask words are written together by the
            // density pass: a row in the bitmap has a nonzero word; testing
            // w here would make the loads below wait for it, 0.279 -> 0.308 ms)
            w = mask(idx);
            const StencilEntry e = P.stab[idx];
            a = start[cb + e.dcell];
            if (sizeof(T) == 4) {
                fy = Ar<T>::sub(pi.y, (T)e.sy);
                if (D == 3) fz = Ar<T>::sub(pi.z, (T)e.sz);
            }
        }
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
        f(j, rx, ry, rz, d2);
    }
}

// Stencil-radius dispatch of the three neighbour iterations.
template <int D, typename T, int K, typename F>
__device__ __forceinline__ void nbr_scan(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                         const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ start,
                                         F &&f)
{
    if (K == 1) for_neighbours_scan<D, T>(P, pi, c, pos, start, f);
    else for_neighbours_scan_rows<D, T>(P, pi, c, pos, start, f);
}
template <int D, typename T, int K, typename M, typename F>
__device__ __forceinline__ void nbr_masked(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                           const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ start,
                                           M &&mask, F &&f)
{
    if (K == 1) for_neighbours_masked<D, T>(P, pi, c, pos, start, mask, f);
    else for_neighbours_masked_rows<D, T>(P, pi, c, pos, start, mask, f);
}
template <int D, typename T, int K, typename M, typename F>
__device__ __forceinline__ void nbr_walk(const DevParams &P, const vec4_t<T> &pi, uint32_t c,
                                         const vec4_t<T> *__restrict__ pos, const uint32_t *__restrict__ start,
                                         M &&mask, int total, F &&f)
{
    if (K == 1) walk_masks<D, T>(P, pi, c, pos, start, mask, total, f);
    else walk_rows<D, T>(P, pi, c, pos, start, mask, total, f);
}

template <typename V>
__device__ __forceinline__ V warp_sum(V v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Mask word of neighbour cell idx of this thread's particle: block-major so
// that a warp's lanes touch consecutive words.
__device__ __forceinline__ size_t mask_index(int NC, int idx)
{
    return (size_t)blockIdx.x * NC * kBlock + (size_t)idx * kBlock + threadIdx.x;
}

}  // namespace sph
