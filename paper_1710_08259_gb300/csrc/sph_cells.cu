// sph_cells.cu -- neighbour-search build: cell hash, binning sort by
// (cell, persistent id), cell start table, reorder.
//
// The uniform cell grid with an edge of at least the support radius is the
// neighbour search of arXiv:1710.08259, Section 3.2.1; it is rebuilt every
// step because positions change every step (Section 4).
//
// GB300 design.  The keys are bounded (linear cell ids < ncells) and, from
// the second step on, the particles arrive nearly sorted (the previous step
// left them in canonical order and few change cell per step).  So instead
// of a multi-pass LSD radix sort the build is a counting sort:
//   1. hash + count: one thread per particle computes its cell in double;
//      lanes of a warp holding the same cell are grouped with __match_any
//      and their leader does one atomicAdd for the group (warp-aggregated
//      binning; near-sorted input makes the groups large); every lane gets
//      its arrival slot inside the cell from the group's popcount prefix;
//   2. exclusive scan of the counts (warp-shuffle prefix sums, three
//      passes over the small count array) -> cell start table, the counts
//      are zeroed for the next step on the way;
//   3. scatter of particle indices to start[cell] + slot (arrival order);
//   4. ordering inside each cell by persistent id, fused with the reorder:
//      the thread of each arrival slot ranks its particle among the cell's
//      members (cells hold ~7 particles in 2D, ~18 in 3D at h = 1.3 dx) and
//      gathers the particle's state straight into its canonical slot.
// All integer work; the result is deterministic and bit-identical to a
// stable sort by (cell, id).
#include <cuda_runtime.h>

#include "sph_internal.cuh"

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

__global__ void k_base_tables(DevParams P, double *bv0, double *bv1, double *bv2, long long *bk0,
                              long long *bk1, long long *bk2)
{
    const int k = blockIdx.y;
    double *bv = k == 0 ? bv0 : (k == 1 ? bv1 : bv2);
    long long *bk = k == 0 ? bk0 : (k == 1 ? bk1 : bk2);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= P.nc[k]; c += gridDim.x * blockDim.x) {
        const double b = cell_base(P.dom_min[k], P.cs, c);
        bv[c] = b;
        bk[c] = okey(b);
    }
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

template <int D>
__global__ void __launch_bounds__(kBlock) k_hash_count(DevParams P, int n, const double *__restrict__ rx,
                                                       const double *__restrict__ ry,
                                                       const double *__restrict__ rz, uint32_t *key,
                                                       uint32_t *rank, uint32_t *cell_count,
                                                       uint32_t *status)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = k < n;
    unsigned mask = __ballot_sync(0xffffffffu, active);
    if (!active) return;
    bool bad = false;
    int cx = cell_axis(P, 0, rx[k], bad);
    int cy = cell_axis(P, 1, ry[k], bad);
    int cz = 0;
    if (D == 3) cz = cell_axis(P, 2, rz[k], bad);
    uint32_t c = (uint32_t)cx + (uint32_t)P.nc[0] * ((uint32_t)cy + (uint32_t)P.nc[1] * (uint32_t)cz);
    unsigned peers = __match_any_sync(mask, c);
    int lane = threadIdx.x & 31;
    int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&cell_count[c], (uint32_t)__popc(peers));
    base = __shfl_sync(peers, base, leader);
    rank[k] = base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    key[k] = c;
    if (bad) atomicOr(status, SPH_STATUS_OUT_OF_DOMAIN);
}

// ---- exclusive scan of the cell counts ----------------------------------

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ cnt,
                                                              uint32_t *block_sums)
{
    const uint4 *c4 = reinterpret_cast<const uint4 *>(cnt + (size_t)blockIdx.x * kScanTile) + threadIdx.x * 2;
    uint4 a = c4[0], b = c4[1];
    uint32_t s = a.x + a.y + a.z + a.w + b.x + b.y + b.z + b.w;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        block_sums[blockIdx.x] = t;
    }
}

// One block: exclusive scan of the block sums in place; total -> *total.
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *block_sums, int nb, uint32_t *total)
{
    __shared__ uint32_t ws[32];
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        uint32_t v = i < nb ? block_sums[i] : 0u;
        uint32_t inc = warp_incl_scan(v);
        if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = inc;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t w = ws[threadIdx.x];
            ws[threadIdx.x] = warp_incl_scan(w) - w;
        }
        __syncthreads();
        uint32_t excl = carry + ws[threadIdx.x >> 5] + inc - v;
        if (i < nb) block_sums[i] = excl;
        __syncthreads();
        if (threadIdx.x == 1023) carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(uint32_t *cnt, const uint32_t *__restrict__ block_sums,
                                                             uint32_t *start, int64_t ncells)
{
    uint4 *c4 = reinterpret_cast<uint4 *>(cnt + (size_t)blockIdx.x * kScanTile) + threadIdx.x * 2;
    uint4 a = c4[0], b = c4[1];
    uint32_t v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t tsum = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) tsum += v[q];
    uint32_t inc = warp_incl_scan(tsum);
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = inc;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t w = threadIdx.x < kScanThreads / 32 ? ws[threadIdx.x] : 0u;
        uint32_t e = warp_incl_scan(w) - w;
        if (threadIdx.x < kScanThreads / 32) ws[threadIdx.x] = e;
    }
    __syncthreads();
    uint32_t run = block_sums[blockIdx.x] + ws[threadIdx.x >> 5] + inc - tsum;
    int64_t c0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * 8;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        if (c0 + q < ncells) start[c0 + q] = run;
        run += v[q];
    }
    // counts are consumed: zero them for the next build
    c4[0] = make_uint4(0, 0, 0, 0);
    c4[1] = make_uint4(0, 0, 0, 0);
}

__global__ void __launch_bounds__(kBlock) k_scatter(int n, const uint32_t *__restrict__ key,
                                                    const uint32_t *__restrict__ rank,
                                                    const uint32_t *__restrict__ start, uint32_t *tmp)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    tmp[start[key[k]] + rank[k]] = (uint32_t)k;
}

// Rank inside the cell by persistent id, then gather the particle's state
// into its canonical slot of the sorted working copy.
template <int D, typename T>
__global__ void __launch_bounds__(kBlock) k_order_gather(DevParams P, int n, sph_state s,
                                                         const uint32_t *__restrict__ key,
                                                         const uint32_t *__restrict__ start,
                                                         const uint32_t *__restrict__ tmp, SortedBufs sb,
                                                         uint32_t *status)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t k = tmp[t];
    uint32_t c = key[k];
    uint32_t s0 = start[c], s1 = start[c + 1];
    uint32_t myid = s.id[k];
    uint32_t pos;
    if (s1 - s0 > (uint32_t)SPH_MAX_CELL) {
        atomicOr(status, SPH_STATUS_CELL_OVERFLOW);
        pos = (uint32_t)t;
    } else {
        uint32_t below = 0, same = 0;
        for (uint32_t q = s0; q < s1; ++q) {
            uint32_t o = s.id[tmp[q]];
            below += (o < myid);
            same += (o == myid);
        }
        if (same != 1) atomicOr(status, SPH_STATUS_DUPLICATE_ID);
        pos = s0 + below;
    }
    const T *vx = static_cast<const T *>(s.v[0]);
    const T *vy = static_cast<const T *>(s.v[1]);
    const T *vz = static_cast<const T *>(s.v[2]);
    double x = s.r[0][k], y = s.r[1][k], z = D == 3 ? s.r[2][k] : 0.0;
    using V4 = vec4_t<T>;
    V4 pv;
    if (sizeof(T) == 4) {
        // cell-relative float offsets: o = (float)(x - base(c))
        uint32_t cx = c % (uint32_t)P.nc[0];
        uint32_t rest = c / (uint32_t)P.nc[0];
        uint32_t cy = rest % (uint32_t)P.nc[1];
        uint32_t cz = rest / (uint32_t)P.nc[1];
        pv.x = (T)__double2float_rn(__dsub_rn(x, P.bval[0][cx]));
        pv.y = (T)__double2float_rn(__dsub_rn(y, P.bval[1][cy]));
        pv.z = D == 3 ? (T)__double2float_rn(__dsub_rn(z, P.bval[2][cz])) : (T)0;
    } else {
        pv.x = (T)x;
        pv.y = (T)y;
        pv.z = (T)z;
    }
    pv.w = (T)0;
    V4 vv;
    vv.x = vx[k];
    vv.y = vy[k];
    vv.z = D == 3 ? vz[k] : (T)0;
    vv.w = (T)0;
    static_cast<V4 *>(sb.pos)[pos] = pv;
    static_cast<V4 *>(sb.vel)[pos] = vv;
    sb.rs[0][pos] = x;
    sb.rs[1][pos] = y;
    if (D == 3) sb.rs[2][pos] = z;
    sb.cell_s[pos] = c;
    sb.id_s[pos] = myid;
    sb.src[pos] = k;
    sb.kind_s[pos] = s.kind[k];
}

template <int D, typename T>
__global__ void __launch_bounds__(kBlock) k_writeback(int n, sph_state s, SortedBufs sb)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    using V4 = vec4_t<T>;
    V4 vv = static_cast<const V4 *>(sb.vel)[i];
    s.r[0][i] = sb.rs[0][i];
    s.r[1][i] = sb.rs[1][i];
    static_cast<T *>(s.v[0])[i] = vv.x;
    static_cast<T *>(s.v[1])[i] = vv.y;
    if (D == 3) {
        s.r[2][i] = sb.rs[2][i];
        static_cast<T *>(s.v[2])[i] = vv.z;
    }
    s.id[i] = sb.id_s[i];
    s.kind[i] = sb.kind_s[i];
}

static inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

template <int D, typename T>
static cudaError_t build_impl(const DevParams &P, int n, const sph_state &s, const CellBufs &cb,
                              const SortedBufs &sb, uint32_t *status, cudaStream_t st)
{
    if (n > 0) {
        k_hash_count<D><<<blocks_for(n, kBlock), kBlock, 0, st>>>(P, n, s.r[0], s.r[1], s.r[2], cb.key,
                                                                   cb.rank, cb.cell_count, status);
    }
    k_scan_reduce<<<cb.scan_blocks, kScanThreads, 0, st>>>(cb.cell_count, cb.block_sums);
    k_scan_top<<<1, 1024, 0, st>>>(cb.block_sums, cb.scan_blocks, cb.cell_start + cb.ncells);
    k_scan_apply<<<cb.scan_blocks, kScanThreads, 0, st>>>(cb.cell_count, cb.block_sums, cb.cell_start,
                                                          cb.ncells);
    if (n > 0) {
        k_scatter<<<blocks_for(n, kBlock), kBlock, 0, st>>>(n, cb.key, cb.rank, cb.cell_start, cb.tmp);
        k_order_gather<D, T><<<blocks_for(n, kBlock), kBlock, 0, st>>>(P, n, s, cb.key, cb.cell_start,
                                                                        cb.tmp, sb, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_build(const DevParams &P, bool f32, int n, const sph_state &s, const CellBufs &cb,
                         const SortedBufs &sb, uint32_t *status, cudaStream_t st)
{
    if (P.dim == 2) return f32 ? build_impl<2, float>(P, n, s, cb, sb, status, st)
                               : build_impl<2, double>(P, n, s, cb, sb, status, st);
    return f32 ? build_impl<3, float>(P, n, s, cb, sb, status, st)
               : build_impl<3, double>(P, n, s, cb, sb, status, st);
}

cudaError_t launch_base_tables(const DevParams &P, double *bval[3], long long *bkey[3], cudaStream_t st)
{
    int mx = P.nc[0] > P.nc[1] ? P.nc[0] : P.nc[1];
    if (P.nc[2] > mx) mx = P.nc[2];
    dim3 grid((mx + 1 + 255) / 256, P.dim);
    k_base_tables<<<grid, 256, 0, st>>>(P, bval[0], bval[1], bval[2], bkey[0], bkey[1], bkey[2]);
    return cudaGetLastError();
}

cudaError_t launch_writeback(const DevParams &P, bool f32, int n, const sph_state &s,
                             const SortedBufs &sb, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int nb = blocks_for(n, kBlock);
    if (P.dim == 2) {
        if (f32) k_writeback<2, float><<<nb, kBlock, 0, st>>>(n, s, sb);
        else k_writeback<2, double><<<nb, kBlock, 0, st>>>(n, s, sb);
    } else {
        if (f32) k_writeback<3, float><<<nb, kBlock, 0, st>>>(n, s, sb);
        else k_writeback<3, double><<<nb, kBlock, 0, st>>>(n, s, sb);
    }
    return cudaGetLastError();
}

}  // namespace sph
