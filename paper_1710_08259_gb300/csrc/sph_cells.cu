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
//      runs of equal cells in adjacent lanes (near-sorted input makes them
//      long) are counted by one atomicAdd each, and every lane gets its
//      arrival slot inside the cell from its place in the run;
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
#include "sph_phases.cuh"

namespace sph {

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

template <int D>
__global__ void __launch_bounds__(kBlock) k_hash_count(DevParams P, int n, sph_state s, uint32_t *key,
                                                       uint32_t *rank, uint32_t *cell_count, uint32_t *status)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    dev_hash<D>(P, k, k < n, s, key, rank, cell_count, status);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ cnt,
                                                              uint32_t *block_sums)
{
    __shared__ uint32_t ws[33];
    dev_scan_reduce(cnt, block_sums, blockIdx.x, ws);
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *block_sums, int nb, uint32_t *total)
{
    __shared__ uint32_t ws[33];
    dev_scan_top(block_sums, nb, total, ws);
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(uint32_t *cnt, const uint32_t *__restrict__ block_sums,
                                                             uint32_t *start, int64_t ncells)
{
    __shared__ uint32_t ws[33];
    dev_scan_apply(cnt, block_sums, start, ncells, blockIdx.x, ws);
}

__global__ void __launch_bounds__(kBlock) k_scatter(int n, const uint32_t *__restrict__ key,
                                                    const uint32_t *__restrict__ rank,
                                                    const uint32_t *__restrict__ start, uint32_t *tmp)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dev_scatter(k, key, rank, start, tmp);
}

template <int D, typename T>
__global__ void __launch_bounds__(kBlock) k_order_gather(DevParams P, int n, sph_state s,
                                                         const uint32_t *__restrict__ key,
                                                         const uint32_t *__restrict__ start,
                                                         const uint32_t *__restrict__ tmp, SortedBufs sb,
                                                         uint32_t *status)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) dev_order_gather<D, T>(P, t, s, key, start, tmp, sb, status);
}

// The gather of a build whose canonical state goes to caller arrays (sb's
// rs / id_s / kind_s point there) and that also reorders up to kMaxFields
// caller fields of W words per element: out[slot] = in[source].
template <int D, typename T, int W>
__global__ void __launch_bounds__(kBlock) k_order_gather_into(DevParams P, int n, sph_state s,
                                                              const uint32_t *__restrict__ key,
                                                              const uint32_t *__restrict__ start,
                                                              const uint32_t *__restrict__ tmp, SortedBufs sb,
                                                              FieldSet fs, uint32_t *status)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint32_t pos = dev_order_gather<D, T>(P, t, s, key, start, tmp, sb, status);
    if (pos == 0xFFFFFFFFu) return;
    const size_t src = (size_t)tmp[t] * W, dst = (size_t)pos * W;
#pragma unroll 1
    for (int f = 0; f < fs.nf; ++f) {
#pragma unroll
        for (int w = 0; w < W; ++w) fs.out[f][dst + w] = fs.in[f][src + w];
    }
}

template <int D, typename T>
__global__ void __launch_bounds__(kBlock) k_writeback(int n, sph_state s, SortedBufs sb, int carry_rho)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    using V4 = vec4_t<T>;
    V4 vv = static_cast<const V4 *>(sb.vel)[i];
    s.r[0][i] = sb.rs[0][i];
    s.r[1][i] = sb.rs[1][i];
    if (D == 3) s.r[2][i] = sb.rs[2][i];
    if (s.v[0]) {  // (the field model's state has no velocity)
        static_cast<T *>(s.v[0])[i] = vv.x;
        static_cast<T *>(s.v[1])[i] = vv.y;
        if (D == 3) static_cast<T *>(s.v[2])[i] = vv.z;
    }
    s.id[i] = sb.id_s[i];
    s.kind[i] = sb.kind_s[i];
    // a density field that the model carries (continuity equation) moves
    // with its particle
    if (carry_rho == 1) static_cast<T *>(s.rho)[i] = vv.w;
    // the radius and mass of a sphere move with it
    if (carry_rho == 2) {
        static_cast<T *>(s.radius)[i] = static_cast<const V4 *>(sb.pos)[i].w;
        static_cast<T *>(s.mass)[i] = vv.w;
    }
}

static inline int blocks_for(int n, int b) { return (n + b - 1) / b; }

template <int D, typename T>
static cudaError_t build_impl(const DevParams &P, int n, const sph_state &s, const CellBufs &cb,
                              const SortedBufs &sb, uint32_t *status, cudaStream_t st)
{
    if (n > 0)
        k_hash_count<D><<<blocks_for(n, kBlock), kBlock, 0, st>>>(P, n, s, cb.key, cb.rank, cb.cell_count, status);
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
template <int D, typename T>
static cudaError_t build_into_impl(const DevParams &P, int n, const sph_state &s, const CellBufs &cb,
                                   const SortedBufs &sb, const FieldSet &fs, int words, uint32_t *status,
                                   cudaStream_t st)
{
    if (n > 0)
        k_hash_count<D><<<blocks_for(n, kBlock), kBlock, 0, st>>>(P, n, s, cb.key, cb.rank, cb.cell_count, status);
    k_scan_reduce<<<cb.scan_blocks, kScanThreads, 0, st>>>(cb.cell_count, cb.block_sums);
    k_scan_top<<<1, 1024, 0, st>>>(cb.block_sums, cb.scan_blocks, cb.cell_start + cb.ncells);
    k_scan_apply<<<cb.scan_blocks, kScanThreads, 0, st>>>(cb.cell_count, cb.block_sums, cb.cell_start,
                                                          cb.ncells);
    if (n > 0) {
        k_scatter<<<blocks_for(n, kBlock), kBlock, 0, st>>>(n, cb.key, cb.rank, cb.cell_start, cb.tmp);
        if (words == 2)
            k_order_gather_into<D, T, 2><<<blocks_for(n, kBlock), kBlock, 0, st>>>(P, n, s, cb.key, cb.cell_start,
                                                                                 cb.tmp, sb, fs, status);
        else
            k_order_gather_into<D, T, 1><<<blocks_for(n, kBlock), kBlock, 0, st>>>(P, n, s, cb.key, cb.cell_start,
                                                                                 cb.tmp, sb, fs, status);
    }
    return cudaGetLastError();
}
cudaError_t launch_build_into(const DevParams &P, bool f32, int n, const sph_state &s, const CellBufs &cb,
                              const SortedBufs &sb, const FieldSet &fs, int elem_bytes, uint32_t *status,
                              cudaStream_t st)
{
    const int words = elem_bytes / 4;
    if (P.dim == 2) return f32 ? build_into_impl<2, float>(P, n, s, cb, sb, fs, words, status, st)
                               : build_into_impl<2, double>(P, n, s, cb, sb, fs, words, status, st);
    return f32 ? build_into_impl<3, float>(P, n, s, cb, sb, fs, words, status, st)
               : build_into_impl<3, double>(P, n, s, cb, sb, fs, words, status, st);
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

// ---- reorder of a caller field by the last build's permutation -------------
template <int W>
__global__ void __launch_bounds__(256) k_reorder_field(int n, const uint32_t *__restrict__ src,
                                                       const uint32_t *__restrict__ in, uint32_t *out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const size_t s = (size_t)src[k] * W, d = (size_t)k * W;
#pragma unroll
    for (int w = 0; w < W; ++w) out[d + w] = in[s + w];
}

cudaError_t launch_reorder_field(int n, const uint32_t *src, const void *in_, void *out_, int elem_bytes,
                                 cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int nb = (n + 255) / 256;
    const uint32_t *in = static_cast<const uint32_t *>(in_);
    uint32_t *out = static_cast<uint32_t *>(out_);
    switch (elem_bytes / 4) {
    case 1: k_reorder_field<1><<<nb, 256, 0, st>>>(n, src, in, out); break;
    case 2: k_reorder_field<2><<<nb, 256, 0, st>>>(n, src, in, out); break;
    case 3: k_reorder_field<3><<<nb, 256, 0, st>>>(n, src, in, out); break;
    case 4: k_reorder_field<4><<<nb, 256, 0, st>>>(n, src, in, out); break;
    case 6: k_reorder_field<6><<<nb, 256, 0, st>>>(n, src, in, out); break;
    default: k_reorder_field<8><<<nb, 256, 0, st>>>(n, src, in, out); break;
    }
    return cudaGetLastError();
}

// Several fields of the same element size in one pass: the permutation is
// read once per particle.
template <int W>
__global__ void __launch_bounds__(256) k_reorder_fields(int n, const uint32_t *__restrict__ src, FieldSet fs)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const size_t s = (size_t)src[k] * W, d = (size_t)k * W;
#pragma unroll 1
    for (int f = 0; f < fs.nf; ++f) {
        const uint32_t *__restrict__ in = fs.in[f];
        uint32_t *__restrict__ out = fs.out[f];
#pragma unroll
        for (int w = 0; w < W; ++w) out[d + w] = in[s + w];
    }
}

cudaError_t launch_reorder_fields(int n, const uint32_t *src, const FieldSet &fs, int elem_bytes, cudaStream_t st)
{
    if (n <= 0 || fs.nf <= 0) return cudaSuccess;
    const int nb = (n + 255) / 256;
    switch (elem_bytes / 4) {
    case 1: k_reorder_fields<1><<<nb, 256, 0, st>>>(n, src, fs); break;
    case 2: k_reorder_fields<2><<<nb, 256, 0, st>>>(n, src, fs); break;
    case 3: k_reorder_fields<3><<<nb, 256, 0, st>>>(n, src, fs); break;
    case 4: k_reorder_fields<4><<<nb, 256, 0, st>>>(n, src, fs); break;
    case 6: k_reorder_fields<6><<<nb, 256, 0, st>>>(n, src, fs); break;
    default: k_reorder_fields<8><<<nb, 256, 0, st>>>(n, src, fs); break;
    }
    return cudaGetLastError();
}

// ---- copies through page-locked host memory --------------------------------
// A copy kernel reads or writes the host array through its device mapping,
// so the transfer runs as loads and stores of many SMs over the chip-to-chip
// link instead of one DMA queue.  16-byte words, the ragged tail by bytes.
__global__ void __launch_bounds__(256) k_copy_bytes(const unsigned char *__restrict__ src,
                                                     unsigned char *__restrict__ dst, size_t bytes)
{
    const size_t nv = bytes / 16;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    for (size_t k = t0; k < nv; k += stride) d4[k] = s4[k];
    for (size_t k = nv * 16 + t0; k < bytes; k += stride) dst[k] = src[k];
}

cudaError_t launch_copy_bytes(const void *src, void *dst, size_t bytes, int sms, cudaStream_t st)
{
    if (bytes == 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u)
        return cudaErrorInvalidValue;  // callers pass 16-byte aligned arrays
    const size_t blocks_needed = (bytes / 16 + 255) / 256 + 1;
    const int grid = (int)(blocks_needed < (size_t)sms * 4 ? blocks_needed : (size_t)sms * 4);
    k_copy_bytes<<<grid, 256, 0, st>>>(static_cast<const unsigned char *>(src), static_cast<unsigned char *>(dst),
                                       bytes);
    return cudaGetLastError();
}

// Several device-to-device copies in one launch (block row y copies section
// y): 16-byte words, the ragged tail by bytes.
__global__ void __launch_bounds__(256) k_copy_sections(CopySections cs)
{
    const int y = blockIdx.y;
    if (y >= cs.m) return;
    const unsigned char *__restrict__ src = static_cast<const unsigned char *>(cs.src[y]);
    unsigned char *__restrict__ dst = static_cast<unsigned char *>(cs.dst[y]);
    const size_t bytes = cs.bytes[y];
    const size_t nv = bytes / 16;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t0 = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (size_t k = t0; k < nv; k += stride) reinterpret_cast<uint4 *>(dst)[k] = reinterpret_cast<const uint4 *>(src)[k];
    for (size_t k = nv * 16 + t0; k < bytes; k += stride) dst[k] = src[k];
}

cudaError_t launch_copy_sections(const CopySections &cs, cudaStream_t st)
{
    if (cs.m <= 0) return cudaSuccess;
    size_t most = 0;
    for (int y = 0; y < cs.m; ++y) {
        if ((reinterpret_cast<uintptr_t>(cs.src[y]) | reinterpret_cast<uintptr_t>(cs.dst[y])) & 15u)
            return cudaErrorInvalidValue;  // sections start 16-byte aligned
        most = cs.bytes[y] > most ? cs.bytes[y] : most;
    }
    const size_t need = (most / 16 + 255) / 256 + 1;
    const unsigned gx = (unsigned)(need < 64 ? need : 64);
    k_copy_sections<<<dim3(gx, (unsigned)cs.m), 256, 0, st>>>(cs);
    return cudaGetLastError();
}

cudaError_t launch_writeback(const DevParams &P, bool f32, int n, const sph_state &s,
                             const SortedBufs &sb, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    int nb = blocks_for(n, kBlock);
    // 1: carry the density field, 2: carry radius and mass
    const int cr = (P.model == SPH_MODEL_EXAMPLE_1A && s.rho)                  ? 1
                   : (P.model == SPH_MODEL_DEM && s.radius && s.mass) ? 2
                                                                      : 0;
    if (P.dim == 2) {
        if (f32) k_writeback<2, float><<<nb, kBlock, 0, st>>>(n, s, sb, cr);
        else k_writeback<2, double><<<nb, kBlock, 0, st>>>(n, s, sb, cr);
    } else {
        if (f32) k_writeback<3, float><<<nb, kBlock, 0, st>>>(n, s, sb, cr);
        else k_writeback<3, double><<<nb, kBlock, 0, st>>>(n, s, sb, cr);
    }
    return cudaGetLastError();
}

}  // namespace sph
