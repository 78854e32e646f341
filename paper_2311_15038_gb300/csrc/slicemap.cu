// slicemap.cu -- multi-resolution slicemap atlases (slices converted into
// slicemaps, Sec. III; a coarse dataset shown before the full one, Sec. II),
// with the keep/discard classification of Sec. III-A / III-D fused in.
//
// Level 0: voxel i along an axis of n source and m level voxels covers source
// voxels [floor(i n/m), floor((i+1) n/m)); its value is the mean of the
// covered (kept) voxels rounded half up.  Level k >= 1: exact 2x2x2 mean of
// level k-1, rounded half up.
//
// One CTA owns a group of G = 2^f x 2^f level-0 rows (f = halvings fused into
// the kernel, at most 2; 4 x 4 rows when nothing is fused), so the source is
// read from HBM exactly once:
//  * accumulate: for each level-0 row, every thread owns 16-byte column
//    vectors of the source rows of that row's (z, y) footprint and sums them
//    in registers (8 loads in flight), then stores the column sums to a
//    double-buffered shared row; when a source row has fewer vectors than
//    the CTA has threads, several level-0 rows are accumulated at once;
//  * x-reduce: threads sum each output voxel's x-footprint from shared
//    memory, divide, write the level-0 atlas row and keep the value in shared
//    memory;
//  * after the group: levels 1..f from shared memory.
// Loads are plain 16-byte streaming loads, 8 in flight per thread, 4 CTAs per
// SM; rows that do not start on a 16-byte boundary are read as pairs of
// aligned loads funnel-shifted together.  For a step keep table on data of at
// most 15 bits two 16-bit values are tested and added per 32-bit word (see
// add_vector; u8 data spreads its bytes over two such words).  Remaining levels run as a
// separate 2x2x2 kernel, and max grids are built by maxgrid_kernel.
// When the keep table is a step (keep[b] = b >= T, as Otsu, ITS and explicit
// thresholds produce) the per-voxel table lookup becomes one comparison.
// A single u8 level from rows of at most 1024 bytes (many small volumes) takes
// a warp-per-row kernel instead (slicemap_rows_u8_kernel below), which sums
// bytes as exact fp16 pairs and reduces x through prefix sums.
#include <algorithm>

#include <cuda_fp16.h>
#include <string.h>

#include "slicemap_common.cuh"

namespace mctp {
namespace {

constexpr int kSmThreads = 256;
constexpr int kSmUnroll = 8;
constexpr int kMaxFused = 2;
constexpr int kGroupUnfused = 4;
constexpr int kMaxGroupRows = 16;  // (2^kMaxFused)^2 and kGroupUnfused^2

template <typename T>
struct L0Args {
    const T *vol;
    int64_t nx, ny, nz;
    int32_t mx, my, mz;
    int32_t fused;              // extra levels produced in-kernel (0..2)
    int32_t group;              // a CTA owns group x group level-0 rows (z, y)
    int32_t rows_per_pass;      // level-0 rows accumulated at once
    int64_t cstride;            // column sums per shared row: nx rounded up to a multiple of 4
    T *atlas[kMaxFused + 1];
    int32_t tiles_x[kMaxFused + 1];
    int64_t pitch[kMaxFused + 1];  // atlas row pitch in elements
    int64_t elems[kMaxFused + 1];  // atlas elements (bounds of the checked build)
    const uint8_t *keep;        // nullptr: no filtering
    int32_t nbins;
    int32_t shift;
    uint32_t limit;             // 2^bits
    int32_t packed;             // two-lane u16 arithmetic is exact for this volume
};

// 16 bytes of a source row starting at byte 16 v of the row, for any row
// alignment: two aligned 16-byte loads funnel-shifted together.  The second
// load is made only when its chunk holds bytes of the row (so no load leaves
// a 16-byte chunk that holds valid data); bytes past the row end are garbage
// and the caller ignores the elements they form.
__device__ __forceinline__ uint4 load_row_vector(const char *row, int64_t v, int64_t row_bytes)
{
    const uintptr_t ad = reinterpret_cast<uintptr_t>(row) + uintptr_t(v) * 16u;
    const uint32_t m = uint32_t(ad & 15u);
    const char *c0 = reinterpret_cast<const char *>(ad - m);
    const uint4 q0 = ld_stream_v4(c0);
    if (m == 0) return q0;
    uint4 q1 = make_uint4(0u, 0u, 0u, 0u);
    if (c0 + 16 < row + row_bytes) q1 = ld_stream_v4(c0 + 16);
    const uint32_t W[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
    const uint32_t sh = (m & 3u) * 8u;
    switch (m >> 2) {
    case 0: return make_uint4(__funnelshift_r(W[0], W[1], sh), __funnelshift_r(W[1], W[2], sh),
                              __funnelshift_r(W[2], W[3], sh), __funnelshift_r(W[3], W[4], sh));
    case 1: return make_uint4(__funnelshift_r(W[1], W[2], sh), __funnelshift_r(W[2], W[3], sh),
                              __funnelshift_r(W[3], W[4], sh), __funnelshift_r(W[4], W[5], sh));
    case 2: return make_uint4(__funnelshift_r(W[2], W[3], sh), __funnelshift_r(W[3], W[4], sh),
                              __funnelshift_r(W[4], W[5], sh), __funnelshift_r(W[5], W[6], sh));
    default: return make_uint4(__funnelshift_r(W[3], W[4], sh), __funnelshift_r(W[4], W[5], sh),
                               __funnelshift_r(W[5], W[6], sh), __funnelshift_r(W[6], W[7], sh));
    }
}

// u8 data, two 16-bit lanes per word: bytes 0,2 of each word into acc[2k],
// bytes 1,3 into acc[2k+1]; for a step table the lane test of add_vector
// (values < 256 never carry).
template <int kMode>
__device__ __forceinline__ void add_vector_u8_packed(const uint4 &q, uint32_t *acc, uint32_t k_fast)
{
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t even, odd;  // bytes 0,2 and 1,3 zero-extended to 16-bit lanes
        asm("prmt.b32 %0, %1, 0, 0x4240;" : "=r"(even) : "r"(w[k]));
        asm("prmt.b32 %0, %1, 0, 0x4341;" : "=r"(odd) : "r"(w[k]));
        if (kMode == 2) {
            even &= lane_sign_mask(even + k_fast);
            odd &= lane_sign_mask(odd + k_fast);
        }
        acc[2 * k] += even;
        acc[2 * k + 1] += odd;
    }
}

// Column sums of one level-0 row, vector path: each thread owns 16-byte column
// vectors of the row and sums them over the footprint's source rows in
// registers (aligned rows: 8 loads in flight; other rows: two loads per vector,
// 4 rows in flight).
template <typename T, int kMode, bool kPacked, bool kAligned, bool kOne>
__device__ __forceinline__ void accumulate_row_vec(const L0Args<T> &a, int zlo, int zhi, int ylo, int yhi,
                                                   uint32_t *colsum, const uint8_t *lut, uint32_t lo, int64_t v0)
{
    constexpr int E = 16 / sizeof(T);
    constexpr int NA = kPacked ? (sizeof(T) == 1 ? 8 : 4) : E;
    constexpr int UNROLL = kAligned ? kSmUnroll : kSmUnroll / 2;
    const int64_t row_bytes = a.nx * int64_t(sizeof(T));
    const int64_t V = (row_bytes + 15) / 16;
    const int wy = yhi - ylo;
    const int R = (zhi - zlo) * wy;
    // source rows of the footprint in (z, y) order: step one row, or jump to
    // the first footprint row of the next slice
    const int64_t slice_jump = (a.ny - wy + 1) * row_bytes;
    const char *first = reinterpret_cast<const char *>(a.vol) + (int64_t(zlo) * a.ny + ylo) * row_bytes;
    const uint32_t k_fast = (0x8000u - lo) * 0x00010001u, ovf_bits = ~((a.limit - 1u) * 0x00010001u);
    // kOne: this thread's single vector v0 (v0 < V); else vectors v0, v0 +
    // blockDim.x, ...
    for (int64_t v = v0; kOne || v < V; v += blockDim.x) {
        uint32_t acc[NA];
#pragma unroll
        for (int e = 0; e < NA; ++e) acc[e] = 0u;
        uint32_t seen = 0;
        const char *rs = first;  // start of the current source row
        int yi = 0;
        for (int r0 = 0; r0 < R; r0 += UNROLL) {
            uint4 q[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                if (r0 + u < R) {
                    q[u] = kAligned ? ld_stream_v4(rs + v * 16) : load_row_vector(rs, v, row_bytes);
                    if (++yi == wy) { yi = 0; rs += slice_jump; }
                    else rs += row_bytes;
                } else {
                    q[u] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                if (kPacked && sizeof(T) == 1) add_vector_u8_packed<kMode>(q[u], acc, k_fast);
                else add_vector<T, kMode, kPacked>(q[u], acc, lut, a.shift, a.limit, lo, k_fast, seen);
            }
        }
        if (kPacked && sizeof(T) == 2 && kMode == 2 && (seen & ovf_bits)) {
            // a value at or above 2^bits: redo this vector with the exact test
            const uint32_t k_lo2 = lo * 0x00010001u, k_lim2 = a.limit * 0x00010001u;
#pragma unroll
            for (int e = 0; e < NA; ++e) acc[e] = 0u;
            rs = first;
            yi = 0;
            for (int r = 0; r < R; ++r) {
                add_vector_exact(kAligned ? ld_stream_v4(rs + v * 16) : load_row_vector(rs, v, row_bytes), acc,
                                 k_lo2, k_lim2);
                if (++yi == wy) { yi = 0; rs += slice_jump; }
                else rs += row_bytes;
            }
        }
        uint32_t sums[E];
        if (kPacked && sizeof(T) == 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                sums[4 * k] = acc[2 * k] & 0xffffu;
                sums[4 * k + 2] = acc[2 * k] >> 16;
                sums[4 * k + 1] = acc[2 * k + 1] & 0xffffu;
                sums[4 * k + 3] = acc[2 * k + 1] >> 16;
            }
        } else if (kPacked) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                sums[2 * k] = acc[k] & 0xffffu;
                sums[2 * k + 1] = acc[k] >> 16;
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) sums[e] = acc[e];
        }
        uint32_t *dst = colsum + v * E;
        if (kAligned) {
#pragma unroll
            for (int e = 0; e < E; e += 4)
                *reinterpret_cast<uint4 *>(dst + e) = make_uint4(sums[e], sums[e + 1], sums[e + 2], sums[e + 3]);
        } else if (v * E + E <= a.nx) {
#pragma unroll
            for (int e = 0; e < E; e += 4)
                *reinterpret_cast<uint4 *>(dst + e) = make_uint4(sums[e], sums[e + 1], sums[e + 2], sums[e + 3]);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e)
                if (v * E + e < a.nx) dst[e] = sums[e];
        }
        if (kOne) break;
    }
}

template <typename T, bool kVec, int kMode, bool kPacked, bool kMulti>
__device__ void level0_group(const L0Args<T> &a, int Z0, int Y0, int gz, int gy, uint32_t *colsum, uint16_t *grp,
                             const int32_t *zb, const int32_t *yb, const int32_t *xb, const uint8_t *lut,
                             uint32_t lo)
{
    // per pass (double-buffered like the column sums): each row's footprint
    // size R in (z, y) (0 for rows past the level) and its atlas row offset
    __shared__ uint32_t row_R[2][kMaxGroupRows];
    __shared__ int64_t row_off[2][kMaxGroupRows];
    const int G = gz * gy;
    const int P = kMulti ? a.rows_per_pass : 1;
    const int64_t V = (a.nx * int64_t(sizeof(T)) + 15) / 16;  // 16-byte vectors per source row
    const int t = int(threadIdx.x);
    int pass = 0;
    for (int g0 = 0; g0 < G; g0 += P, ++pass) {
        const int b = pass & 1;
        uint32_t *buf = colsum + b * (int64_t(P) * a.cstride);
        if (t < P && g0 + t < G) {
            const int g = g0 + t, zz = g / gy, yy = g - zz * gy;
            const bool in = Z0 + zz < a.mz && Y0 + yy < a.my;
            row_R[b][t] = in ? uint32_t((zb[zz + 1] - zb[zz]) * (yb[yy + 1] - yb[yy])) : 0u;
            row_off[b][t] = in ? atlas_ptr(a.atlas[0], a.pitch[0], a.tiles_x[0], a.mx, a.my, 0, Y0 + yy, Z0 + zz) -
                                     a.atlas[0]
                               : 0;
        }
        // accumulate: one row with all threads striding over its vectors, or
        // (kMulti) P rows at once, thread t on vector t % V of row g0 + t / V
        const int j = kMulti ? int(t / V) : 0;
        const int g = g0 + j;
        const int zz = g / gy, yy = g - zz * gy;
        if (j < P && g < G && Z0 + zz < a.mz && Y0 + yy < a.my)
            accumulate_row_vec<T, kMode, kPacked, kVec, kMulti>(a, zb[zz], zb[zz + 1], yb[yy], yb[yy + 1],
                                                                buf + int64_t(j) * a.cstride, lut, lo,
                                                                kMulti ? t - int64_t(j) * V : int64_t(t));
        __syncthreads();
        // x-reduce: each thread takes output columns x and all rows of the pass
        const int rows = min(P, G - g0);
        for (int x = t; x < a.mx; x += blockDim.x) {
            const int xlo = xb[x];
            const uint32_t xw = uint32_t(xb[x + 1] - xlo);
            for (int jj = 0; jj < rows; ++jj) {
                const uint32_t R = row_R[b][jj];
                if (R == 0) continue;  // past the level (ragged group)
                const uint32_t *cs = buf + int64_t(jj) * a.cstride + xlo;
                uint32_t sum = 0;
                for (uint32_t k = 0; k < xw; ++k) sum += cs[k];
                const uint32_t cnt = xw * R;
                const uint32_t val = (sum + cnt / 2u) / cnt;
                if (in_range(row_off[b][jj] + x, a.elems[0], kFaultAtlasWrite)) a.atlas[0][row_off[b][jj] + x] = (T)val;
                if (grp) grp[(g0 + jj) * a.mx + x] = uint16_t(val);
            }
        }
        // no barrier: the next pass accumulates into the other buffers, and the
        // barrier after it orders this pass's reads before their reuse
    }
}

template <typename T, bool kVec, bool kMulti>
__global__ void __launch_bounds__(kSmThreads, 4) slicemap_level0_kernel(L0Args<T> a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int gz = a.group, gy = a.group;
    const int ngy = (a.my + gy - 1) / gy;
    const int Z0 = (blockIdx.x / ngy) * gz, Y0 = (blockIdx.x % ngy) * gy;

    uint32_t *colsum = reinterpret_cast<uint32_t *>(smem);                     // 2 * rows_per_pass * cstride
    int32_t *xb = reinterpret_cast<int32_t *>(colsum + 2 * a.rows_per_pass * a.cstride);  // mx + 1
    int32_t *zb = xb + a.mx + 1;                                               // gz + 1 (this group)
    int32_t *yb = zb + gz + 1;                                                 // gy + 1
    uint16_t *grp = reinterpret_cast<uint16_t *>(yb + gy + 1);                 // gz*gy*mx (when fused)
    uint16_t *grp1 = grp + (a.fused ? gz * gy * a.mx : 0);                     // (gz/2)(gy/2)(mx/2)
    uint8_t *lut = reinterpret_cast<uint8_t *>(grp1 + (a.fused > 1 ? (gz / 2) * (gy / 2) * (a.mx / 2) : 0));

    for (int i = threadIdx.x; i <= a.mx; i += blockDim.x) xb[i] = int32_t((int64_t(i) * a.nx) / a.mx);
    for (int i = threadIdx.x; i <= gz; i += blockDim.x) zb[i] = int32_t((int64_t(min(Z0 + i, a.mz)) * a.nz) / a.mz);
    for (int i = threadIdx.x; i <= gy; i += blockDim.x) yb[i] = int32_t((int64_t(min(Y0 + i, a.my)) * a.ny) / a.my);
    __syncthreads();

    __shared__ int sh_keep[2];
    uint32_t lo = 0;
    const int mode = load_keep_table(a.keep, a.nbins, a.shift, a.limit, lut, sh_keep, int(threadIdx.x),
                                     int(blockDim.x), &lo, [] { __syncthreads(); });
    uint16_t *g0 = a.fused ? grp : nullptr;
    if (mode == 0 && sizeof(T) == 1 && a.packed)
        level0_group<T, kVec, 0, true, kMulti>(a, Z0, Y0, gz, gy, colsum, g0, zb, yb, xb, lut, lo);
    else if (mode == 0) level0_group<T, kVec, 0, false, kMulti>(a, Z0, Y0, gz, gy, colsum, g0, zb, yb, xb, lut, lo);
    else if (mode == 1) level0_group<T, kVec, 1, false, kMulti>(a, Z0, Y0, gz, gy, colsum, g0, zb, yb, xb, lut, lo);
    else if (a.packed) level0_group<T, kVec, 2, true, kMulti>(a, Z0, Y0, gz, gy, colsum, g0, zb, yb, xb, lut, lo);
    else level0_group<T, kVec, 2, false, kMulti>(a, Z0, Y0, gz, gy, colsum, g0, zb, yb, xb, lut, lo);
    if (!a.fused) return;
    __syncthreads();

    // level 1 from the group's level-0 values
    {
        const int hz = gz / 2, hy = gy / 2, hx = a.mx / 2;
        const int my1 = a.my / 2;
        for (int i = threadIdx.x; i < hz * hy * hx; i += blockDim.x) {
            const int x = i % hx, t = i / hx, b = t % hy, c = t / hy;
            uint32_t s = 0;
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const uint16_t *src = grp + ((2 * c + dz) * gy + (2 * b + dy)) * a.mx + 2 * x;
                    s += uint32_t(src[0]) + uint32_t(src[1]);
                }
            const uint32_t val = (s + 4u) / 8u;
            T *w1 = atlas_ptr(a.atlas[1], a.pitch[1], a.tiles_x[1], hx, my1, x, Y0 / 2 + b, Z0 / 2 + c);
            if (in_range(w1 - a.atlas[1], a.elems[1], kFaultAtlasWrite)) *w1 = (T)val;
            if (a.fused > 1) grp1[(c * hy + b) * hx + x] = uint16_t(val);
        }
    }
    if (a.fused < 2) return;
    __syncthreads();
    // level 2 from level 1
    {
        const int hz = gz / 4, hy = gy / 4, hx = a.mx / 4;
        const int gy1 = gy / 2, mx1 = a.mx / 2, my2 = a.my / 4;
        for (int i = threadIdx.x; i < hz * hy * hx; i += blockDim.x) {
            const int x = i % hx, t = i / hx, b = t % hy, c = t / hy;
            uint32_t s = 0;
#pragma unroll
            for (int dz = 0; dz < 2; ++dz)
#pragma unroll
                for (int dy = 0; dy < 2; ++dy) {
                    const uint16_t *src = grp1 + ((2 * c + dz) * gy1 + (2 * b + dy)) * mx1 + 2 * x;
                    s += uint32_t(src[0]) + uint32_t(src[1]);
                }
            T *w2 = atlas_ptr(a.atlas[2], a.pitch[2], a.tiles_x[2], hx, my2, x, Y0 / 4 + b, Z0 / 4 + c);
            if (in_range(w2 - a.atlas[2], a.elems[2], kFaultAtlasWrite)) *w2 = (T)((s + 4u) / 8u);
        }
    }
}

// ---- level 0 alone, u8 source rows of at most 1024 bytes (many small volumes)
//
// One warp per level-0 row (z, y) at a time, persistent warps, no CTA barrier
// in the loop.  Lane l owns source columns [32 l, 32 l + 32): for each source
// row of the footprint it loads the aligned 16-byte chunks around its 32
// bytes (any row alignment), funnel-shifts them into place and adds the kept
// bytes into column sums.  For a step keep table (or none) the sums are fp16
// pairs: byte b is the fp16 value b 2^-24, the sum of up to 8 bytes is exact,
// and an fp16 value k 2^-24 with integer k <= 2048 has the bit pattern k, so
// the pair registers are at the same time packed 16-bit column sums; they are
// folded into the warp's shared row after every 8 source rows.  A general
// keep table adds bytes into packed 16-bit integer sums.  The warp then turns
// the row's column sums into exclusive prefix sums E (a scan within each lane
// and across the warp), and output voxel x takes E[c1] - E[c0] over its
// footprint [c0, c1), divided and rounded.
constexpr int kRowsWarps = 8;
constexpr int kRowsMaxCols = 1024;     // source row bytes the kernel takes
constexpr int kRowsMaxYZ = 4096;       // level rows / slices the tables take
constexpr int kRowsScratch = 1064;     // u32 per warp: column sums (80 B per lane), then E (see below)

struct RowsArgs {
    const uint8_t *vol;
    int64_t nx, ny, nz;
    int32_t mx, my, mz;
    uint8_t *atlas;
    int32_t tiles_x;
    int64_t pitch;
    int64_t elems;  // atlas elements (bounds of the checked build)
    const uint8_t *keep;
    int32_t nbins, shift;
    uint32_t limit;
};

// The 32 bytes at p (lane-uniform p & 15) from the aligned chunks c0, c0 + 16,
// c0 + 32; a chunk that holds no byte of [row, end) is not loaded (its bytes
// form columns past the row, which no output reads).
__device__ __forceinline__ void load_lane32(const char *p, const char *end, uint4 &lo, uint4 &hi)
{
    const uint32_t m = uint32_t(reinterpret_cast<uintptr_t>(p) & 15u);
    const uint4 *c = reinterpret_cast<const uint4 *>(p - m);
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    const uint4 q0 = __ldg(c);
    const uint4 q1 = reinterpret_cast<const char *>(c + 1) < end ? __ldg(c + 1) : z;
    if (m == 0) {
        lo = q0;
        hi = q1;
        return;
    }
    const uint4 q2 = reinterpret_cast<const char *>(c + 2) < end ? __ldg(c + 2) : z;
    const uint32_t W[12] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y, q2.z, q2.w};
    const uint32_t sh = (m & 3u) * 8u;
    uint32_t o[8];
    switch (m >> 2) {
    case 0:
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = __funnelshift_r(W[k], W[k + 1], sh);
        break;
    case 1:
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = __funnelshift_r(W[k + 1], W[k + 2], sh);
        break;
    case 2:
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = __funnelshift_r(W[k + 2], W[k + 3], sh);
        break;
    default:
#pragma unroll
        for (int k = 0; k < 8; ++k) o[k] = __funnelshift_r(W[k + 3], W[k + 4], sh);
        break;
    }
    lo = make_uint4(o[0], o[1], o[2], o[3]);
    hi = make_uint4(o[4], o[5], o[6], o[7]);
}

// 16 bytes into packed even/odd column sums for a general keep table (mode 1).
__device__ __forceinline__ void add_vector_u8_lut(const uint4 &q, uint32_t *acc, const uint8_t *lut, int shift)
{
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t b[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t v = (w[k] >> (8 * j)) & 0xffu;
            b[j] = lut[v >> shift] ? v : 0u;
        }
        acc[2 * k] += b[0] | (b[2] << 16);
        acc[2 * k + 1] += b[1] | (b[3] << 16);
    }
}

__device__ __forceinline__ __half2 bits_h2(uint32_t u)
{
    __half2 h;
    memcpy(&h, &u, 4);
    return h;
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h)
{
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}

// 16 bytes into fp16 pair sums: acc[2 k] gets bytes 0, 2 of word k, acc[2 k + 1]
// bytes 1, 3; with a step table (mode 2) only bytes >= thr (the pair value of
// the lowest kept byte).
template <int kMode>
__device__ __forceinline__ void add_vector_u8_h2(const uint4 &q, __half2 *acc, __half2 thr)
{
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        uint32_t e, o;
        asm("prmt.b32 %0, %1, 0, 0x4240;" : "=r"(e) : "r"(w[k]));
        asm("prmt.b32 %0, %1, 0, 0x4341;" : "=r"(o) : "r"(w[k]));
        const __half2 he = bits_h2(e), ho = bits_h2(o);
        if (kMode == 2) {
            acc[2 * k] = __hfma2(he, __hge2(he, thr), acc[2 * k]);
            acc[2 * k + 1] = __hfma2(ho, __hge2(ho, thr), acc[2 * k + 1]);
        } else {
            acc[2 * k] = __hadd2(acc[2 * k], he);
            acc[2 * k + 1] = __hadd2(acc[2 * k + 1], ho);
        }
    }
}

// Even/odd pair sums of 32 columns (acc[8 g + 2 k]: columns 16 g + 4 k + {0, 2},
// acc[8 g + 2 k + 1]: + {1, 3}) as 16 words of consecutive column pairs, stored
// or added into dst.
__device__ __forceinline__ void store_columns(const uint32_t *acc, uint4 *dst, bool add)
{
#pragma unroll
    for (int g = 0; g < 2; ++g) {
        uint32_t w[8];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t ev = acc[8 * g + 2 * k], od = acc[8 * g + 2 * k + 1];
            asm("prmt.b32 %0, %1, %2, 0x5410;" : "=r"(w[2 * k]) : "r"(ev), "r"(od));
            asm("prmt.b32 %0, %1, %2, 0x7632;" : "=r"(w[2 * k + 1]) : "r"(ev), "r"(od));
        }
        uint4 v0 = make_uint4(w[0], w[1], w[2], w[3]), v1 = make_uint4(w[4], w[5], w[6], w[7]);
        if (add) {
            const uint4 o0 = dst[2 * g], o1 = dst[2 * g + 1];
            v0 = make_uint4(v0.x + o0.x, v0.y + o0.y, v0.z + o0.z, v0.w + o0.w);
            v1 = make_uint4(v1.x + o1.x, v1.y + o1.y, v1.z + o1.z, v1.w + o1.w);
        }
        dst[2 * g] = v0;
        dst[2 * g + 1] = v1;
    }
}

// Column sums of a level row's footprint into the lane's 32 columns of dst.
template <int kMode>
__device__ __forceinline__ void rows_accumulate(const RowsArgs &a, const uint8_t *lut, __half2 thr, int zlo, int ylo,
                                                int wy, int R, int lane, uint4 *dst)
{
    const int64_t nx = a.nx;
    const char *rs = reinterpret_cast<const char *>(a.vol) + (int64_t(zlo) * a.ny + ylo) * nx;
    const int64_t slice_jump = (a.ny - wy + 1) * nx;
    int yi = 0;
    auto next_row = [&]() {
        const char *r = rs;
        if (++yi == wy) { yi = 0; rs += slice_jump; } else { rs += nx; }
        return r;
    };
    if constexpr (kMode == 1) {
        uint32_t acc[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = 0u;
        for (int r = 0; r < R; r += 2) {
            uint4 q[4];
            const char *r1 = next_row();
            load_lane32(r1 + 32 * lane, r1 + nx, q[0], q[1]);
            if (r + 1 < R) {
                const char *r2 = next_row();
                load_lane32(r2 + 32 * lane, r2 + nx, q[2], q[3]);
            } else {
                q[2] = q[3] = make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) add_vector_u8_lut(q[u], acc + 8 * (u & 1), lut, a.shift);
        }
        store_columns(acc, dst, false);
    } else {
    for (int r = 0; r < R;) {
        __half2 h[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) h[e] = bits_h2(0u);
        const int first = r;
        const int rend = min(R, r + 8);  // 8 rows of bytes sum to at most 2040: exact in fp16
        for (; r < rend; r += 2) {
            uint4 q[4];
            const char *r1 = next_row();
            load_lane32(r1 + 32 * lane, r1 + nx, q[0], q[1]);
            if (r + 1 < rend) {
                const char *r2 = next_row();
                load_lane32(r2 + 32 * lane, r2 + nx, q[2], q[3]);
            } else {
                q[2] = q[3] = make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) add_vector_u8_h2<kMode>(q[u], h + 8 * (u & 1), thr);
        }
        uint32_t acc[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = h2_bits(h[e]);
        store_columns(acc, dst, first > 0);
    }
    }
}

// floor((sum + cnt / 2) / cnt) for a quotient of at most a few hundred, from
// an approximate reciprocal of cnt: the estimate is within one of the
// quotient, and one correction step each way makes it exact.
__device__ __forceinline__ uint32_t div_round(uint32_t sum, uint32_t cnt, float rcp)
{
    const uint32_t n = sum + cnt / 2u;
    uint32_t q = __float2uint_rz(__fmul_rn(float(n), rcp));
    if ((q + 1u) * cnt <= n) ++q;
    else if (q * cnt > n) --q;
    return q;
}

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__global__ void __launch_bounds__(kRowsWarps * 32, 4) slicemap_rows_u8_kernel(const __grid_constant__ RowsArgs a)
{
    extern __shared__ __align__(16) uint8_t smem_rows[];
    int32_t *xb = reinterpret_cast<int32_t *>(smem_rows);  // mx + 1
    int32_t *yb = xb + a.mx + 1;                           // my + 1
    int32_t *zb = yb + a.my + 1;                           // mz + 1
    const int ntab = a.mx + a.my + a.mz + 3;
    uint32_t *scratch = reinterpret_cast<uint32_t *>(smem_rows + ((size_t(ntab) * 4 + 15) / 16) * 16);
    uint8_t *lut = reinterpret_cast<uint8_t *>(scratch + kRowsWarps * kRowsScratch);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i <= a.mx; i += blockDim.x) xb[i] = int32_t((int64_t(i) * a.nx) / a.mx);
    for (int i = threadIdx.x; i <= a.my; i += blockDim.x) yb[i] = int32_t((int64_t(i) * a.ny) / a.my);
    for (int i = threadIdx.x; i <= a.mz; i += blockDim.x) zb[i] = int32_t((int64_t(i) * a.nz) / a.mz);
    __shared__ int sh_keep[2];
    uint32_t lo = 0;
    const int mode = load_keep_table(a.keep, a.nbins, a.shift, a.limit, lut, sh_keep, int(threadIdx.x),
                                     int(blockDim.x), &lo, [] { __syncthreads(); });
    __syncthreads();
    // the fp16 pair of the lowest kept byte (bit pattern lo, see above)
    const __half2 thr = bits_h2(lo | (lo << 16));
    uint32_t *mine = scratch + warp * kRowsScratch;
    uint4 *cols = reinterpret_cast<uint4 *>(mine) + 5 * lane;  // this lane's 32 column sums (80 bytes)
    // E[c], c = 0..nx, at word c + c / 32: a lane's 32 stores fall in 32 different banks
    uint32_t *E = mine;
    const int64_t nrows = int64_t(a.mz) * a.my;
    const int64_t nwarps = int64_t(gridDim.x) * kRowsWarps;
    const bool active = 32 * lane < a.nx;
    const int wlo = int(a.nx / a.mx);  // footprint widths along x are wlo or wlo + 1
    const int64_t first_row = int64_t(blockIdx.x) * kRowsWarps + warp;
    const int step_z = int(nwarps / a.my), step_y = int(nwarps - int64_t(step_z) * a.my);
    int z = int(first_row / a.my), y = int(first_row - int64_t(z) * a.my);
    for (int64_t row = first_row; row < nrows; row += nwarps) {
        const int zlo = zb[z], ylo = yb[y];
        const int wy = yb[y + 1] - ylo, R = (zb[z + 1] - zlo) * wy;
        if (active) {
            if (mode == 0) rows_accumulate<0>(a, lut, thr, zlo, ylo, wy, R, lane, cols);
            else if (mode == 1) rows_accumulate<1>(a, lut, thr, zlo, ylo, wy, R, lane, cols);
            else rows_accumulate<2>(a, lut, thr, zlo, ylo, wy, R, lane, cols);
        }
        __syncwarp();
        // exclusive prefix sums of the row's columns (E[32 l + j + 1] from lane l)
        uint32_t v[16];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            const uint4 t = cols[g];
            v[4 * g] = t.x; v[4 * g + 1] = t.y; v[4 * g + 2] = t.z; v[4 * g + 3] = t.w;
        }
        uint32_t total = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i) total += (v[i] & 0xffffu) + (v[i] >> 16);
        uint32_t incl = total;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        __syncwarp();
        uint32_t run = incl - total;
        if (lane == 0) E[0] = 0u;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int c = 32 * lane + 2 * i + 1;
            run += v[i] & 0xffffu;
            E[c + (c >> 5)] = run;
            run += v[i] >> 16;
            E[c + 1 + ((c + 1) >> 5)] = run;
        }
        __syncwarp();
        uint8_t *out = atlas_ptr(a.atlas, a.pitch, a.tiles_x, a.mx, a.my, 0, y, z);
        const float rcp_lo = rcp_approx(float(wlo * R)), rcp_hi = rcp_approx(float((wlo + 1) * R));
        for (int x = lane; x < a.mx; x += 32) {
            const int c0 = xb[x], c1 = xb[x + 1];
            const uint32_t sum = E[c1 + (c1 >> 5)] - E[c0 + (c0 >> 5)];
            const int w = c1 - c0;
            const uint32_t q = div_round(sum, uint32_t(w * R), w == wlo ? rcp_lo : rcp_hi);
            if (in_range((out - a.atlas) + x, a.elems, kFaultAtlasWrite)) out[x] = uint8_t(q);
        }
        __syncwarp();
        y += step_y;
        z += step_z;
        if (y >= a.my) { y -= a.my; ++z; }
    }
}

// Level k+1 from level k, atlas to atlas: exact 2x2x2 mean, rounded half up.
template <typename T>
__global__ void __launch_bounds__(256) halve_kernel(const T *__restrict__ src, int64_t src_pitch, int src_tx, int mx,
                                                     int my, T *__restrict__ dst, int64_t dst_pitch, int dst_tx,
                                                     int64_t total, int64_t dst_elems)
{
    const int hx = mx / 2, hy = my / 2;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int x = int(i % hx);
        const int64_t t = i / hx;
        const int y = int(t % hy), z = int(t / hy);
        uint32_t s = 0;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                const T *p = atlas_ptr(const_cast<T *>(src), src_pitch, src_tx, mx, my, 2 * x, 2 * y + dy, 2 * z + dz);
                s += uint32_t(__ldg(p)) + uint32_t(__ldg(p + 1));
            }
        T *w = atlas_ptr(dst, dst_pitch, dst_tx, hx, hy, x, y, z);
        if (in_range(w - dst, dst_elems, kFaultAtlasWrite)) *w = (T)((s + 4u) / 8u);
    }
}

// Per-cell maxima of a level (occupancy data for the renderer): cell c covers
// voxels [8c, 8c + 8] per axis, clamped (the cell plus the first voxel of the
// next one: everything a trilinear sample with its lower corner in the cell
// reads).  One block per (cz, cy) row of cells; each thread keeps column
// maxima of its x positions over the cell rows' 9 x 9 (y, z) atlas rows,
// loading the 9 rows of a slice together, then each cell takes the maximum of
// its 9 columns from shared memory.
// Block `block` of a level's max grid: cell row (cz, cy) = (block / gy, block % gy).
template <typename T>
__device__ __forceinline__ void maxgrid_row(const T *__restrict__ atlas, int64_t pitch, int tiles_x, int mx, int my,
                                            int mz, uint16_t *__restrict__ grid, int gx, int gy, int block,
                                            uint32_t *colmax)
{
    constexpr int c = MCTP_MAXGRID_CELL;
    const int cy = block % gy, cz = block / gy;
    const int z1 = min(cz * c + c, mz - 1), y0 = cy * c, ny_rows = min(cy * c + c, my - 1) - y0 + 1;
    for (int x = threadIdx.x; x < mx; x += blockDim.x) {
        uint32_t m = 0;
        for (int z = cz * c; z <= z1; ++z) {
            const T *row = atlas_ptr(const_cast<T *>(atlas), pitch, tiles_x, mx, my, x, y0, z);
            uint32_t v[c + 1];
#pragma unroll
            for (int r = 0; r <= c; ++r) v[r] = r < ny_rows ? uint32_t(__ldg(row + int64_t(r) * pitch)) : 0u;
#pragma unroll
            for (int r = 0; r <= c; ++r) m = max(m, v[r]);
        }
        colmax[x] = m;
    }
    __syncthreads();
    for (int cx = threadIdx.x; cx < gx; cx += blockDim.x) {
        uint32_t m = 0;
        const int x1 = min(cx * c + c, mx - 1);
        for (int x = cx * c; x <= x1; ++x) m = max(m, colmax[x]);
        grid[(int64_t(cz) * gy + cy) * gx + cx] = uint16_t(m);
    }
}


// Block `block` of a level's max grid with 32-bit loads: 4 u8 or 2 u16
// columns per word (SIMD byte / halfword maxima), 64 words by 4 row groups
// per 256 threads, so a thread makes about 20 loads per cell row instead of
// 81; needs mx and the atlas pitch in whole words and a 4-byte-aligned atlas.
template <typename T>
__device__ __forceinline__ void maxgrid_row_vec(const T *__restrict__ atlas, int64_t pitch, int tiles_x, int mx,
                                                int my, int mz, uint16_t *__restrict__ grid, int gx, int gy, int block,
                                                uint32_t *colmax)
{
    constexpr int c = MCTP_MAXGRID_CELL;
    constexpr int EPW = 4 / int(sizeof(T));
    const int cy = block % gy, cz = block / gy;
    const int z0 = cz * c, z1 = min(cz * c + c, mz - 1), y0 = cy * c, y1 = min(cy * c + c, my - 1);
    const int nw = mx / EPW;
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    uint32_t *part = colmax + mx;  // [4][nw]
    for (int w = tx; w < nw; w += 64) {
        uint32_t m = 0;
        for (int z = z0; z <= z1; ++z) {
            const uint32_t *row = reinterpret_cast<const uint32_t *>(
                atlas_ptr(const_cast<T *>(atlas), pitch, tiles_x, mx, my, w * EPW, 0, z));
            const int64_t wp = pitch / EPW;
            for (int y = y0 + ty; y <= y1; y += 4) {
                const uint32_t v = __ldg(row + int64_t(y) * wp);
                m = sizeof(T) == 1 ? __vmaxu4(m, v) : __vmaxu2(m, v);
            }
        }
        part[ty * nw + w] = m;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < nw; w += blockDim.x) {
        uint32_t m = part[w];
        for (int k = 1; k < 4; ++k) m = sizeof(T) == 1 ? __vmaxu4(m, part[k * nw + w]) : __vmaxu2(m, part[k * nw + w]);
        for (int e = 0; e < EPW; ++e) colmax[w * EPW + e] = sizeof(T) == 1 ? (m >> (8 * e)) & 0xffu : (m >> (16 * e)) & 0xffffu;
    }
    __syncthreads();
    for (int cx = threadIdx.x; cx < gx; cx += blockDim.x) {
        uint32_t m = 0;
        const int x1 = min(cx * c + c, mx - 1);
        for (int x = cx * c; x <= x1; ++x) m = max(m, colmax[x]);
        grid[(int64_t(cz) * gy + cy) * gx + cx] = uint16_t(m);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) maxgrid_kernel(const T *__restrict__ atlas, int64_t pitch, int tiles_x, int mx,
                                                      int my, int mz, uint16_t *__restrict__ grid, int gx, int gy,
                                                      int vec)
{
    extern __shared__ uint32_t colmax[];
    if (vec)
        maxgrid_row_vec<T>(atlas, pitch, tiles_x, mx, my, mz, grid, gx, gy, int(blockIdx.x), colmax);
    else
        maxgrid_row<T>(atlas, pitch, tiles_x, mx, my, mz, grid, gx, gy, int(blockIdx.x), colmax);
}

// The max grids of up to kGridBatch levels (of one element type) in one
// launch: item i owns blocks [first[i], first[i + 1]).  Many small volumes
// then share one launch instead of one short launch each.
constexpr int kGridBatch = 64;
struct MaxgridItem {
    const void *atlas;
    uint16_t *grid;
    int64_t pitch;
    int32_t tiles_x, mx, my, mz, gx, gy;
    int32_t vec;  // maxgrid_row_vec applies (see maxgrid_vec_ok)
};
struct MaxgridBatch {
    int32_t count;
    int32_t first[kGridBatch + 1];
    MaxgridItem item[kGridBatch];
};

template <typename T>
__global__ void __launch_bounds__(256) maxgrid_batch_kernel(const __grid_constant__ MaxgridBatch b)
{
    extern __shared__ uint32_t colmax[];
    int lo = 0, hi = b.count - 1;  // the item whose block range holds blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.first[mid] <= int(blockIdx.x)) lo = mid;
        else hi = mid - 1;
    }
    const MaxgridItem &it = b.item[lo];
    if (it.vec)
        maxgrid_row_vec<T>(static_cast<const T *>(it.atlas), it.pitch, it.tiles_x, it.mx, it.my, it.mz, it.grid, it.gx,
                           it.gy, int(blockIdx.x) - b.first[lo], colmax);
    else
        maxgrid_row<T>(static_cast<const T *>(it.atlas), it.pitch, it.tiles_x, it.mx, it.my, it.mz, it.grid, it.gx,
                       it.gy, int(blockIdx.x) - b.first[lo], colmax);
}

// Zero the tiles of an atlas that hold no slice.
int zero_unused_tiles(void *atlas, int esize, int mx, int my, int mz, int tx, int ty, cudaStream_t s)
{
    const size_t pitch = size_t(tx) * mx * esize;
    const int full_rows = mz / tx, rem = mz % tx;
    if (rem) {
        char *p = static_cast<char *>(atlas) + size_t(full_rows) * my * pitch + size_t(rem) * mx * esize;
        if (cudaMemset2DAsync(p, pitch, 0, size_t(tx - rem) * mx * esize, my, s) != cudaSuccess) return MCTP_ECUDA;
    }
    const int used_rows = full_rows + (rem ? 1 : 0);
    if (used_rows < ty) {
        char *p = static_cast<char *>(atlas) + size_t(used_rows) * my * pitch;
        if (cudaMemsetAsync(p, 0, size_t(ty - used_rows) * my * pitch, s) != cudaSuccess) return MCTP_ECUDA;
    }
    return MCTP_OK;
}

// Whether level k takes the 32-bit-load max grid, and the shared memory its
// blocks need either way.
template <typename T>
bool maxgrid_vec_ok(const mctp_slicemap *sm, int k, size_t &smem)
{
    constexpr int EPW = 4 / int(sizeof(T));
    const int mx = sm->dims[k][0];
    const int64_t pitch = int64_t(sm->tiles_x[k]) * mx;
    const size_t vsmem = size_t(mx) * sizeof(uint32_t) + size_t(4) * (size_t(mx) + 3) * sizeof(uint32_t);
    // u8 only: with two u16 columns per word a thread makes about as many
    // loads as the one-column kernel, which measured faster on u16 levels
    const bool vec = sizeof(T) == 1 && mx % EPW == 0 && pitch % EPW == 0 &&
                     (reinterpret_cast<uintptr_t>(sm->atlas[k]) & 3) == 0 && vsmem <= 200 * 1024;
    smem = vec ? vsmem : size_t(mx) * sizeof(uint32_t);
    return vec;
}

template <typename T>
int launch_maxgrid(const mctp_slicemap *sm, int k, cudaStream_t s)
{
    const int c = MCTP_MAXGRID_CELL;
    const int mx = sm->dims[k][0], my = sm->dims[k][1], mz = sm->dims[k][2];
    const int gx = (mx + c - 1) / c, gy = (my + c - 1) / c, gz = (mz + c - 1) / c;
    size_t smem = 0;
    const bool vec = maxgrid_vec_ok<T>(sm, k, smem);
    if (smem > 200 * 1024) return MCTP_EUNSUPPORTED;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(maxgrid_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return MCTP_ECUDA;
    maxgrid_kernel<T><<<unsigned(int64_t(gy) * gz), 256, smem, s>>>(
        static_cast<const T *>(sm->atlas[k]), int64_t(sm->tiles_x[k]) * mx, sm->tiles_x[k], mx, my, mz,
        static_cast<uint16_t *>(sm->maxgrid[k]), gx, gy, vec ? 1 : 0);
    return launch_status();
}

template <typename T>
int launch_slicemap(const T *vol, const mctp_volume_desc *d, const uint8_t *keep, int nbins, const mctp_slicemap *sm,
                    cudaStream_t s, bool maxgrids = true)
{
    int rc = MCTP_OK;
    int done_levels = 0;   // levels 1..done_levels written by the level-0 kernel
    const int64_t rmax_all = ((d->ny + sm->dims[0][1] - 1) / sm->dims[0][1]) *
                             ((d->nz + sm->dims[0][2] - 1) / sm->dims[0][2]);
    if (sizeof(T) == 1 && sm->nlevels == 1 && d->nx <= kRowsMaxCols && sm->dims[0][1] <= kRowsMaxYZ &&
        sm->dims[0][2] <= kRowsMaxYZ && rmax_all * 255 < 65536) {
        // a single u8 level with short rows: the warp-per-row kernel
        RowsArgs a{};
        a.vol = reinterpret_cast<const uint8_t *>(vol);
        a.nx = d->nx; a.ny = d->ny; a.nz = d->nz;
        a.mx = sm->dims[0][0]; a.my = sm->dims[0][1]; a.mz = sm->dims[0][2];
        a.atlas = static_cast<uint8_t *>(sm->atlas[0]);
        a.tiles_x = sm->tiles_x[0];
        a.pitch = int64_t(sm->tiles_x[0]) * sm->dims[0][0];
        a.elems = a.pitch * sm->tiles_y[0] * sm->dims[0][1];
        a.keep = keep;
        a.nbins = keep ? nbins : 0;
        a.shift = keep ? bin_shift(d->bits, nbins) : 0;
        a.limit = 1u << d->bits;
        const size_t smem = ((size_t(a.mx + a.my + a.mz + 3) * 4 + 15) / 16) * 16 +
                            size_t(kRowsWarps) * kRowsScratch * 4 + (keep ? size_t(nbins) : 0);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(slicemap_rows_u8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
                cudaSuccess)
            return MCTP_ECUDA;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, slicemap_rows_u8_kernel, kRowsWarps * 32, smem) !=
            cudaSuccess)
            return MCTP_ECUDA;
        per_sm = std::max(per_sm, 1);
        const int64_t rows = int64_t(a.mz) * a.my;
        const int64_t grid = std::min<int64_t>((rows + kRowsWarps - 1) / kRowsWarps, int64_t(per_sm) * num_sms());
        slicemap_rows_u8_kernel<<<unsigned(grid), kRowsWarps * 32, smem, s>>>(a);
        rc = launch_status();
        if (rc != MCTP_OK) return rc;
        done_levels = sm->nlevels;  // nothing left for the other kernels
    } else {
        const int fused = std::min(sm->nlevels - 1, kMaxFused);
        L0Args<T> a{};
        a.vol = vol;
        a.nx = d->nx; a.ny = d->ny; a.nz = d->nz;
        a.mx = sm->dims[0][0]; a.my = sm->dims[0][1]; a.mz = sm->dims[0][2];
        a.fused = fused;
        for (int k = 0; k <= fused; ++k) {
            a.atlas[k] = static_cast<T *>(sm->atlas[k]);
            a.tiles_x[k] = sm->tiles_x[k];
            a.pitch[k] = int64_t(sm->tiles_x[k]) * sm->dims[k][0];
            a.elems[k] = a.pitch[k] * sm->tiles_y[k] * sm->dims[k][1];
        }
        a.keep = keep;
        a.nbins = keep ? nbins : 0;
        a.shift = keep ? bin_shift(d->bits, nbins) : 0;
        a.limit = 1u << d->bits;
        // groups of 2^f x 2^f rows when f levels are fused, else 4 x 4 rows
        // (ragged at the level's edges)
        a.group = fused ? (1 << fused) : kGroupUnfused;
        const int gz = a.group, gy = a.group;
        const int64_t V = (a.nx * int64_t(sizeof(T)) + 15) / 16;
        a.rows_per_pass = int(std::max<int64_t>(1, std::min<int64_t>(int64_t(gz) * gy, kSmThreads / V)));
        // two 16-bit lanes per word stay exact when a footprint's sum fits 16 bits
        const int64_t rmax = ((d->ny + a.my - 1) / a.my) * ((d->nz + a.mz - 1) / a.mz);
        a.packed = d->bits <= 15 && rmax * ((int64_t(1) << d->bits) - 1) < 65536;
        a.cstride = (a.nx + 3) & ~int64_t(3);
        size_t smem = size_t(2) * a.rows_per_pass * a.cstride * 4 + size_t(a.mx + 1 + gz + 1 + gy + 1) * 4;
        if (fused) smem += size_t(gz) * gy * a.mx * 2;
        if (fused > 1) smem += size_t(gz / 2) * (gy / 2) * (a.mx / 2) * 2;
        smem += keep ? size_t(nbins) : 0;
        if (smem > 220 * 1024) return MCTP_EUNSUPPORTED;
        const bool vec = (reinterpret_cast<uintptr_t>(vol) & 15) == 0 && ((a.nx * int64_t(sizeof(T))) & 15) == 0;
        const bool multi = a.rows_per_pass > 1;
        auto kern = vec ? (multi ? slicemap_level0_kernel<T, true, true> : slicemap_level0_kernel<T, true, false>)
                        : (multi ? slicemap_level0_kernel<T, false, true> : slicemap_level0_kernel<T, false, false>);
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
            return MCTP_ECUDA;
        const int64_t blocks = int64_t((a.mz + gz - 1) / gz) * ((a.my + gy - 1) / gy);
        if (blocks > 0x7fffffff) return MCTP_EUNSUPPORTED;
        kern<<<unsigned(blocks), kSmThreads, smem, s>>>(a);
        rc = launch_status();
        if (rc != MCTP_OK) return rc;
        done_levels = fused;
    }
    for (int k = done_levels + 1; k < sm->nlevels; ++k) {
        const int mx = sm->dims[k - 1][0], my = sm->dims[k - 1][1];
        const int64_t total = int64_t(sm->dims[k][0]) * sm->dims[k][1] * sm->dims[k][2];
        const int64_t grid = std::min<int64_t>((total + 255) / 256, int64_t(num_sms()) * 16);
        halve_kernel<T><<<unsigned(std::max<int64_t>(grid, 1)), 256, 0, s>>>(
            static_cast<const T *>(sm->atlas[k - 1]), int64_t(sm->tiles_x[k - 1]) * mx, sm->tiles_x[k - 1], mx, my,
            static_cast<T *>(sm->atlas[k]), int64_t(sm->tiles_x[k]) * sm->dims[k][0], sm->tiles_x[k], total,
            int64_t(sm->tiles_x[k]) * sm->dims[k][0] * sm->tiles_y[k] * sm->dims[k][1]);
        rc = launch_status();
        if (rc != MCTP_OK) return rc;
    }
    for (int k = 0; k < sm->nlevels; ++k) {
        rc = zero_unused_tiles(sm->atlas[k], int(sizeof(T)), sm->dims[k][0], sm->dims[k][1], sm->dims[k][2],
                               sm->tiles_x[k], sm->tiles_y[k], s);
        if (rc != MCTP_OK) return rc;
    }
    for (int k = 0; maxgrids && k < sm->nlevels; ++k) {
        if (!sm->maxgrid[k]) continue;
        rc = launch_maxgrid<T>(sm, k, s);
        if (rc != MCTP_OK) return rc;
    }
    return MCTP_OK;
}

// The max grids of every level of sms[0..count) that has one, kGridBatch
// levels per launch.
template <typename T>
int launch_maxgrid_batch(const mctp_slicemap *sms, int count, cudaStream_t s)
{
    MaxgridBatch b{};
    size_t smem = 0;
    auto flush = [&]() -> int {
        if (b.count == 0) return MCTP_OK;
        if (smem > 48 * 1024 &&
            cudaFuncSetAttribute(maxgrid_batch_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
                cudaSuccess)
            return MCTP_ECUDA;
        maxgrid_batch_kernel<T><<<unsigned(b.first[b.count]), 256, smem, s>>>(b);
        b.count = 0;
        smem = 0;
        return launch_status();
    };
    for (int i = 0; i < count; ++i) {
        const mctp_slicemap *sm = &sms[i];
        for (int k = 0; k < sm->nlevels; ++k) {
            if (!sm->maxgrid[k]) continue;
            const int c = MCTP_MAXGRID_CELL;
            const int mx = sm->dims[k][0], my = sm->dims[k][1], mz = sm->dims[k][2];
            const int gx = (mx + c - 1) / c, gy = (my + c - 1) / c, gz = (mz + c - 1) / c;
            size_t need = 0;
            const bool vec = maxgrid_vec_ok<T>(sm, k, need);
            if (need > 200 * 1024) return MCTP_EUNSUPPORTED;
            if (b.count == kGridBatch || int64_t(b.first[b.count]) + int64_t(gy) * gz > 0x7fffffff) {
                const int rc = flush();
                if (rc != MCTP_OK) return rc;
            }
            MaxgridItem &it = b.item[b.count];
            it.atlas = sm->atlas[k];
            it.grid = static_cast<uint16_t *>(sm->maxgrid[k]);
            it.pitch = int64_t(sm->tiles_x[k]) * mx;
            it.tiles_x = sm->tiles_x[k];
            it.mx = mx; it.my = my; it.mz = mz; it.gx = gx; it.gy = gy;
            it.vec = vec ? 1 : 0;
            b.first[b.count + 1] = b.first[b.count] + gy * gz;
            ++b.count;
            smem = std::max(smem, need);
        }
    }
    return flush();
}

}  // namespace

// Validation shared by the slicemap builder and the renderer.
int check_slicemap(const mctp_slicemap *sm)
{
    if (!sm) return MCTP_EINVAL;
    int rc = check_type(sm->dtype, sm->bits);
    if (rc != MCTP_OK) return rc;
    if (sm->nlevels < 1 || sm->nlevels > MCTP_MAX_LEVELS) return MCTP_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (sm->src_dims[a] < 1 || sm->src_dims[a] > (int64_t(1) << 31)) return MCTP_EINVAL;
    for (int k = 0; k < sm->nlevels; ++k) {
        for (int a = 0; a < 3; ++a) {
            if (sm->dims[k][a] < 1) return MCTP_EINVAL;
            if (k == 0 && sm->dims[0][a] > sm->src_dims[a]) return MCTP_EINVAL;
            if (k > 0 && 2 * sm->dims[k][a] != sm->dims[k - 1][a]) return MCTP_EINVAL;
        }
        if (!sm->atlas[k] || sm->tiles_x[k] < 1 || sm->tiles_y[k] < 1) return MCTP_EINVAL;
        if (int64_t(sm->tiles_x[k]) * sm->tiles_y[k] < sm->dims[k][2]) return MCTP_ESIZE;
        if (int64_t(sm->tiles_x[k]) * sm->dims[k][0] > (int64_t(1) << 31) ||
            int64_t(sm->tiles_y[k]) * sm->dims[k][1] > (int64_t(1) << 31))
            return MCTP_ESIZE;
    }
    return MCTP_OK;
}

MCTP_FAULT_READER(slicemap)

}  // namespace mctp

namespace mctp {
namespace {
constexpr int kForks = 2;
struct Forks {
    int device = -1;
    cudaStream_t stream[kForks] = {};
    cudaEvent_t ev[kForks + 1] = {};
};

// This host thread's fork streams and events for the current device, made on
// first use (nullptr when they cannot be made).
Forks *thread_forks()
{
    thread_local Forks f[8];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 8) return nullptr;
    Forks &k = f[dev];
    if (k.device == dev) return &k;
    bool ok = true;
    for (int j = 0; j < kForks && ok; ++j)
        ok = cudaStreamCreateWithFlags(&k.stream[j], cudaStreamNonBlocking) == cudaSuccess;
    for (int j = 0; j <= kForks && ok; ++j) ok = cudaEventCreateWithFlags(&k.ev[j], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        for (int j = 0; j < kForks; ++j)
            if (k.stream[j]) cudaStreamDestroy(k.stream[j]);
        for (int j = 0; j <= kForks; ++j)
            if (k.ev[j]) cudaEventDestroy(k.ev[j]);
        k = Forks{};
        return nullptr;
    }
    k.device = dev;
    return &k;
}

int check_build(const void *vol, const mctp_volume_desc *d, const uint8_t *keep_lut, int32_t nbins,
                const mctp_slicemap *sm)
{
    int rc = check_desc(d);
    if (rc != MCTP_OK) return rc;
    rc = check_slicemap(sm);
    if (rc != MCTP_OK) return rc;
    if (!vol) return MCTP_EINVAL;
    if (sm->dtype != d->dtype || sm->bits != d->bits || sm->src_dims[0] != d->nx || sm->src_dims[1] != d->ny ||
        sm->src_dims[2] != d->nz)
        return MCTP_EINVAL;
    if (keep_lut && bin_shift(d->bits, nbins) < 0) return MCTP_EINVAL;
    // every footprint sum must fit in 32 bits
    int64_t fp = 1;
    const int64_t n3[3] = {d->nx, d->ny, d->nz};
    for (int a = 0; a < 3; ++a) fp *= (n3[a] + sm->dims[0][a] - 1) / sm->dims[0][a];
    if (fp * ((int64_t(1) << d->bits) - 1) >= (int64_t(1) << 32)) return MCTP_EUNSUPPORTED;
    return MCTP_OK;
}
}  // namespace
}  // namespace mctp

extern "C" int mctp_build_slicemap(const void *vol, const mctp_volume_desc *d, const uint8_t *keep_lut,
                                   int32_t nbins, const mctp_slicemap *sm, void *stream)
{
    using namespace mctp;
    const int rc = check_build(vol, d, keep_lut, nbins, sm);
    if (rc != MCTP_OK) return rc;
    cudaStream_t s = as_stream(stream);
    if (d->dtype == MCTP_U8)
        return launch_slicemap(static_cast<const uint8_t *>(vol), d, keep_lut, nbins, sm, s);
    return launch_slicemap(static_cast<const uint16_t *>(vol), d, keep_lut, nbins, sm, s);
}

extern "C" int mctp_build_slicemap_batch(const void *const *vols, const mctp_volume_desc *descs,
                                         const uint8_t *keep_luts, int32_t nbins, const mctp_slicemap *sms,
                                         int32_t count, void *stream)
{
    using namespace mctp;
    if (count < 0 || (count > 0 && (!vols || !descs || !sms))) return MCTP_EINVAL;
    if (count == 0) return MCTP_OK;
    if (keep_luts && (nbins < 1 || int64_t(count) * nbins > (int64_t(1) << 40))) return MCTP_EINVAL;
    for (int i = 0; i < count; ++i) {
        const int rc = check_build(vols[i], &descs[i], keep_luts ? keep_luts + int64_t(i) * nbins : nullptr, nbins,
                                   &sms[i]);
        if (rc != MCTP_OK) return rc;
        if (descs[i].dtype != descs[0].dtype) return MCTP_EINVAL;
    }
    cudaStream_t s = as_stream(stream);
    // The level-0 builds go round-robin to `s` and two streams forked from it,
    // so that one build's last blocks overlap the next build's first ones; the
    // forks join `s` again before the max grids (a capture into a CUDA graph
    // records the same fork and join).  The fork streams and events are made
    // once per host thread and device and kept; without them the builds stay
    // on `s`.
    Forks *fk = count > 1 ? thread_forks() : nullptr;
    if (fk && cudaEventRecord(fk->ev[0], s) != cudaSuccess) {
        // handles from a context that no longer exists: make new ones next time
        cudaGetLastError();
        *fk = Forks{};
        fk = nullptr;
    }
    const int nlanes = fk ? kForks + 1 : 1;
    cudaStream_t lanes[kForks + 1] = {s};
    int rc = MCTP_OK;
    if (fk) {
        for (int j = 0; j < kForks; ++j) lanes[j + 1] = fk->stream[j];
        for (int j = 1; j < nlanes && rc == MCTP_OK; ++j)
            if (cudaStreamWaitEvent(lanes[j], fk->ev[0], 0) != cudaSuccess) rc = MCTP_ECUDA;
    }
    for (int i = 0; i < count && rc == MCTP_OK; ++i) {
        const uint8_t *keep = keep_luts ? keep_luts + int64_t(i) * nbins : nullptr;
        cudaStream_t li = lanes[i % nlanes];
        rc = descs[i].dtype == MCTP_U8
                 ? launch_slicemap(static_cast<const uint8_t *>(vols[i]), &descs[i], keep, nbins, &sms[i], li, false)
                 : launch_slicemap(static_cast<const uint16_t *>(vols[i]), &descs[i], keep, nbins, &sms[i], li, false);
    }
    // join the forks (also after an error, so that no fork is left outside s)
    for (int j = 1; j < nlanes; ++j) {
        if (cudaEventRecord(fk->ev[j], lanes[j]) != cudaSuccess || cudaStreamWaitEvent(s, fk->ev[j], 0) != cudaSuccess)
            rc = MCTP_ECUDA;
    }
    if (rc != MCTP_OK) return rc;
    return descs[0].dtype == MCTP_U8 ? launch_maxgrid_batch<uint8_t>(sms, count, s)
                                     : launch_maxgrid_batch<uint16_t>(sms, count, s);
}
