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
// the kernel, at most 2), so the source is read from HBM exactly once:
//  * accumulate: for each level-0 row, every thread owns 16-byte column
//    vectors of the source rows of that row's (z, y) footprint and sums them
//    in registers (8 loads in flight), then stores the column sums to a
//    double-buffered shared row;
//  * x-reduce: threads sum each output voxel's x-footprint from shared
//    memory, divide, write the level-0 atlas row and keep the value in shared
//    memory;
//  * after the group: levels 1..f from shared memory.
// Remaining levels (f < nlevels - 1) run as a separate 2x2x2 kernel.
// When the keep table is a step (keep[b] = b >= T, as Otsu, ITS and explicit
// thresholds produce) the per-voxel table lookup becomes one comparison.
#include <algorithm>

#include "mctp_internal.cuh"

namespace mctp {
namespace {

constexpr int kSmThreads = 256;
constexpr int kSmUnroll = 8;
constexpr int kMaxFused = 2;

template <typename T>
struct L0Args {
    const T *vol;
    int64_t nx, ny, nz;
    int32_t mx, my, mz;
    int32_t fused;              // extra levels produced in-kernel (0..2)
    T *atlas[kMaxFused + 1];
    int32_t tiles_x[kMaxFused + 1];
    int64_t pitch[kMaxFused + 1];  // atlas row pitch in elements
    const uint8_t *keep;        // nullptr: no filtering
    int32_t nbins;
    int32_t shift;
    uint32_t limit;             // 2^bits
};

// Keep/discard of one grey value: 0 = no table, 1 = table lookup, 2 = step.
template <int kMode>
__device__ __forceinline__ uint32_t kept(uint32_t v, const uint8_t *lut, int shift, uint32_t limit,
                                         uint32_t lo)
{
    if (kMode == 0) return v;
    if (kMode == 2) return (v - lo) < (limit - lo) ? v : 0u;
    return (v < limit && lut[v >> shift]) ? v : 0u;
}

template <typename T>
__device__ __forceinline__ T *atlas_ptr(T *atlas, int64_t pitch, int tiles_x, int m_x, int m_y, int x, int y,
                                        int z)
{
    const int row = z / tiles_x, col = z - (z / tiles_x) * tiles_x;
    return atlas + (int64_t(row) * m_y + y) * pitch + int64_t(col) * m_x + x;
}

// Column sums of one level-0 row, vector path (rows 16-byte aligned).
template <typename T, int kMode>
__device__ __forceinline__ void accumulate_row_vec(const L0Args<T> &a, int64_t zlo, int64_t zhi, int64_t ylo,
                                                   int64_t yhi, uint32_t *colsum, const uint8_t *lut,
                                                   uint32_t lo)
{
    constexpr int E = 16 / sizeof(T);
    const int64_t V = a.nx / E;
    const int wy = int(yhi - ylo);
    const int R = int(zhi - zlo) * wy;
    const int64_t row_bytes = a.nx * int64_t(sizeof(T));
    // source rows of the footprint in (z, y) order: step one row, or jump to
    // the first footprint row of the next slice
    const int64_t slice_jump = (a.ny - wy + 1) * row_bytes;
    const char *first = reinterpret_cast<const char *>(a.vol) + (zlo * a.ny + ylo) * row_bytes;
    for (int64_t v = threadIdx.x; v < V; v += blockDim.x) {
        uint32_t sum[E];
#pragma unroll
        for (int e = 0; e < E; ++e) sum[e] = 0u;
        const char *p = first + v * 16;
        int yi = 0;
        for (int r0 = 0; r0 < R; r0 += kSmUnroll) {
            uint4 q[kSmUnroll];
#pragma unroll
            for (int u = 0; u < kSmUnroll; ++u) {
                if (r0 + u < R) {
                    q[u] = ld_stream_v4(p);
                    if (++yi == wy) { yi = 0; p += slice_jump; }
                    else p += row_bytes;
                } else {
                    q[u] = make_uint4(0u, 0u, 0u, 0u);
                }
            }
#pragma unroll
            for (int u = 0; u < kSmUnroll; ++u) {
                const uint32_t w[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (sizeof(T) == 1) {
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            sum[4 * k + b] += kept<kMode>((w[k] >> (8 * b)) & 0xffu, lut, a.shift, a.limit, lo);
                    } else {
                        sum[2 * k] += kept<kMode>(w[k] & 0xffffu, lut, a.shift, a.limit, lo);
                        sum[2 * k + 1] += kept<kMode>(w[k] >> 16, lut, a.shift, a.limit, lo);
                    }
                }
            }
        }
        uint32_t *dst = colsum + v * E;
#pragma unroll
        for (int e = 0; e < E; e += 4) *reinterpret_cast<uint4 *>(dst + e) = make_uint4(sum[e], sum[e + 1], sum[e + 2], sum[e + 3]);
    }
}

// Column sums of one level-0 row, scalar path (any alignment).
template <typename T, int kMode>
__device__ __forceinline__ void accumulate_row_scalar(const L0Args<T> &a, int64_t zlo, int64_t zhi, int64_t ylo,
                                                      int64_t yhi, uint32_t *colsum, const uint8_t *lut,
                                                      uint32_t lo)
{
    for (int64_t x = threadIdx.x; x < a.nx; x += blockDim.x) {
        uint32_t s = 0;
        for (int64_t z = zlo; z < zhi; ++z)
            for (int64_t y = ylo; y < yhi; ++y)
                s += kept<kMode>(__ldg(a.vol + (z * a.ny + y) * a.nx + x), lut, a.shift, a.limit, lo);
        colsum[x] = s;
    }
}

template <typename T, bool kVec, int kMode>
__device__ void level0_group(const L0Args<T> &a, int Z0, int Y0, int gz, int gy, uint32_t *colsum, uint32_t *grp,
                             const uint8_t *lut, uint32_t lo)
{
    const int G = gz * gy;
    for (int g = 0; g < G; ++g) {
        const int zo = Z0 + g / gy, yo = Y0 + g % gy;
        const int64_t zlo = (int64_t(zo) * a.nz) / a.mz, zhi = (int64_t(zo + 1) * a.nz) / a.mz;
        const int64_t ylo = (int64_t(yo) * a.ny) / a.my, yhi = (int64_t(yo + 1) * a.ny) / a.my;
        uint32_t *cs = colsum + (g & 1) * a.nx;
        if (kVec) accumulate_row_vec<T, kMode>(a, zlo, zhi, ylo, yhi, cs, lut, lo);
        else accumulate_row_scalar<T, kMode>(a, zlo, zhi, ylo, yhi, cs, lut, lo);
        __syncthreads();
        const uint32_t R = uint32_t((zhi - zlo) * (yhi - ylo));
        T *row = atlas_ptr(a.atlas[0], a.pitch[0], a.tiles_x[0], a.mx, a.my, 0, yo, zo);
        for (int x = threadIdx.x; x < a.mx; x += blockDim.x) {
            const int64_t xlo = (int64_t(x) * a.nx) / a.mx, xhi = (int64_t(x + 1) * a.nx) / a.mx;
            uint32_t s = 0;
            for (int64_t i = xlo; i < xhi; ++i) s += cs[i];
            const uint32_t cnt = uint32_t(xhi - xlo) * R;
            const uint32_t val = (s + cnt / 2u) / cnt;
            row[x] = (T)val;
            if (grp) grp[g * a.mx + x] = val;
        }
        // no barrier: the next row accumulates into the other buffer, and the
        // barrier after it orders this row's reads before that buffer's reuse
    }
}

template <typename T, bool kVec>
__global__ void __launch_bounds__(kSmThreads) slicemap_level0_kernel(L0Args<T> a)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int gz = 1 << a.fused, gy = 1 << a.fused;
    const int ngy = a.my / gy;
    const int Z0 = (blockIdx.x / ngy) * gz, Y0 = (blockIdx.x % ngy) * gy;

    uint32_t *colsum = reinterpret_cast<uint32_t *>(smem);              // 2 * nx
    uint32_t *grp = colsum + 2 * a.nx;                                   // gz*gy*mx (when fused)
    uint32_t *grp1 = grp + (a.fused ? gz * gy * a.mx : 0);              // (gz/2)(gy/2)(mx/2)
    uint8_t *lut = reinterpret_cast<uint8_t *>(grp1 + (a.fused > 1 ? (gz / 2) * (gy / 2) * (a.mx / 2) : 0));

    __shared__ int sh_first, sh_violation;
    int mode = 0;
    uint32_t lo = 0;
    if (a.keep) {
        if (threadIdx.x == 0) { sh_first = a.nbins; sh_violation = 0; }
        for (int b = threadIdx.x; b < a.nbins; b += blockDim.x) lut[b] = a.keep[b];
        __syncthreads();
        for (int b = threadIdx.x; b < a.nbins; b += blockDim.x)
            if (lut[b]) atomicMin(&sh_first, b);
        __syncthreads();
        for (int b = threadIdx.x; b < a.nbins; b += blockDim.x)
            if (b >= sh_first && !lut[b]) sh_violation = 1;
        __syncthreads();
        if (sh_violation) {
            mode = 1;
        } else {
            mode = 2;
            const uint64_t l = uint64_t(sh_first) << a.shift;
            lo = l >= a.limit ? a.limit : uint32_t(l);
        }
    }
    uint32_t *g0 = a.fused ? grp : nullptr;
    if (mode == 0) level0_group<T, kVec, 0>(a, Z0, Y0, gz, gy, colsum, g0, lut, lo);
    else if (mode == 1) level0_group<T, kVec, 1>(a, Z0, Y0, gz, gy, colsum, g0, lut, lo);
    else level0_group<T, kVec, 2>(a, Z0, Y0, gz, gy, colsum, g0, lut, lo);
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
                    const uint32_t *src = grp + ((2 * c + dz) * gy + (2 * b + dy)) * a.mx + 2 * x;
                    s += src[0] + src[1];
                }
            const uint32_t val = (s + 4u) / 8u;
            *atlas_ptr(a.atlas[1], a.pitch[1], a.tiles_x[1], hx, my1, x, Y0 / 2 + b, Z0 / 2 + c) = (T)val;
            if (a.fused > 1) grp1[(c * hy + b) * hx + x] = val;
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
                    const uint32_t *src = grp1 + ((2 * c + dz) * gy1 + (2 * b + dy)) * mx1 + 2 * x;
                    s += src[0] + src[1];
                }
            *atlas_ptr(a.atlas[2], a.pitch[2], a.tiles_x[2], hx, my2, x, Y0 / 4 + b, Z0 / 4 + c) =
                (T)((s + 4u) / 8u);
        }
    }
}

// Level k+1 from level k, atlas to atlas: exact 2x2x2 mean, rounded half up.
template <typename T>
__global__ void __launch_bounds__(256) halve_kernel(const T *__restrict__ src, int64_t src_pitch, int src_tx, int mx,
                                                     int my, T *__restrict__ dst, int64_t dst_pitch, int dst_tx,
                                                     int64_t total)
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
        *atlas_ptr(dst, dst_pitch, dst_tx, hx, hy, x, y, z) = (T)((s + 4u) / 8u);
    }
}

// Per-cell maxima of a level (occupancy data for the renderer): cell c covers
// voxels [8c, 8c + 8] per axis, clamped.  One block per (cz, cy) row of
// cells: the 9 x 9 (y, z) atlas rows of the row are read coalesced and their
// column maxima kept in shared memory, then each cell takes the maximum of
// its 9 columns.
template <typename T>
__global__ void __launch_bounds__(256) maxgrid_kernel(const T *__restrict__ atlas, int64_t pitch, int tiles_x, int mx,
                                                      int my, int mz, uint16_t *__restrict__ grid, int gx, int gy)
{
    extern __shared__ uint32_t colmax[];
    const int cy = blockIdx.x % gy, cz = blockIdx.x / gy;
    const int c = MCTP_MAXGRID_CELL;
    for (int x = threadIdx.x; x < mx; x += blockDim.x) colmax[x] = 0u;
    const int z1 = min(cz * c + c, mz - 1), y1 = min(cy * c + c, my - 1);
    for (int z = cz * c; z <= z1; ++z)
        for (int y = cy * c; y <= y1; ++y) {
            const T *row = atlas_ptr(const_cast<T *>(atlas), pitch, tiles_x, mx, my, 0, y, z);
            for (int x = threadIdx.x; x < mx; x += blockDim.x) colmax[x] = max(colmax[x], uint32_t(__ldg(row + x)));
        }
    __syncthreads();
    for (int cx = threadIdx.x; cx < gx; cx += blockDim.x) {
        uint32_t m = 0;
        const int x1 = min(cx * c + c, mx - 1);
        for (int x = cx * c; x <= x1; ++x) m = max(m, colmax[x]);
        grid[(int64_t(cz) * gy + cy) * gx + cx] = uint16_t(m);
    }
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

template <typename T>
int launch_slicemap(const T *vol, const mctp_volume_desc *d, const uint8_t *keep, int nbins, const mctp_slicemap *sm,
                    cudaStream_t s)
{
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
    }
    a.keep = keep;
    a.nbins = keep ? nbins : 0;
    a.shift = keep ? bin_shift(d->bits, nbins) : 0;
    a.limit = d->bits >= 32 ? 0xffffffffu : (1u << d->bits);
    const int gz = 1 << fused, gy = 1 << fused;
    size_t smem = size_t(2) * a.nx * 4;
    if (fused) smem += size_t(gz) * gy * a.mx * 4;
    if (fused > 1) smem += size_t(gz / 2) * (gy / 2) * (a.mx / 2) * 4;
    smem += keep ? size_t(nbins) : 0;
    if (smem > 220 * 1024) return MCTP_EUNSUPPORTED;
    const bool vec = (reinterpret_cast<uintptr_t>(vol) & 15) == 0 && ((a.nx * int64_t(sizeof(T))) & 15) == 0;
    auto kern = vec ? slicemap_level0_kernel<T, true> : slicemap_level0_kernel<T, false>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return MCTP_ECUDA;
    const int64_t blocks = int64_t(a.mz / gz) * (a.my / gy);
    if (blocks > 0x7fffffff) return MCTP_EUNSUPPORTED;
    kern<<<unsigned(blocks), kSmThreads, smem, s>>>(a);
    int rc = launch_status();
    if (rc != MCTP_OK) return rc;
    for (int k = fused + 1; k < sm->nlevels; ++k) {
        const int mx = sm->dims[k - 1][0], my = sm->dims[k - 1][1];
        const int64_t total = int64_t(sm->dims[k][0]) * sm->dims[k][1] * sm->dims[k][2];
        const int64_t grid = std::min<int64_t>((total + 255) / 256, int64_t(num_sms()) * 16);
        halve_kernel<T><<<unsigned(std::max<int64_t>(grid, 1)), 256, 0, s>>>(
            static_cast<const T *>(sm->atlas[k - 1]), int64_t(sm->tiles_x[k - 1]) * mx, sm->tiles_x[k - 1], mx, my,
            static_cast<T *>(sm->atlas[k]), int64_t(sm->tiles_x[k]) * sm->dims[k][0], sm->tiles_x[k], total);
        rc = launch_status();
        if (rc != MCTP_OK) return rc;
    }
    for (int k = 0; k < sm->nlevels; ++k) {
        rc = zero_unused_tiles(sm->atlas[k], int(sizeof(T)), sm->dims[k][0], sm->dims[k][1], sm->dims[k][2],
                               sm->tiles_x[k], sm->tiles_y[k], s);
        if (rc != MCTP_OK) return rc;
    }
    for (int k = 0; k < sm->nlevels; ++k) {
        if (!sm->maxgrid[k]) continue;
        const int c = MCTP_MAXGRID_CELL;
        const int mx = sm->dims[k][0], my = sm->dims[k][1], mz = sm->dims[k][2];
        const int gx = (mx + c - 1) / c, gy = (my + c - 1) / c, gz = (mz + c - 1) / c;
        const size_t smem = size_t(mx) * sizeof(uint32_t);
        if (smem > 200 * 1024) return MCTP_EUNSUPPORTED;
        if (smem > 48 * 1024 && cudaFuncSetAttribute(maxgrid_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     int(smem)) != cudaSuccess)
            return MCTP_ECUDA;
        maxgrid_kernel<T><<<unsigned(int64_t(gy) * gz), 256, smem, s>>>(
            static_cast<const T *>(sm->atlas[k]), int64_t(sm->tiles_x[k]) * mx, sm->tiles_x[k], mx, my, mz,
            static_cast<uint16_t *>(sm->maxgrid[k]), gx, gy);
        rc = launch_status();
        if (rc != MCTP_OK) return rc;
    }
    return MCTP_OK;
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

}  // namespace mctp

extern "C" int mctp_build_slicemap(const void *vol, const mctp_volume_desc *d, const uint8_t *keep_lut,
                                   int32_t nbins, const mctp_slicemap *sm, void *stream)
{
    using namespace mctp;
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
    cudaStream_t s = as_stream(stream);
    if (d->dtype == MCTP_U8)
        return launch_slicemap(static_cast<const uint8_t *>(vol), d, keep_lut, nbins, sm, s);
    return launch_slicemap(static_cast<const uint16_t *>(vol), d, keep_lut, nbins, sm, s);
}
