// texture.cu -- a slicemap level's atlas as a 2D texture (Sec. III-B/C: the
// paper's client uploads every atlas as a 2D texture and samples it there).
//
// The atlas is copied into a 2D CUDA array made for texture gathers, with a
// texture object that reads the stored integers as they are (point
// sampling, coordinates in texels).  Each mx x my tile of the atlas sits in
// a cell of (mx + 2) x (my + 2) texels whose one-texel border repeats the
// tile's edge texels, so a gather whose 2x2 block reaches one texel past a
// tile's edge reads the edge value, which is what clamping the corner index
// to the level gives.  The batched renderer fetches the 2x2 in-slice corners
// of a sample with one gather per slice and no clamping or selection; the
// gathered integers are the atlas values, so the interpolation that follows
// is the same arithmetic on the same inputs.
#include <algorithm>

#include "mctp_internal.cuh"

namespace mctp {
int check_slicemap(const mctp_slicemap *sm);
}

struct mctp_atlas_texture {
    cudaArray_t array = nullptr;
    cudaTextureObject_t tex = 0;
    cudaSurfaceObject_t surf = 0;   // the update kernel's stores
    int64_t width = 0, height = 0;  // texels, with the one-texel border of every cell
    int32_t dtype = 0;
    int32_t mx = 0, my = 0, tiles_x = 0, tiles_y = 0;  // the level geometry at creation
};

namespace {

constexpr int kSurfThreads = 512;

// Rows Y0 .. Y0 + rows_per_block - 1 of a padded array (Y0 = block x
// rows_per_block; several short rows per block keep more loads in flight).
// The block stages each row's atlas row (the row ly of tile row `row`) in
// shared memory, with 16-byte loads when the row is 16-byte aligned, then
// writes the padded rows: texel X of cell (col, row) holds atlas texel
// (col mx + lx, ...) with lx = X - col (mx + 2) - 1 clamped to the tile.
// Consecutive threads store consecutive texels; the cell of X comes from a
// float estimate (X < 2^16 is exact) and one correction.
template <typename T>
__device__ __forceinline__ void pad_rows(const T *__restrict__ atlas, int64_t pitch, int32_t mx, int32_t my,
                                         int32_t width, cudaSurfaceObject_t surf, int32_t height,
                                         int32_t rows_per_block, int block, unsigned char *sh_row_bytes)
{
    constexpr int E = 16 / int(sizeof(T));
    const int Y0 = block * rows_per_block;
    const int nrows = min(rows_per_block, height - Y0);
    const int64_t stride = (pitch + E - 1) / E * E;  // staged row stride in elements (16-byte multiple)
    for (int k = 0; k < nrows; ++k) {
        const int Y = Y0 + k;
        T *sh_row = reinterpret_cast<T *>(sh_row_bytes) + k * stride;
        const int row = Y / (my + 2);
        const int ly = min(max(Y - row * (my + 2) - 1, 0), my - 1);
        const T *src = atlas + (int64_t(row) * my + ly) * pitch;
        if ((reinterpret_cast<uintptr_t>(src) & 15) == 0) {
            const uint4 *v = reinterpret_cast<const uint4 *>(src);
            const int nvec = int(pitch / E);
            for (int i = threadIdx.x; i < nvec; i += blockDim.x) reinterpret_cast<uint4 *>(sh_row)[i] = __ldg(v + i);
            for (int i = nvec * E + threadIdx.x; i < pitch; i += blockDim.x) sh_row[i] = __ldg(src + i);
        } else {
            for (int i = threadIdx.x; i < pitch; i += blockDim.x) sh_row[i] = __ldg(src + i);
        }
    }
    __syncthreads();
    const int cw = mx + 2;
    const float inv = 1.0f / float(cw);
    const T *sh = reinterpret_cast<const T *>(sh_row_bytes);
    const int st = int(stride);  // staged rows hold at most 200 KB
    for (int X = threadIdx.x; X < width; X += blockDim.x) {
        int col = int(float(X) * inv);
        if (col * cw > X) --col;
        else if ((col + 1) * cw <= X) ++col;
        const int src = col * mx + min(max(X - col * cw - 1, 0), mx - 1);
        surf2Dwrite<T>(sh[src], surf, X * int(sizeof(T)), Y0, cudaBoundaryModeZero);
        for (int k = 1; k < nrows; ++k)
            surf2Dwrite<T>(sh[k * st + src], surf, X * int(sizeof(T)), Y0 + k, cudaBoundaryModeZero);
    }
}

// Up to kPadBatch textures (of one element type) in one launch: item i owns
// blocks [first[i], first[i + 1]).
constexpr int kPadBatch = 64;
struct PadItem {
    const void *atlas;
    cudaSurfaceObject_t surf;
    int64_t pitch;
    int32_t mx, my, width, height, rows_per_block;
};
struct PadBatch {
    int32_t count;
    int32_t first[kPadBatch + 1];
    PadItem item[kPadBatch];
};

template <typename T>
__global__ void __launch_bounds__(kSurfThreads) atlas_pad_batch_kernel(const __grid_constant__ PadBatch b)
{
    extern __shared__ __align__(16) unsigned char sh_row_bytes[];
    int lo = 0, hi = b.count - 1;  // the item whose block range holds blockIdx.x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.first[mid] <= int(blockIdx.x)) lo = mid;
        else hi = mid - 1;
    }
    const PadItem &it = b.item[lo];
    pad_rows<T>(static_cast<const T *>(it.atlas), it.pitch, it.mx, it.my, it.width, it.surf, it.height,
                it.rows_per_block, int(blockIdx.x) - b.first[lo], sh_row_bytes);
}

// Rows per block for staged rows of row_bytes: 8 for short rows (<= 6 KB, launched
// with 256 threads), else up to 4 while they fit 48 KB.
int pad_rows_per_block(size_t row_bytes)
{
    return row_bytes <= 6 * 1024 ? 8 : int(std::max<size_t>(1, std::min<size_t>(4, (48 * 1024) / row_bytes)));
}

int texture_geometry(const mctp_slicemap *sm, int32_t level, int64_t &w, int64_t &h)
{
    const int rc = mctp::check_slicemap(sm);
    if (rc != MCTP_OK) return rc;
    if (level < 0 || level >= sm->nlevels) return MCTP_EINVAL;
    w = int64_t(sm->tiles_x[level]) * (sm->dims[level][0] + 2);
    h = int64_t(sm->tiles_y[level]) * (sm->dims[level][1] + 2);
    return MCTP_OK;
}

}  // namespace

extern "C" int mctp_atlas_texture_create(const mctp_slicemap *sm, int32_t level, mctp_atlas_texture **out,
                                         uint64_t *handle)
{
    if (!out || !handle) return MCTP_EINVAL;
    *out = nullptr;
    *handle = 0;
    int64_t w = 0, h = 0;
    int rc = texture_geometry(sm, level, w, h);
    if (rc != MCTP_OK) return rc;
    int dev = 0, gw = 0, gh = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MCTP_ECUDA;
    if (cudaDeviceGetAttribute(&gw, cudaDevAttrMaxTexture2DGatherWidth, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&gh, cudaDevAttrMaxTexture2DGatherHeight, dev) != cudaSuccess)
        return MCTP_ECUDA;
    // slice origins are packed as two 16-bit texel coordinates
    if (w > gw || h > gh || w > 65535 || h > 65535) return MCTP_ESIZE;
    const cudaChannelFormatDesc cd = sm->dtype == MCTP_U8 ? cudaCreateChannelDesc<unsigned char>()
                                                          : cudaCreateChannelDesc<unsigned short>();
    auto *t = new mctp_atlas_texture;
    t->width = w;
    t->height = h;
    t->dtype = sm->dtype;
    t->mx = sm->dims[level][0];
    t->my = sm->dims[level][1];
    t->tiles_x = sm->tiles_x[level];
    t->tiles_y = sm->tiles_y[level];
    // the update kernel writes the padded cells with surface stores
    if (cudaMallocArray(&t->array, &cd, size_t(w), size_t(h), cudaArrayTextureGather | cudaArraySurfaceLoadStore) !=
        cudaSuccess) {
        cudaGetLastError();
        delete t;
        return MCTP_ECUDA;
    }
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = t->array;
    if (cudaCreateSurfaceObject(&t->surf, &rd) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeArray(t->array);
        delete t;
        return MCTP_ECUDA;
    }
    cudaTextureDesc td{};
    td.addressMode[0] = cudaAddressModeClamp;
    td.addressMode[1] = cudaAddressModeClamp;
    td.filterMode = cudaFilterModePoint;
    td.readMode = cudaReadModeElementType;
    td.normalizedCoords = 0;
    if (cudaCreateTextureObject(&t->tex, &rd, &td, nullptr) != cudaSuccess) {
        if (t->surf) cudaDestroySurfaceObject(t->surf);
        cudaFreeArray(t->array);
        delete t;
        return MCTP_ECUDA;
    }
    *out = t;
    *handle = uint64_t(t->tex);
    return MCTP_OK;
}

namespace {
// The texture t was made for this level's geometry.
int check_update(const mctp_atlas_texture *t, const mctp_slicemap *sm, int32_t level)
{
    if (!t) return MCTP_EINVAL;
    int64_t w = 0, h = 0;
    const int rc = texture_geometry(sm, level, w, h);
    if (rc != MCTP_OK) return rc;
    if (w != t->width || h != t->height || sm->dtype != t->dtype || sm->dims[level][0] != t->mx ||
        sm->dims[level][1] != t->my || sm->tiles_x[level] != t->tiles_x || sm->tiles_y[level] != t->tiles_y)
        return MCTP_EINVAL;
    return MCTP_OK;
}

template <typename T>
int launch_pad_batch(const PadBatch &b, size_t smem, cudaStream_t s)
{
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(atlas_pad_batch_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) !=
            cudaSuccess)
        return MCTP_ECUDA;
    const int threads = b.item[0].rows_per_block >= 8 ? 256 : kSurfThreads;
    atlas_pad_batch_kernel<T><<<unsigned(b.first[b.count]), threads, smem, s>>>(b);
    return mctp::launch_status();
}
}  // namespace

extern "C" int mctp_atlas_texture_update(mctp_atlas_texture *t, const mctp_slicemap *sm, int32_t level,
                                         void *stream)
{
    return mctp_atlas_texture_update_batch(&t, sm, &level, 1, stream);
}

extern "C" int mctp_atlas_texture_update_batch(mctp_atlas_texture *const *textures, const mctp_slicemap *sms,
                                               const int32_t *levels, int32_t count, void *stream)
{
    if (count < 0 || (count > 0 && (!textures || !sms || !levels))) return MCTP_EINVAL;
    for (int i = 0; i < count; ++i) {
        const int rc = check_update(textures[i], &sms[i], levels[i]);
        if (rc != MCTP_OK) return rc;
        if (sms[i].dtype != sms[0].dtype) return MCTP_EINVAL;
    }
    if (count == 0) return MCTP_OK;
    cudaStream_t s = mctp::as_stream(stream);
    const bool u8 = sms[0].dtype == MCTP_U8;
    PadBatch b{};
    size_t smem = 0;
    auto flush = [&]() -> int {
        if (b.count == 0) return MCTP_OK;
        const int rc = u8 ? launch_pad_batch<uint8_t>(b, smem, s) : launch_pad_batch<uint16_t>(b, smem, s);
        b.count = 0;
        smem = 0;
        return rc;
    };
    for (int i = 0; i < count; ++i) {
        const mctp_slicemap &sm = sms[i];
        const int k = levels[i];
        const mctp_atlas_texture *t = textures[i];
        const int64_t pitch = int64_t(sm.tiles_x[k]) * sm.dims[k][0];
        const size_t row_bytes = (size_t(pitch) * size_t(mctp::elem_size(sm.dtype)) + 15) / 16 * 16;
        const int rpb = pad_rows_per_block(row_bytes);
        if (row_bytes * size_t(rpb) > 200 * 1024) return MCTP_ESIZE;
        const int64_t blocks = (t->height + rpb - 1) / rpb;
        if (b.count == kPadBatch || int64_t(b.first[b.count]) + blocks > 0x7fffffff) {
            const int rc = flush();
            if (rc != MCTP_OK) return rc;
        }
        PadItem &it = b.item[b.count];
        it.atlas = sm.atlas[k];
        it.surf = t->surf;
        it.pitch = pitch;
        it.mx = sm.dims[k][0];
        it.my = sm.dims[k][1];
        it.width = int32_t(t->width);
        it.height = int32_t(t->height);
        it.rows_per_block = rpb;
        b.first[b.count + 1] = b.first[b.count] + int32_t(blocks);
        ++b.count;
        smem = std::max(smem, row_bytes * size_t(rpb));
    }
    return flush();
}

extern "C" int mctp_atlas_texture_destroy(mctp_atlas_texture *t)
{
    if (!t) return MCTP_OK;
    int rc = MCTP_OK;
    if (t->tex && cudaDestroyTextureObject(t->tex) != cudaSuccess) rc = MCTP_ECUDA;
    if (t->surf && cudaDestroySurfaceObject(t->surf) != cudaSuccess) rc = MCTP_ECUDA;
    if (t->array && cudaFreeArray(t->array) != cudaSuccess) rc = MCTP_ECUDA;
    delete t;
    return rc;
}
