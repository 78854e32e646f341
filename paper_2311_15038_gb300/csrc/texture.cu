// texture.cu -- a slicemap level's atlas as a 2D texture (Sec. III-B/C: the
// paper's client uploads every atlas as a 2D texture and samples it there).
//
// The atlas is copied into a 2D CUDA array made for texture gathers, with a
// texture object that reads the stored integers as they are (point
// sampling, coordinates in texels, clamped at the edges).  The batched
// renderer then fetches the 2x2 in-slice corners of a sample with one gather
// per slice; the gathered integers are the atlas values, so the
// interpolation that follows is the same arithmetic on the same inputs.
#include "mctp_internal.cuh"

namespace mctp {
int check_slicemap(const mctp_slicemap *sm);
}

struct mctp_atlas_texture {
    cudaArray_t array = nullptr;
    cudaTextureObject_t tex = 0;
    cudaSurfaceObject_t surf = 0;   // 0: the array takes no surface stores; updates use a 2D copy
    int64_t width = 0, height = 0;  // texels
    int32_t dtype = 0;
};

namespace {

constexpr int kSurfThreads = 256;

// Row y of the atlas into the array.  Each warp moves 32 16-byte vectors:
// coalesced loads into shared memory, then one surface store per texel with
// the lanes on consecutive texels, so a warp's stores cover one contiguous
// run of the row.  Rows hold a whole number of 16-byte vectors.
template <typename T>
__global__ void __launch_bounds__(kSurfThreads) atlas_surface_kernel(const T *__restrict__ atlas, int32_t w,
                                                                     cudaSurfaceObject_t surf)
{
    constexpr int E = 16 / int(sizeof(T));
    __shared__ __align__(16) uint4 stage[kSurfThreads];
    const int y = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint4 *row = reinterpret_cast<const uint4 *>(atlas + int64_t(y) * w);
    const int nvec = w / E;
    const int nchunks = (nvec + 31) / 32;
    const T *mine = reinterpret_cast<const T *>(stage + warp * 32);
    for (int c = blockIdx.x * (kSurfThreads / 32) + warp; c < nchunks; c += gridDim.x * (kSurfThreads / 32)) {
        const int v = c * 32 + lane;
        if (v < nvec) stage[warp * 32 + lane] = __ldg(row + v);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < E; ++k) {
            const int t = k * 32 + lane;
            const int x = c * 32 * E + t;
            if (x < w) surf2Dwrite<T>(mine[t], surf, x * int(sizeof(T)), y, cudaBoundaryModeZero);
        }
        __syncwarp();
    }
}

int texture_geometry(const mctp_slicemap *sm, int32_t level, int64_t &w, int64_t &h)
{
    const int rc = mctp::check_slicemap(sm);
    if (rc != MCTP_OK) return rc;
    if (level < 0 || level >= sm->nlevels) return MCTP_EINVAL;
    w = int64_t(sm->tiles_x[level]) * sm->dims[level][0];
    h = int64_t(sm->tiles_y[level]) * sm->dims[level][1];
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
    // surface stores for the update kernel where the array allows them, else 2D copies
    const bool vec_rows = (w * mctp::elem_size(sm->dtype)) % 16 == 0;
    if (!vec_rows ||
        cudaMallocArray(&t->array, &cd, size_t(w), size_t(h), cudaArrayTextureGather | cudaArraySurfaceLoadStore) !=
            cudaSuccess) {
        cudaGetLastError();
        t->array = nullptr;
        if (cudaMallocArray(&t->array, &cd, size_t(w), size_t(h), cudaArrayTextureGather) != cudaSuccess) {
            delete t;
            return MCTP_ECUDA;
        }
    }
    cudaResourceDesc rd{};
    rd.resType = cudaResourceTypeArray;
    rd.res.array.array = t->array;
    unsigned int flags = 0;
    if (cudaArrayGetInfo(nullptr, nullptr, &flags, t->array) == cudaSuccess && (flags & cudaArraySurfaceLoadStore)) {
        if (cudaCreateSurfaceObject(&t->surf, &rd) != cudaSuccess) {
            cudaGetLastError();
            t->surf = 0;
        }
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

extern "C" int mctp_atlas_texture_update(mctp_atlas_texture *t, const mctp_slicemap *sm, int32_t level,
                                         void *stream)
{
    if (!t) return MCTP_EINVAL;
    int64_t w = 0, h = 0;
    const int rc = texture_geometry(sm, level, w, h);
    if (rc != MCTP_OK) return rc;
    if (w != t->width || h != t->height || sm->dtype != t->dtype) return MCTP_EINVAL;
    const size_t row = size_t(w) * size_t(mctp::elem_size(sm->dtype));
    cudaStream_t s = mctp::as_stream(stream);
    if (t->surf && (reinterpret_cast<uintptr_t>(sm->atlas[level]) & 15) == 0) {
        const int nchunks = int((row / 16 + 31) / 32);
        const int per_block = kSurfThreads / 32;
        const dim3 grid(unsigned((nchunks + per_block - 1) / per_block), unsigned(h));
        if (sm->dtype == MCTP_U8)
            atlas_surface_kernel<uint8_t>
                <<<grid, kSurfThreads, 0, s>>>(static_cast<const uint8_t *>(sm->atlas[level]), int32_t(w), t->surf);
        else
            atlas_surface_kernel<uint16_t>
                <<<grid, kSurfThreads, 0, s>>>(static_cast<const uint16_t *>(sm->atlas[level]), int32_t(w), t->surf);
        return mctp::launch_status();
    }
    if (cudaMemcpy2DToArrayAsync(t->array, 0, 0, sm->atlas[level], row, row, size_t(h), cudaMemcpyDeviceToDevice,
                                 s) != cudaSuccess)
        return MCTP_ECUDA;
    return MCTP_OK;
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
