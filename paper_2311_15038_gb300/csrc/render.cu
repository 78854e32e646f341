// render.cu -- server-side rendering of slicemap views (Sec. III-C) in one
// call: orthographic emission-absorption ray marching, front to back, with
// trilinear sampling of a slicemap level, a 1D RGBA transfer function and
// early ray termination.  The per-ray march lives in render_common.cuh.
//
// Empty-space skipping: when the level has a max grid, every CTA turns it
// into a shared-memory bitmap of the cells that can produce a nonzero opacity
// under this call's transfer function (see render_common.cuh for why skipping
// them is exact).
//
// CTAs are persistent (one wave sized by occupancy) and walk the 16 x 16 pixel
// tiles of all views in order; a warp covers an 8 x 4 pixel sub-tile so its
// rays sample neighbouring texels together.
#include "render_common.cuh"

namespace mctp {

int check_slicemap(const mctp_slicemap *sm);

namespace {

using namespace render;

constexpr int kMaxViewsPerLaunch = 64;
constexpr int kRenderThreads = kTileW * kTileH;
constexpr int kMaxBitmapWords = 8192;  // 64^3 cells

struct LevelParams {
    const void *atlas;
    const uint16_t *maxgrid;  // nullptr: no skipping
    int32_t mx, my, mz;
    int32_t tiles_x;
    int32_t gx, gy, gz;       // max-grid cells per axis
    int32_t pad;
    int64_t pitch;            // elements per atlas row
};

struct RenderParams {
    int32_t nviews;
    int32_t nlut;
    float alpha_stop;
    float inv_vmax;  // 1 / (2^bits - 1)
    int32_t vmax_int;
    int32_t pad;
    int64_t total_tiles;
    int64_t out4_total;  // float4 pixels of the output (bounds of the checked build)
    const float4 *lut;
    float *out;
    unsigned long long *samples;
    LevelParams level[MCTP_MAX_LEVELS];
    ViewParams view[kMaxViewsPerLaunch];
};

template <typename T>
__global__ void __launch_bounds__(kRenderThreads, 3) render_kernel(const __grid_constant__ RenderParams P)
{
    extern __shared__ __align__(16) uint8_t smem[];
    float4 *lut = reinterpret_cast<float4 *>(smem);
    uint32_t *slice_off = reinterpret_cast<uint32_t *>(lut + P.nlut);
    __shared__ uint32_t occ[kMaxBitmapWords];
    __shared__ int sh_skip;

    for (int i = threadIdx.x; i < P.nlut; i += blockDim.x) lut[i] = P.lut[i];
    __syncthreads();
    if (threadIdx.x == 0) sh_skip = skip_threshold(lut, P.nlut, P.inv_vmax, P.vmax_int);
    __syncthreads();
    const int skip_S = sh_skip;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t taken = 0, evaluated = 0;  // the evaluated count is not reported by this renderer
    int v = 0, cur_level = -1;
    bool use_skip = false;
    LevelGeom G{};
    const SharedTables tab{lut, slice_off, occ};

    for (int64_t tile = blockIdx.x; tile < P.total_tiles; tile += gridDim.x) {
        while (v + 1 < P.nviews && tile >= P.view[v + 1].tile_begin) ++v;
        const ViewParams &V = P.view[v];
        const LevelParams &Lv = P.level[V.level];
        if (V.level != cur_level) {  // uniform across the CTA
            __syncthreads();
            cur_level = V.level;
            for (int z = threadIdx.x; z < Lv.mz; z += blockDim.x) {
                const int row = z / Lv.tiles_x, col = z - row * Lv.tiles_x;
                slice_off[z] = uint32_t(int64_t(row) * Lv.my * Lv.pitch + int64_t(col) * Lv.mx);
            }
            // occupancy bitmap, one bit per cell, rows of wpr words per (cz, cy)
            G.m1[0] = Lv.mx - 1;
            G.m1[1] = Lv.my - 1;
            G.m1[2] = Lv.mz - 1;
            G.pitch = uint32_t(Lv.pitch);
            G.wpr = (Lv.gx + 31) / 32;
            G.gy = Lv.gy;
            G.elems = Lv.pitch * ((Lv.mz + Lv.tiles_x - 1) / Lv.tiles_x) * Lv.my;
            const int nrows = Lv.gy * Lv.gz;
            use_skip = Lv.maxgrid != nullptr && skip_S >= 0 && int64_t(nrows) * G.wpr <= kMaxBitmapWords;
            if (use_skip)
                for (int w = threadIdx.x; w < nrows * G.wpr; w += blockDim.x)
                    occ[w] = occupancy_word(Lv.maxgrid, Lv.gx, G.wpr, w, skip_S);
            __syncthreads();
        }

        const int64_t t = tile - V.tile_begin;
        const int px = int(t % V.tiles_w) * kTileW + (warp & 1) * 8 + (lane & 7);
        const int py = int(t / V.tiles_w) * kTileH + (warp >> 1) * 4 + (lane >> 3);
        if (px >= V.W || py >= V.H) continue;
        const float4 acc = march_ray<T>(V, static_cast<const T *>(Lv.atlas), G, use_skip, tab, P.nlut,
                                        P.inv_vmax, P.alpha_stop, px, py, taken, evaluated);
        const int64_t pix = V.out_offset / 4 + int64_t(py) * V.W + px;
        if (in_range(pix, P.out4_total, kFaultImageWrite)) reinterpret_cast<float4 *>(P.out)[pix] = acc;
        flush_count(taken, P.samples);
        evaluated = 0;
    }
    warp_add_count(taken, P.samples);
}

}  // namespace

MCTP_FAULT_READER(render)

}  // namespace mctp

extern "C" int mctp_render_views(const mctp_slicemap *sm, const mctp_view *views, int32_t nviews,
                                 const float *lut_rgba, int32_t nlut, float alpha_stop, float *out_rgba,
                                 uint64_t *samples_taken, void *stream)
{
    using namespace mctp;
    using namespace mctp::render;
    int rc = check_slicemap(sm);
    if (rc != MCTP_OK) return rc;
    if (!views || nviews < 0 || !lut_rgba || !out_rgba) return MCTP_EINVAL;
    if (nlut < 2 || nlut > kMaxLut) return MCTP_EINVAL;
    if (!(alpha_stop > 0.0f && alpha_stop <= 1.0f)) return MCTP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(lut_rgba) & 15) || (reinterpret_cast<uintptr_t>(out_rgba) & 15))
        return MCTP_EINVAL;
    for (int i = 0; i < nviews; ++i) {
        rc = check_view(views[i], sm->nlevels);
        if (rc != MCTP_OK) return rc;
    }
    cudaStream_t s = as_stream(stream);
    if (samples_taken && cudaMemsetAsync(samples_taken, 0, sizeof(uint64_t), s) != cudaSuccess) return MCTP_ECUDA;
    if (nviews == 0) return MCTP_OK;

    RenderParams P{};  // copied into each launch's parameter buffer
    P.nlut = nlut;
    P.alpha_stop = alpha_stop;
    P.inv_vmax = float(1.0 / double((1u << sm->bits) - 1u));
    P.vmax_int = int((1u << sm->bits) - 1u);
    P.lut = reinterpret_cast<const float4 *>(lut_rgba);
    P.samples = reinterpret_cast<unsigned long long *>(samples_taken);
    int max_mz = 1;
    for (int k = 0; k < sm->nlevels; ++k) {
        LevelParams &L = P.level[k];
        L.atlas = sm->atlas[k];
        L.maxgrid = static_cast<const uint16_t *>(sm->maxgrid[k]);
        L.mx = sm->dims[k][0];
        L.my = sm->dims[k][1];
        L.mz = sm->dims[k][2];
        L.tiles_x = sm->tiles_x[k];
        const int c = MCTP_MAXGRID_CELL;
        L.gx = (L.mx + c - 1) / c;
        L.gy = (L.my + c - 1) / c;
        L.gz = (L.mz + c - 1) / c;
        L.pitch = int64_t(sm->tiles_x[k]) * sm->dims[k][0];
        if (!level_fits_32bit(sm, k)) return MCTP_ESIZE;  // texel offsets are 32-bit
        max_mz = std::max(max_mz, sm->dims[k][2]);
    }
    if (max_mz > 16384) return MCTP_ESIZE;
    const size_t smem = size_t(nlut) * sizeof(float4) + size_t(max_mz) * sizeof(uint32_t);
    auto kern = sm->dtype == MCTP_U8 ? render_kernel<uint8_t> : render_kernel<uint16_t>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return MCTP_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRenderThreads, smem) != cudaSuccess)
        return MCTP_ECUDA;
    per_sm = std::max(per_sm, 1);

    int64_t out_off = 0;
    P.out4_total = 0;
    for (int i = 0; i < nviews; ++i) P.out4_total += int64_t(views[i].width) * views[i].height;
    for (int first = 0; first < nviews; first += kMaxViewsPerLaunch) {
        const int cnt = std::min(kMaxViewsPerLaunch, nviews - first);
        int64_t tiles = 0;
        for (int i = 0; i < cnt; ++i) {
            const mctp_view &w = views[first + i];
            ViewParams &V = P.view[i];
            fill_view(sm, w, V);
            V.out_offset = out_off;
            V.tile_begin = tiles;
            tiles += int64_t(V.tiles_w) * ((w.height + kTileH - 1) / kTileH);
            out_off += int64_t(w.width) * w.height * 4;
        }
        P.nviews = cnt;
        P.total_tiles = tiles;
        P.out = out_rgba;
        const int64_t grid = std::min<int64_t>(tiles, int64_t(per_sm) * num_sms());
        kern<<<unsigned(grid), kRenderThreads, smem, s>>>(P);
        rc = launch_status();
        if (rc != MCTP_OK) return rc;
    }
    return MCTP_OK;
}
