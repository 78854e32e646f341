// render_batch.cu -- many views of many slicemaps in one persistent launch.
//
// A batch mixes slicemaps of any sizes, levels and transfer functions.  Work
// is a queue of warp tiles (32 rays: warp_w x 32/warp_w pixels) over all views
// in order; every warp takes `chunk` consecutive warp tiles at a time with one
// atomic add on a counter (issued one grab ahead), so no warp idles while
// others still march long rays, and there is one tail for the whole batch
// rather than one per view.
// Eight warp tiles form a super tile of about 16 x 16 pixels, so consecutive
// grabs stay close together in the image and share texels in L1/L2.
//
// Per-view constants and per-(slicemap, level, transfer function) tables
// (slice offsets of the atlas, the cell bitmap for empty-space skipping) are
// built once per call into a caller-provided device workspace by small
// set-up kernels, and read by the march through the read-only cache.
//
// Depth bounds: a set-up kernel projects every marked cell of a view's level
// into the view's image and records, per 16 x 16 pixel tile, the least and
// greatest depth along the rays at which a marked cell lies.  A ray marches
// only the samples between those depths (its first and last samples that can
// reach a marked cell, with a margin); the samples before and after lie in
// unmarked cells and add exactly nothing, so images and sample counts do not
// change, while rays that meet no marked cell take no step at all.  The
// march itself is the one of the single-call renderer (render_common.cuh), so
// a view's image and sample count are bit-identical to rendering it alone.
//
// Every step is a kernel launch or a memset on the caller's stream, so a call
// can be captured in a CUDA graph.
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "render_common.cuh"

namespace mctp {

int check_slicemap(const mctp_slicemap *sm);

namespace {

using namespace render;

constexpr int kBatchThreads = 256;
constexpr int kUploadViews = 128;
constexpr int kPrepPairs = 256;
constexpr size_t kLutSmemMax = 48 * 1024;  // all transfer functions go to shared memory up to this size
constexpr size_t kAlign = 256;
constexpr int kBoundsTile = 16;  // pixels per side of a depth-bounds tile

// One (slicemap, level, transfer function) combination used by the batch.
struct BatchPair {
    const void *atlas;
    uint64_t tex;             // atlas texture (0: loads from the atlas)
    const uint16_t *maxgrid;  // nullptr: no skipping
    uint32_t *slice_off;      // workspace: atlas offset of each slice
    uint32_t *occ;            // workspace: cell bitmap (when maxgrid is set)
    int32_t mx, my, mz, tiles_x;
    int32_t gx, gy, gz, wpr;
    int64_t pitch;
    int32_t lut;              // transfer-function index
    int32_t use_skip;         // filled by the set-up kernel
    float inv_vmax;
    int32_t vmax_int;
};

struct BatchView {
    ViewParams vp;
    int32_t pair;
    int32_t stiles_x;       // super tiles along x
    uint32_t item_begin;    // first warp tile of this view in the queue
    uint32_t bounds_begin;  // first depth-bounds tile of this view
    int32_t btiles_x;       // depth-bounds tiles along x
    int32_t pad;
};

struct UploadArgs {
    BatchView *dst;
    uint32_t *item_begin;
    int32_t first, count;
    uint32_t total_items;
    int32_t last;  // this launch carries the final view
    BatchView view[kUploadViews];
};

struct PrepArgs {
    BatchPair *dst;
    const float4 *luts;
    int32_t first, count;
    int32_t nlut;
    int32_t pad;
    BatchPair pair[kPrepPairs];
};

struct BatchArgs {
    const BatchView *views;
    const uint32_t *item_begin;  // nviews + 1 entries
    const BatchPair *pairs;
    const float4 *luts;
    float *out;
    unsigned long long *samples;
    unsigned int *counter;                  // the queue counter (workspace bytes 64..67)
    unsigned long long *counter_evaluated;  // workspace bytes 8..15
    const uint32_t *bounds_lo, *bounds_hi;  // per depth-bounds tile; nullptr: no bounds
    int32_t nviews, nlut, nluts;
    uint32_t total_items;
    int32_t wx_log2;  // log2 warp_w
    int32_t chunk;
    float alpha_stop;
    int64_t out4_total;  // float4 pixels the output buffer holds (bounds of the checked build)
};

__global__ void __launch_bounds__(kBatchThreads) batch_upload_kernel(const __grid_constant__ UploadArgs A)
{
    static_assert(sizeof(BatchView) % 4 == 0, "word copy");
    static_assert(sizeof(PrepArgs) <= 32000 && sizeof(UploadArgs) <= 32000, "kernel parameter space");
    const uint32_t *src = reinterpret_cast<const uint32_t *>(A.view);
    uint32_t *dst = reinterpret_cast<uint32_t *>(A.dst + A.first);
    const int nw = A.count * int(sizeof(BatchView) / 4);
    for (int i = threadIdx.x; i < nw; i += blockDim.x) dst[i] = src[i];
    for (int i = threadIdx.x; i < A.count; i += blockDim.x) A.item_begin[A.first + i] = A.view[i].item_begin;
    if (A.last && threadIdx.x == 0) A.item_begin[A.first + A.count] = A.total_items;
}

// Block (p, y): part y of pair p's slice-offset table and cell bitmap; block
// (p, 0) also writes the pair's record.
__global__ void __launch_bounds__(kBatchThreads) batch_prep_kernel(const __grid_constant__ PrepArgs A)
{
    const BatchPair &p = A.pair[blockIdx.x];
    __shared__ int sh_first;
    __shared__ int sh_S;
    if (threadIdx.x == 0) sh_first = A.nlut;
    __syncthreads();
    const float4 *lut = A.luts + int64_t(p.lut) * A.nlut;
    if (p.maxgrid)
        for (int i = threadIdx.x; i < A.nlut; i += blockDim.x)
            if (__ldg(&lut[i].w) != 0.0f) atomicMin(&sh_first, i);
    __syncthreads();
    if (threadIdx.x == 0) sh_S = p.maxgrid ? skip_threshold_from(sh_first - 1, A.nlut, p.inv_vmax, p.vmax_int) : -1;
    __syncthreads();
    const int S = sh_S;
    const bool use_skip = p.maxgrid != nullptr && S >= 0;

    const int parts = gridDim.y, part = blockIdx.y;
    const int zper = (p.mz + parts - 1) / parts;
    const int z1 = min(p.mz, (part + 1) * zper);
    for (int z = part * zper + threadIdx.x; z < z1; z += blockDim.x) {
        const int row = z / p.tiles_x, col = z - row * p.tiles_x;
        // with a texture: the first interior texel of the slice's padded cell
        p.slice_off[z] = p.tex ? uint32_t(col * (p.mx + 2) + 1) | (uint32_t(row * (p.my + 2) + 1) << 16)
                               : uint32_t(int64_t(row) * p.my * p.pitch + int64_t(col) * p.mx);
    }
    if (use_skip) {
        const int nwords = p.gy * p.gz * p.wpr;
        const int wper = (nwords + parts - 1) / parts;
        const int w1 = min(nwords, (part + 1) * wper);
        for (int w = part * wper + threadIdx.x; w < w1; w += blockDim.x)
            p.occ[w] = occupancy_word(p.maxgrid, p.gx, p.wpr, w, S);
    }
    if (part == 0 && threadIdx.x == 0) {
        BatchPair r = p;
        r.use_skip = use_skip ? 1 : 0;
        A.dst[A.first + blockIdx.x] = r;
    }
}

// Block (x, y): bitmap words x, x + gridDim.x, ... of view y's level.  Each
// marked cell c covers the level coordinates [8c - 1, 8c + 9] per axis (its
// samples' positions, [8c, 8c + 8) or up to half a voxel past a face, with a
// voxel of margin), a box in the world; the box's image footprint (one pixel
// of margin) and its depth range along the view direction go to the tiles.
// Views whose pair does not skip get the full range on every tile.
__global__ void __launch_bounds__(kBatchThreads) batch_bounds_kernel(const BatchView *__restrict__ views,
                                                                    const BatchPair *__restrict__ pairs,
                                                                    int32_t nviews, uint32_t *__restrict__ lo,
                                                                    uint32_t *__restrict__ hi)
{
    for (int vi = blockIdx.y; vi < nviews; vi += gridDim.y) {
        const BatchView &BV = views[vi];
        const ViewParams &V = BV.vp;
        const BatchPair &PR = pairs[BV.pair];
        const int btx = BV.btiles_x, bty = (V.H + kBoundsTile - 1) / kBoundsTile;
        uint32_t *vlo = lo + BV.bounds_begin, *vhi = hi + BV.bounds_begin;
        if (!PR.use_skip) {
            for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < btx * bty; t += gridDim.x * blockDim.x) {
                vlo[t] = 0u;
                vhi[t] = __float_as_uint(3.0e38f);
            }
            continue;
        }
        const float s[3] = {V.N[0] / float(PR.mx), V.N[1] / float(PR.my), V.N[2] / float(PR.mz)};
        const float invL = 1.0f / V.L;
        const int nwords = PR.gy * PR.gz * PR.wpr;
        for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += gridDim.x * blockDim.x) {
            uint32_t bits = __ldg(PR.occ + w);
            if (!bits) continue;
            const int r = w / PR.wpr, wx = w - r * PR.wpr;
            const int cy = r % PR.gy, cz = r / PR.gy;
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1u;
                const int cell[3] = {wx * 32 + b, cy, cz};
                // extremes of <p - centre, e> over the box, for e = r, u, b
                float xr[2] = {0.f, 0.f}, xu[2] = {0.f, 0.f}, xb[2] = {0.f, 0.f};
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float p0 = (float(8 * cell[a] - 1) + 0.5f) * s[a] - V.c[a];
                    const float p1 = (float(8 * cell[a] + 9) + 0.5f) * s[a] - V.c[a];
                    xr[0] += fminf(p0 * V.r[a], p1 * V.r[a]);
                    xr[1] += fmaxf(p0 * V.r[a], p1 * V.r[a]);
                    xu[0] += fminf(p0 * V.u[a], p1 * V.u[a]);
                    xu[1] += fmaxf(p0 * V.u[a], p1 * V.u[a]);
                    xb[0] += fminf(p0 * V.b[a], p1 * V.b[a]);
                    xb[1] += fmaxf(p0 * V.b[a], p1 * V.b[a]);
                }
                // pixel (px, py) looks along the line with sx = (px + 1/2) / W - 1/2,
                // sy = 1/2 - (py + 1/2) / H, sx = <p - centre, r> / L, sy likewise with u
                const float fx0 = (xr[0] * invL + 0.5f) * float(V.W) - 0.5f;
                const float fx1 = (xr[1] * invL + 0.5f) * float(V.W) - 0.5f;
                const float fy0 = (0.5f - xu[1] * invL) * float(V.H) - 0.5f;
                const float fy1 = (0.5f - xu[0] * invL) * float(V.H) - 0.5f;
                const float wmax = float(V.W) + 2.0f, hmax = float(V.H) + 2.0f;
                const int px0 = max(int(ceilf(fminf(fmaxf(fx0, -2.0f), wmax))) - 1, 0);
                const int px1 = min(int(floorf(fminf(fmaxf(fx1, -2.0f), wmax))) + 1, V.W - 1);
                const int py0 = max(int(ceilf(fminf(fmaxf(fy0, -2.0f), hmax))) - 1, 0);
                const int py1 = min(int(floorf(fminf(fmaxf(fy1, -2.0f), hmax))) + 1, V.H - 1);
                if (px0 > px1 || py0 > py1) continue;
                // depth along d = -b, plus L: positive inside the box
                const uint32_t dlo = __float_as_uint(V.L - xb[1]), dhi = __float_as_uint(V.L - xb[0]);
                for (int ty = py0 / kBoundsTile; ty <= py1 / kBoundsTile; ++ty)
                    for (int tx = px0 / kBoundsTile; tx <= px1 / kBoundsTile; ++tx) {
                        atomicMin(vlo + ty * btx + tx, dlo);
                        atomicMax(vhi + ty * btx + tx, dhi);
                    }
            }
        }
    }
}

template <typename T, bool kLutShared, bool kGather, bool kCount>
__global__ void __launch_bounds__(kBatchThreads, 4) render_batch_kernel(const __grid_constant__ BatchArgs P)
{
    extern __shared__ __align__(16) float4 slut[];
    if (kLutShared) {
        const int n = P.nluts * P.nlut;
        for (int i = threadIdx.x; i < n; i += blockDim.x) slut[i] = P.luts[i];
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    // warp tile wx x wy pixels; super tile of gx x gy warp tiles (gx gy = 8)
    const int wxl = P.wx_log2, wyl = 5 - wxl;
    const int gxl = wxl >= 4 ? 0 : 4 - wxl, gyl = 3 - gxl;
    const int lx = lane & ((1 << wxl) - 1), ly = lane >> wxl;

    uint32_t taken = 0, evaluated = 0;
    int v = -1;
    uint32_t vbegin = 0, vend = 0;
    // The next grab is issued before the current chunk is marched, so the
    // atomic's round trip overlaps the work instead of stalling the warp.
    const uint32_t chunk = uint32_t(P.chunk);
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(P.counter, chunk);
    base = __shfl_sync(0xffffffffu, base, 0);
    while (base < P.total_items) {
        uint32_t next = 0;
        if (lane == 0) next = atomicAdd(P.counter, chunk);
        const uint32_t end = min(base + chunk, P.total_items);
        for (uint32_t item = base; item < end; ++item) {
            if (item >= vend) {
                // the last view whose first warp tile is <= item (warp-uniform)
                int lo = v + 1, hi = P.nviews - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__ldg(P.item_begin + mid) <= item) lo = mid;
                    else hi = mid - 1;
                }
                v = lo;
                vbegin = __ldg(P.item_begin + v);
                vend = __ldg(P.item_begin + v + 1);
            }
            const BatchView &BV = P.views[v];
            const uint32_t local = item - vbegin;
            const uint32_t st = local >> 3, sub = local & 7;
            const uint32_t sty = st / uint32_t(BV.stiles_x), stx = st - sty * uint32_t(BV.stiles_x);
            const int px = int(stx << (gxl + wxl)) + int((sub & ((1u << gxl) - 1)) << wxl) + lx;
            const int py = int(sty << (gyl + wyl)) + int((sub >> gxl) << wyl) + ly;
            if (px >= BV.vp.W || py >= BV.vp.H) continue;
            const BatchPair &PR = P.pairs[BV.pair];
            const LevelGeom G{{PR.mx - 1, PR.my - 1, PR.mz - 1}, uint32_t(PR.pitch), PR.gy, PR.wpr,
                              PR.pitch * ((PR.mz + PR.tiles_x - 1) / PR.tiles_x) * PR.my};
            const float4 *lut = (kLutShared ? slut : P.luts) + int64_t(PR.lut) * P.nlut;
            DepthRange range{false, 0u, 0u};
            if (P.bounds_lo) {
                const uint32_t bt = BV.bounds_begin + uint32_t(py / kBoundsTile) * uint32_t(BV.btiles_x) +
                                    uint32_t(px / kBoundsTile);
                range = DepthRange{true, __ldg(P.bounds_lo + bt), __ldg(P.bounds_hi + bt)};
            }
            float4 acc;
            if constexpr (kGather) {
                const GatherTables<kLutShared> tab{lut, PR.slice_off, PR.occ, cudaTextureObject_t(PR.tex)};
                acc = march_ray<T, kCount>(BV.vp, static_cast<const T *>(PR.atlas), G, PR.use_skip != 0, tab, P.nlut,
                                           PR.inv_vmax, P.alpha_stop, px, py, taken, evaluated, range);
            } else {
                const CachedTables<kLutShared> tab{lut, PR.slice_off, PR.occ};
                acc = march_ray<T, kCount>(BV.vp, static_cast<const T *>(PR.atlas), G, PR.use_skip != 0, tab, P.nlut,
                                           PR.inv_vmax, P.alpha_stop, px, py, taken, evaluated, range);
            }
            const int64_t pix = BV.vp.out_offset / 4 + int64_t(py) * BV.vp.W + px;
            if (in_range(pix, P.out4_total, kFaultImageWrite)) reinterpret_cast<float4 *>(P.out)[pix] = acc;
            flush_count(taken, P.samples);
            if (kCount) flush_count(evaluated, P.counter_evaluated);
        }
        base = __shfl_sync(0xffffffffu, next, 0);
    }
    warp_add_count(taken, P.samples);
    if (kCount) warp_add_count(evaluated, P.counter_evaluated);
}

template <typename T>
auto pick_kernel(bool lut_shared, bool gather, bool count) -> void (*)(BatchArgs)
{
    if (gather)
        return lut_shared ? (count ? render_batch_kernel<T, true, true, true> : render_batch_kernel<T, true, true, false>)
                          : (count ? render_batch_kernel<T, false, true, true>
                                   : render_batch_kernel<T, false, true, false>);
    return lut_shared ? (count ? render_batch_kernel<T, true, false, true> : render_batch_kernel<T, true, false, false>)
                      : (count ? render_batch_kernel<T, false, false, true>
                               : render_batch_kernel<T, false, false, false>);
}

inline size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Workspace layout of a batch: the count of evaluated samples (bytes 8..15)
// and the queue counter (bytes 64..67) in the first 256 bytes, view records, the queue
// start of each view, pair records, then per pair its slice offsets and cell
// bitmap.
struct Plan {
    std::vector<std::tuple<int, int, int>> pairs;  // (slicemap, level, lut)
    std::vector<int> view_pair;
    std::vector<size_t> slice_at, occ_at;  // byte offsets of each pair's tables
    std::vector<uint32_t> bounds_begin;    // first depth-bounds tile of each view
    size_t views_at = 0, begin_at = 0, pairs_at = 0, total = 0;
    size_t bounds_lo_at = 0, bounds_hi_at = 0;  // 0: no depth bounds
    uint64_t bounds_tiles = 0;
    int max_words = 0;  // bitmap words of the largest level
};

int make_plan(const mctp_slicemap *sms, int32_t nsm, const mctp_view *views, const int32_t *view_sm,
              const int32_t *view_lut, int32_t nviews, int32_t nluts, bool bounds, Plan &plan)
{
    if (!sms || nsm < 1 || nviews < 0 || nluts < 1) return MCTP_EINVAL;
    if (nviews > 0 && (!views || !view_sm || !view_lut)) return MCTP_EINVAL;
    for (int i = 0; i < nsm; ++i) {
        const int rc = check_slicemap(&sms[i]);
        if (rc != MCTP_OK) return rc;
        if (sms[i].dtype != sms[0].dtype) return MCTP_EUNSUPPORTED;  // one element type per batch
    }
    std::map<std::tuple<int, int, int>, int> index;
    plan.view_pair.resize(size_t(nviews));
    for (int i = 0; i < nviews; ++i) {
        const int s = view_sm[i], l = view_lut[i];
        if (s < 0 || s >= nsm || l < 0 || l >= nluts) return MCTP_EINVAL;
        const int rc = check_view(views[i], sms[s].nlevels);
        if (rc != MCTP_OK) return rc;
        if (!level_fits_32bit(&sms[s], views[i].level)) return MCTP_ESIZE;  // texel offsets are 32-bit
        const auto key = std::make_tuple(s, views[i].level, l);
        auto it = index.find(key);
        if (it == index.end()) {
            it = index.emplace(key, int(plan.pairs.size())).first;
            plan.pairs.push_back(key);
        }
        plan.view_pair[size_t(i)] = it->second;
    }
    size_t at = kAlign;  // the counters
    plan.views_at = at;
    at = align_up(at + size_t(nviews) * sizeof(BatchView));
    plan.begin_at = at;
    at = align_up(at + (size_t(nviews) + 1) * sizeof(uint32_t));
    plan.pairs_at = at;
    at = align_up(at + plan.pairs.size() * sizeof(BatchPair));
    for (const auto &pr : plan.pairs) {
        const mctp_slicemap &sm = sms[std::get<0>(pr)];
        const int k = std::get<1>(pr);
        const int c = MCTP_MAXGRID_CELL;
        plan.slice_at.push_back(at);
        at = align_up(at + size_t(sm.dims[k][2]) * sizeof(uint32_t));
        plan.occ_at.push_back(at);
        if (sm.maxgrid[k]) {
            const size_t wpr = ((size_t(sm.dims[k][0]) + c - 1) / c + 31) / 32;
            const size_t rows = ((size_t(sm.dims[k][1]) + c - 1) / c) * ((size_t(sm.dims[k][2]) + c - 1) / c);
            at = align_up(at + rows * wpr * sizeof(uint32_t));
            plan.max_words = std::max(plan.max_words, int(rows * wpr));
        }
    }
    if (bounds && nviews > 0) {
        plan.bounds_begin.resize(size_t(nviews));
        uint64_t tiles = 0;
        for (int i = 0; i < nviews; ++i) {
            plan.bounds_begin[size_t(i)] = uint32_t(tiles);
            tiles += uint64_t((views[i].width + kBoundsTile - 1) / kBoundsTile) *
                     uint64_t((views[i].height + kBoundsTile - 1) / kBoundsTile);
            if (tiles > (uint64_t(1) << 31)) return MCTP_ESIZE;
        }
        plan.bounds_tiles = tiles;
        plan.bounds_lo_at = at;
        at = align_up(at + size_t(tiles) * sizeof(uint32_t));
        plan.bounds_hi_at = at;
        at = align_up(at + size_t(tiles) * sizeof(uint32_t));
    }
    plan.total = at;
    return MCTP_OK;
}

}  // namespace

MCTP_FAULT_READER(render_batch)

}  // namespace mctp

extern "C" int mctp_render_batch_workspace(const mctp_slicemap *sms, int32_t nsm, const mctp_view *views,
                                           const int32_t *view_slicemap, const int32_t *view_lut, int32_t nviews,
                                           int32_t nluts, size_t *bytes)
{
    using namespace mctp;
    if (!bytes) return MCTP_EINVAL;
    Plan plan;
    const int rc = make_plan(sms, nsm, views, view_slicemap, view_lut, nviews, nluts, true, plan);
    if (rc != MCTP_OK) return rc;
    *bytes = plan.total;
    return MCTP_OK;
}

namespace mctp {

// mctp_render_batch with optional per-view output offsets (in floats from
// out_rgba, 16-byte aligned); NULL: the images follow one another.
int render_batch_impl(const mctp_slicemap *sms, int32_t nsm, const mctp_view *views, const int32_t *view_slicemap,
                      const int32_t *view_lut, int32_t nviews, const float *luts_rgba, int32_t nluts, int32_t nlut,
                      float alpha_stop, const mctp_batch_tuning *tuning, float *out_rgba, const int64_t *out_offsets,
                      uint64_t *samples_taken, void *workspace, size_t workspace_bytes, cudaStream_t s,
                      int depth_bounds)
{
    using namespace mctp::render;
    Plan plan;
    int rc = make_plan(sms, nsm, views, view_slicemap, view_lut, nviews, nluts, depth_bounds != kBoundsOff, plan);
    if (rc != MCTP_OK) return rc;
    if (depth_bounds == kBoundsIfRoom && workspace_bytes < plan.total) {
        plan = Plan();
        rc = make_plan(sms, nsm, views, view_slicemap, view_lut, nviews, nluts, false, plan);
        if (rc != MCTP_OK) return rc;
    }
    if (!luts_rgba || !out_rgba || nlut < 2 || nlut > kMaxLut) return MCTP_EINVAL;
    if (!(alpha_stop > 0.0f && alpha_stop <= 1.0f)) return MCTP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(luts_rgba) & 15) || (reinterpret_cast<uintptr_t>(out_rgba) & 15))
        return MCTP_EINVAL;
    mctp_batch_tuning tun{8, 2, 0, 0};
    if (tuning) {
        tun = *tuning;
        if (tun.warp_w == 0) tun.warp_w = 8;
        if (tun.chunk == 0) tun.chunk = 2;
    }
    const int wxl = log2_exact(tun.warp_w);
    if (wxl < 2 || wxl > 5 || tun.chunk < 1 || tun.chunk > 64 || tun.ctas_per_sm < 0 ||
        (tun.flags & ~MCTP_BATCH_COUNT_EVALUATED) != 0)
        return MCTP_EINVAL;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & (kAlign - 1))) return MCTP_EINVAL;
    if (workspace_bytes < plan.total) return MCTP_ESIZE;

    if (out_offsets)
        for (int i = 0; i < nviews; ++i)
            if (out_offsets[i] < 0 || (out_offsets[i] & 3)) return MCTP_EINVAL;
    if (samples_taken && cudaMemsetAsync(samples_taken, 0, sizeof(uint64_t), s) != cudaSuccess) return MCTP_ECUDA;
    if (nviews == 0) return cudaMemsetAsync(workspace, 0, 16, s) == cudaSuccess ? MCTP_OK : MCTP_ECUDA;
    uint8_t *ws = static_cast<uint8_t *>(workspace);
    BatchView *ws_views = reinterpret_cast<BatchView *>(ws + plan.views_at);
    uint32_t *ws_begin = reinterpret_cast<uint32_t *>(ws + plan.begin_at);
    BatchPair *ws_pairs = reinterpret_cast<BatchPair *>(ws + plan.pairs_at);
    const float4 *luts = reinterpret_cast<const float4 *>(luts_rgba);
    // corners by texture gathers when every (slicemap, level) of the batch has an atlas texture
    bool gather = !plan.pairs.empty();
    for (const auto &pr : plan.pairs) gather = gather && sms[std::get<0>(pr)].texture[std::get<1>(pr)] != 0;

    // ---- pair records and tables
    {
        PrepArgs A{};
        A.dst = ws_pairs;
        A.luts = luts;
        A.nlut = nlut;
        const int npairs = int(plan.pairs.size());
        for (int first = 0; first < npairs; first += kPrepPairs) {
            const int cnt = std::min(kPrepPairs, npairs - first);
            int parts = 1;
            for (int i = 0; i < cnt; ++i) {
                const auto &pr = plan.pairs[size_t(first + i)];
                const mctp_slicemap &sm = sms[std::get<0>(pr)];
                const int k = std::get<1>(pr);
                BatchPair &p = A.pair[i];
                p = BatchPair{};
                const int c = MCTP_MAXGRID_CELL;
                p.atlas = sm.atlas[k];
                p.tex = gather ? sm.texture[k] : 0;
                p.maxgrid = static_cast<const uint16_t *>(sm.maxgrid[k]);
                p.slice_off = reinterpret_cast<uint32_t *>(ws + plan.slice_at[size_t(first + i)]);
                p.occ = reinterpret_cast<uint32_t *>(ws + plan.occ_at[size_t(first + i)]);
                p.mx = sm.dims[k][0];
                p.my = sm.dims[k][1];
                p.mz = sm.dims[k][2];
                p.tiles_x = sm.tiles_x[k];
                p.gx = (p.mx + c - 1) / c;
                p.gy = (p.my + c - 1) / c;
                p.gz = (p.mz + c - 1) / c;
                p.wpr = (p.gx + 31) / 32;
                p.pitch = int64_t(sm.tiles_x[k]) * sm.dims[k][0];
                p.lut = std::get<2>(pr);
                p.inv_vmax = float(1.0 / double((1u << sm.bits) - 1u));
                p.vmax_int = int((1u << sm.bits) - 1u);
                const int64_t words = p.maxgrid ? int64_t(p.gy) * p.gz * p.wpr : 0;
                parts = int(std::max<int64_t>(parts, std::min<int64_t>(64, (words + 1023) / 1024)));
            }
            A.first = first;
            A.count = cnt;
            batch_prep_kernel<<<dim3(unsigned(cnt), unsigned(parts)), kBatchThreads, 0, s>>>(A);
            rc = launch_status();
            if (rc != MCTP_OK) return rc;
        }
    }

    // ---- view records and the queue
    const int wyl = 5 - wxl, gxl = wxl >= 4 ? 0 : 4 - wxl, gyl = 3 - gxl;
    const int sw = 1 << (gxl + wxl), sh = 1 << (gyl + wyl);  // super tile in pixels
    uint64_t items = 0;
    int64_t out_off = 0;
    {
        UploadArgs A{};
        A.dst = ws_views;
        A.item_begin = ws_begin;
        std::vector<BatchView> recs(static_cast<size_t>(nviews));
        for (int i = 0; i < nviews; ++i) {
            const mctp_view &w = views[i];
            BatchView &B = recs[size_t(i)];
            fill_view(&sms[view_slicemap[i]], w, B.vp);
            B.vp.out_offset = out_offsets ? out_offsets[i] : out_off;
            B.pair = plan.view_pair[size_t(i)];
            B.stiles_x = (w.width + sw - 1) / sw;
            B.item_begin = uint32_t(items);
            B.bounds_begin = plan.bounds_tiles ? plan.bounds_begin[size_t(i)] : 0u;
            B.btiles_x = (w.width + kBoundsTile - 1) / kBoundsTile;
            items += uint64_t(B.stiles_x) * uint64_t((w.height + sh - 1) / sh) * 8u;
            out_off += int64_t(w.width) * w.height * 4;
            if (items > (uint64_t(1) << 31)) return MCTP_ESIZE;  // queue positions are 32-bit
        }
        for (int first = 0; first < nviews; first += kUploadViews) {
            const int cnt = std::min(kUploadViews, nviews - first);
            for (int i = 0; i < cnt; ++i) A.view[i] = recs[size_t(first + i)];
            A.first = first;
            A.count = cnt;
            A.total_items = uint32_t(items);
            A.last = first + cnt == nviews ? 1 : 0;
            batch_upload_kernel<<<1, kBatchThreads, 0, s>>>(A);
            rc = launch_status();
            if (rc != MCTP_OK) return rc;
        }
    }

    // ---- depth bounds of the marked cells per view tile
    uint32_t *bounds_lo = nullptr, *bounds_hi = nullptr;
    if (plan.bounds_tiles) {
        bounds_lo = reinterpret_cast<uint32_t *>(ws + plan.bounds_lo_at);
        bounds_hi = reinterpret_cast<uint32_t *>(ws + plan.bounds_hi_at);
        const size_t nb = size_t(plan.bounds_tiles) * sizeof(uint32_t);
        if (cudaMemsetAsync(bounds_lo, 0xff, nb, s) != cudaSuccess || cudaMemsetAsync(bounds_hi, 0, nb, s) != cudaSuccess)
            return MCTP_ECUDA;
        const int gx = std::max(1, std::min(64, (plan.max_words + kBatchThreads - 1) / kBatchThreads));
        const int gy = std::min(nviews, 65535);
        batch_bounds_kernel<<<dim3(unsigned(gx), unsigned(gy)), kBatchThreads, 0, s>>>(ws_views, ws_pairs, nviews,
                                                                                       bounds_lo, bounds_hi);
        rc = launch_status();
        if (rc != MCTP_OK) return rc;
    }

    // ---- the persistent march over the queue
    if (cudaMemsetAsync(ws, 0, kAlign, s) != cudaSuccess) return MCTP_ECUDA;  // evaluated samples, queue counters
    BatchArgs P{};
    P.views = ws_views;
    P.item_begin = ws_begin;
    P.pairs = ws_pairs;
    P.luts = luts;
    P.out = out_rgba;
    P.samples = reinterpret_cast<unsigned long long *>(samples_taken);
    P.counter = reinterpret_cast<unsigned int *>(ws + 64);
    P.counter_evaluated = reinterpret_cast<unsigned long long *>(ws + 8);
    P.bounds_lo = bounds_lo;
    P.bounds_hi = bounds_hi;
    P.nviews = nviews;
    P.nlut = nlut;
    P.nluts = nluts;
    P.total_items = uint32_t(items);
    P.wx_log2 = wxl;
    P.chunk = tun.chunk;
    P.alpha_stop = alpha_stop;
    P.out4_total = 0;
    {
        int64_t off = 0;
        for (int i = 0; i < nviews; ++i) {
            const int64_t first = out_offsets ? out_offsets[i] : off;
            P.out4_total = std::max<int64_t>(P.out4_total, first / 4 + int64_t(views[i].width) * views[i].height);
            off += int64_t(views[i].width) * views[i].height * 4;
        }
    }
    const size_t lut_bytes = size_t(nluts) * size_t(nlut) * sizeof(float4);
    const bool lut_shared = lut_bytes <= kLutSmemMax;
    const size_t smem = lut_shared ? lut_bytes : 0;
    const bool count = (tun.flags & MCTP_BATCH_COUNT_EVALUATED) != 0;
    void (*kern)(BatchArgs) = sms[0].dtype == MCTP_U8 ? pick_kernel<uint8_t>(lut_shared, gather, count)
                                                      : pick_kernel<uint16_t>(lut_shared, gather, count);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, smem) != cudaSuccess)
        return MCTP_ECUDA;
    per_sm = std::max(per_sm, 1);
    if (tun.ctas_per_sm > 0) per_sm = std::min(per_sm, int(tun.ctas_per_sm));
    const uint64_t warps_needed = (items + uint64_t(tun.chunk) - 1) / uint64_t(tun.chunk);
    const uint64_t ctas_needed = (warps_needed + kBatchThreads / 32 - 1) / (kBatchThreads / 32);
    const uint64_t grid = std::min<uint64_t>(ctas_needed, uint64_t(per_sm) * uint64_t(num_sms()));
    kern<<<unsigned(grid), kBatchThreads, smem, s>>>(P);
    return launch_status();
}

// Upper bound of mctp_render_batch_workspace over every batch of at most
// max_views views of these slicemaps.
size_t batch_workspace_bound(const mctp_slicemap *sms, int32_t nsm, int32_t max_views)
{
    size_t per_pair = 0;
    for (int i = 0; i < nsm; ++i)
        for (int k = 0; k < sms[i].nlevels; ++k) {
            const int c = MCTP_MAXGRID_CELL;
            size_t t = align_up(size_t(sms[i].dims[k][2]) * sizeof(uint32_t));
            if (sms[i].maxgrid[k]) {
                const size_t wpr = ((size_t(sms[i].dims[k][0]) + c - 1) / c + 31) / 32;
                const size_t rows = ((size_t(sms[i].dims[k][1]) + c - 1) / c) * ((size_t(sms[i].dims[k][2]) + c - 1) / c);
                t += align_up(rows * wpr * sizeof(uint32_t));
            }
            per_pair = std::max(per_pair, t);
        }
    const size_t v = size_t(std::max(max_views, 0));
    const size_t tiles = (size_t(1024) / kBoundsTile + 1) * (size_t(1024) / kBoundsTile + 1);  // a 1024^2 view
    return kAlign + align_up(v * sizeof(BatchView)) + align_up((v + 1) * sizeof(uint32_t)) +
           align_up(v * sizeof(BatchPair)) + v * per_pair + 2 * align_up(v * tiles * sizeof(uint32_t));
}

}  // namespace mctp

extern "C" int mctp_render_batch(const mctp_slicemap *sms, int32_t nsm, const mctp_view *views,
                                 const int32_t *view_slicemap, const int32_t *view_lut, int32_t nviews,
                                 const float *luts_rgba, int32_t nluts, int32_t nlut, float alpha_stop,
                                 const mctp_batch_tuning *tuning, float *out_rgba, uint64_t *samples_taken,
                                 void *workspace, size_t workspace_bytes, void *stream)
{
    return mctp::render_batch_impl(sms, nsm, views, view_slicemap, view_lut, nviews, luts_rgba, nluts, nlut,
                                   alpha_stop, tuning, out_rgba, nullptr, samples_taken, workspace, workspace_bytes,
                                   mctp::as_stream(stream), mctp::kBoundsOn);
}

// ---- batched rendering without a caller workspace
//
// Some callers cannot hand the library device memory for the workspace: a
// plain C host program with no device allocator of its own, or a serving loop
// that must never enter an allocator once it runs.  For them the scratch lives
// in a fixed-size array of this module's device memory, created with the
// module, so no call allocates.  Its address is looked up once per device, on
// the first call made with that device current.
namespace {

constexpr size_t kStaticScratchBytes = size_t(8) << 20;  // MCTP_BATCH_STATIC_SCRATCH
static_assert(kStaticScratchBytes == MCTP_BATCH_STATIC_SCRATCH, "header and library disagree");
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_batch_scratch[kStaticScratchBytes];

std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Address of g_batch_scratch on the current device (looked up once per device).
int static_scratch(void **ptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCTP_ECUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_batch_scratch) != cudaSuccess || !p) return MCTP_ECUDA;
        g_scratch_ptr[dev] = p;
    }
    *ptr = g_scratch_ptr[dev];
    return MCTP_OK;
}

}  // namespace

extern "C" int mctp_render_batch_static(const mctp_slicemap *sms, int32_t nsm, const mctp_view *views,
                                        const int32_t *view_slicemap, const int32_t *view_lut, int32_t nviews,
                                        const float *luts_rgba, int32_t nluts, int32_t nlut, float alpha_stop,
                                        const mctp_batch_tuning *tuning, float *out_rgba, uint64_t *samples_taken,
                                        void *stream)
{
    size_t need = 0;
    int rc = mctp_render_batch_workspace(sms, nsm, views, view_slicemap, view_lut, nviews, nluts, &need);
    if (rc != MCTP_OK) return rc;
    if (need > kStaticScratchBytes) return MCTP_ESIZE;
    void *scratch = nullptr;
    rc = static_scratch(&scratch);
    if (rc != MCTP_OK) return rc;
    return mctp_render_batch(sms, nsm, views, view_slicemap, view_lut, nviews, luts_rgba, nluts, nlut, alpha_stop,
                             tuning, out_rgba, samples_taken, scratch, kStaticScratchBytes, stream);
}
