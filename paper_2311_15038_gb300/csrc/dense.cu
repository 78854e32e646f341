// dense.cu -- differentiable rendering of a dense FP32 intensity volume, its
// adjoint, and the two small kernels of a fit (L2 loss, Adam step).
//
// The previews show a reduced volume in place of the full one (Sec. I,
// Sec. III).  Here the reduced volume (and the transfer function) can be
// fitted so that its renders match renders of the full-resolution source: the
// forward march is that of the slicemap renderer (same FP32 ray set-up,
// fixed-point sample positions, trilinear interpolation, linear LUT lookup,
// premultiplied compositing, early exit) on an FP32 volume of intensities,
// v = min(max(raw, 0), 1), without empty-space skipping (the LUT changes
// while fitting).
//
// Adjoint, per ray, with the stop index of the forward march held fixed: for
// sample k with transmittance T_k = 1 - A_k, opacity a_k and colour c_k, and
// the colour RC / opacity RA that the samples after k composite to from a
// fresh start,
//   dL/da_k = T_k (gC . (c_k - RC) + gA (1 - RA)),   dL/dc_k = T_k a_k gC,
// and then RC <- a_k c_k + (1 - a_k) RC, RA <- a_k + (1 - a_k) RA walking
// back to front.  The walk needs T_k in reverse order: a first pass records
// A at every 64th sample (per-ray checkpoints), then each 64-sample segment,
// last to first, is re-marched forward from its checkpoint to recover its
// T_k (no division by T, so no loss of accuracy when T is small) and then
// walked backward.  The LUT gradient is accumulated per CTA in shared memory;
// the volume gradient is scattered with trilinear weights by atomic adds.  Both
// are first summed in registers over runs of consecutive samples that touch the
// same table entries / corner voxels.
#include "render_common.cuh"

namespace mctp {
namespace {

using namespace render;

constexpr int kDenseViews = 48;  // views per launch (kernel parameter space)
constexpr int kSeg = 64;         // samples per checkpoint segment
constexpr int kMaxSeg = 32;      // so rays of at most 2048 samples
constexpr int kThreads = kTileW * kTileH;

struct DenseArgs {
    const float *vol;
    int32_t mx, my, mz;
    int32_t nviews;
    const float4 *lut;
    int32_t nlut;
    float alpha_stop;
    float *out;               // forward: premultiplied RGBA
    unsigned long long *samples;  // forward: samples taken (or nullptr)
    const float *grad_out;    // backward: dL/dRGBA
    float *grad_vol;          // backward, accumulated with atomics
    float *grad_lut;
    int64_t total_tiles;
    ViewParams view[kDenseViews];
};

// One sample of the dense volume at fixed-point coordinates U.
struct Tap {
    uint32_t o000;          // offset of the lower corner
    uint32_t dx, dy, dz;    // offsets to the upper corner per axis (0 when clamped together)
    float fx, fy, fz;
    float raw;
};

__device__ __forceinline__ Tap dense_tap(const float *vol, int mx, int my, int mz, const long long U[3])
{
    const int ix = int(U[0] >> 32), iy = int(U[1] >> 32), iz = int(U[2] >> 32);
    const int x0 = min(max(ix, 0), mx - 1), y0 = min(max(iy, 0), my - 1), z0 = min(max(iz, 0), mz - 1);
    const int x1 = min(max(ix + 1, 0), mx - 1), y1 = min(max(iy + 1, 0), my - 1), z1 = min(max(iz + 1, 0), mz - 1);
    Tap t;
    const uint32_t sy = uint32_t(mx), sz = uint32_t(mx) * uint32_t(my);
    t.o000 = uint32_t(z0) * sz + uint32_t(y0) * sy + uint32_t(x0);
    t.dx = uint32_t(x1 - x0);
    t.dy = uint32_t(y1 - y0) * sy;
    t.dz = uint32_t(z1 - z0) * sz;
    t.fx = float(uint32_t(U[0])) * 2.3283064365386963e-10f;
    t.fy = float(uint32_t(U[1])) * 2.3283064365386963e-10f;
    t.fz = float(uint32_t(U[2])) * 2.3283064365386963e-10f;
    const float *p = vol + t.o000;
    const float v000 = __ldg(p), v100 = __ldg(p + t.dx);
    const float v010 = __ldg(p + t.dy), v110 = __ldg(p + t.dy + t.dx);
    const float v001 = __ldg(p + t.dz), v101 = __ldg(p + t.dz + t.dx);
    const float v011 = __ldg(p + t.dz + t.dy), v111 = __ldg(p + t.dz + t.dy + t.dx);
    const float c00 = fmaf(t.fx, v100 - v000, v000), c10 = fmaf(t.fx, v110 - v010, v010);
    const float c01 = fmaf(t.fx, v101 - v001, v001), c11 = fmaf(t.fx, v111 - v011, v011);
    const float c0 = fmaf(t.fy, c10 - c00, c00), c1 = fmaf(t.fy, c11 - c01, c01);
    t.raw = fmaf(t.fz, c1 - c0, c0);
    return t;
}

struct Look {
    float4 e;   // interpolated RGBA (straight colour)
    float fl;   // fraction between entries j and j + 1
    int j;
};

__device__ __forceinline__ Look lookup(const float4 *lut, int nlut, float raw)
{
    const float x = __fmul_rn(fminf(fmaxf(raw, 0.0f), 1.0f), float(nlut - 1));
    Look l;
    l.j = min(int(x), nlut - 2);
    l.fl = x - float(l.j);
    const float4 e0 = lut[l.j], e1 = lut[l.j + 1];
    l.e = make_float4(fmaf(l.fl, e1.x - e0.x, e0.x), fmaf(l.fl, e1.y - e0.y, e0.y), fmaf(l.fl, e1.z - e0.z, e0.z),
                      fmaf(l.fl, e1.w - e0.w, e0.w));
    return l;
}

// FP32 set-up of the ray of pixel (px, py) (that of the slicemap renderer):
// sample count n and the fixed-point coordinates of sample 0.
__device__ __forceinline__ int ray_start(const ViewParams &V, int px, int py, long long U0[3])
{
    const float sx = __fsub_rn(__fdiv_rn(__fadd_rn(float(px), 0.5f), float(V.W)), 0.5f);
    const float sy = __fsub_rn(0.5f, __fdiv_rn(__fadd_rn(float(py), 0.5f), float(V.H)));
    const float sxL = __fmul_rn(sx, V.L), syL = __fmul_rn(sy, V.L);
    float o[3], d[3];
    float tmin = -INFINITY, tmax = INFINITY;
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t1 = __fadd_rn(V.c[a], __fmul_rn(sxL, V.r[a]));
        const float t2 = __fadd_rn(t1, __fmul_rn(syL, V.u[a]));
        o[a] = __fadd_rn(t2, __fmul_rn(V.L, V.b[a]));
        d[a] = -V.b[a];
        if (d[a] != 0.0f) {
            const float inv = __frcp_rn(d[a]);
            const float s0 = __fmul_rn(__fsub_rn(0.0f, o[a]), inv);
            const float s1 = __fmul_rn(__fsub_rn(V.N[a], o[a]), inv);
            tmin = fmaxf(tmin, fminf(s0, s1));
            tmax = fminf(tmax, fmaxf(s0, s1));
        } else if (!(o[a] >= 0.0f && o[a] <= V.N[a])) {
            miss = true;
        }
    }
    int n = 0;
    if (!miss && tmax > tmin) n = int(floorf(__fdiv_rn(__fsub_rn(tmax, tmin), V.delta)));
    if (n > 0)
#pragma unroll
        for (int a = 0; a < 3; ++a) U0[a] = start_coord(o[a], d[a], tmin, 0.5f * V.delta, V.sc_hi[a], V.sc_lo[a]);
    return n;
}

__device__ __forceinline__ void sample_coords(const ViewParams &V, const long long U0[3], int k, long long U[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a) U[a] = U0[a] + (long long)k * V.dU[a];
}

// Pixel of this thread in tile `tile` of the launch; false past the image.
__device__ __forceinline__ bool pixel_of(const DenseArgs &P, int64_t tile, int &v, int &px, int &py)
{
    while (v + 1 < P.nviews && tile >= P.view[v + 1].tile_begin) ++v;
    const ViewParams &V = P.view[v];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = tile - V.tile_begin;
    px = int(t % V.tiles_w) * kTileW + (warp & 1) * 8 + (lane & 7);
    py = int(t / V.tiles_w) * kTileH + (warp >> 1) * 4 + (lane >> 3);
    return px < V.W && py < V.H;
}

__global__ void __launch_bounds__(kThreads) dense_forward_kernel(const __grid_constant__ DenseArgs P)
{
    extern __shared__ __align__(16) float4 lut[];
    for (int i = threadIdx.x; i < P.nlut; i += blockDim.x) lut[i] = P.lut[i];
    __syncthreads();
    int v = 0;
    unsigned long long taken = 0;
    for (int64_t tile = blockIdx.x; tile < P.total_tiles; tile += gridDim.x) {
        int px, py;
        if (!pixel_of(P, tile, v, px, py)) continue;
        const ViewParams &V = P.view[v];
        long long U0[3];
        const int n = ray_start(V, px, py, U0);
        float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
        int k = 0;
        while (k < n) {
            long long U[3];
            sample_coords(V, U0, k, U);
            const Look l = lookup(lut, P.nlut, dense_tap(P.vol, P.mx, P.my, P.mz, U).raw);
            const float w = (1.0f - A) * l.e.w;
            C0 = fmaf(w, l.e.x, C0);
            C1 = fmaf(w, l.e.y, C1);
            C2 = fmaf(w, l.e.z, C2);
            A += w;
            ++k;
            if (A >= P.alpha_stop) break;
        }
        taken += (unsigned long long)k;
        reinterpret_cast<float4 *>(P.out + V.out_offset)[int64_t(py) * V.W + px] = make_float4(C0, C1, C2, A);
    }
    if (P.samples) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) taken += __shfl_xor_sync(0xffffffffu, taken, o);
        if ((threadIdx.x & 31) == 0 && taken) atomicAdd(P.samples, taken);
    }
}

__global__ void __launch_bounds__(kThreads) dense_backward_kernel(const __grid_constant__ DenseArgs P)
{
    extern __shared__ __align__(16) float4 lut[];
    float *glut = reinterpret_cast<float *>(lut + P.nlut);  // nlut * 4, this CTA's LUT gradient
    for (int i = threadIdx.x; i < P.nlut; i += blockDim.x) lut[i] = P.lut[i];
    for (int i = threadIdx.x; i < 4 * P.nlut; i += blockDim.x) glut[i] = 0.0f;
    __syncthreads();
    const float nl1 = float(P.nlut - 1);
    int v = 0;
    for (int64_t tile = blockIdx.x; tile < P.total_tiles; tile += gridDim.x) {
        int px, py;
        if (!pixel_of(P, tile, v, px, py)) continue;
        const ViewParams &V = P.view[v];
        long long U0[3];
        const int n = ray_start(V, px, py, U0);
        if (n <= 0) continue;
        const float4 g = reinterpret_cast<const float4 *>(P.grad_out + V.out_offset)[int64_t(py) * V.W + px];
        // pass 1: the forward march's opacity at every segment start, and its stop
        float ck[kMaxSeg];
        float A = 0.f;
        int ne = 0;
        while (ne < n) {
            if ((ne & (kSeg - 1)) == 0) ck[ne / kSeg] = A;
            long long U[3];
            sample_coords(V, U0, ne, U);
            const Look l = lookup(lut, P.nlut, dense_tap(P.vol, P.mx, P.my, P.mz, U).raw);
            A += (1.0f - A) * l.e.w;
            ++ne;
            if (A >= P.alpha_stop) break;
        }
        // pass 2: segments last to first, each re-marched for its T_k, then walked back
        float RC0 = 0.f, RC1 = 0.f, RC2 = 0.f, RA = 0.f;
        int run_j = -1;
        float run_lo[4] = {0.f, 0.f, 0.f, 0.f}, run_hi[4] = {0.f, 0.f, 0.f, 0.f};
        uint32_t cell_o = 0xffffffffu, cell_dx = 0, cell_dy = 0, cell_dz = 0;
        float cw[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        auto flush_cell = [&]() {
            if (cell_o == 0xffffffffu) return;
            float *q = P.grad_vol + cell_o;
            const uint32_t off[8] = {0u, cell_dx, cell_dy, cell_dy + cell_dx, cell_dz, cell_dz + cell_dx,
                                     cell_dz + cell_dy, cell_dz + cell_dy + cell_dx};
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (cw[c] != 0.0f) atomicAdd(q + off[c], cw[c]);
                cw[c] = 0.f;
            }
        };
        auto flush_run = [&]() {
            if (run_j < 0) return;
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) {
                if (run_lo[ch] != 0.0f) atomicAdd(&glut[4 * run_j + ch], run_lo[ch]);
                if (run_hi[ch] != 0.0f) atomicAdd(&glut[4 * (run_j + 1) + ch], run_hi[ch]);
                run_lo[ch] = 0.f;
                run_hi[ch] = 0.f;
            }
        };
        for (int seg = (ne - 1) / kSeg; seg >= 0; --seg) {
            const int k0 = seg * kSeg, k1 = min(k0 + kSeg, ne);
            float T[kSeg];
            A = ck[seg];
            for (int k = k0; k < k1; ++k) {
                T[k - k0] = 1.0f - A;
                long long U[3];
                sample_coords(V, U0, k, U);
                const Look l = lookup(lut, P.nlut, dense_tap(P.vol, P.mx, P.my, P.mz, U).raw);
                A += (1.0f - A) * l.e.w;
            }
            for (int k = k1 - 1; k >= k0; --k) {
                long long U[3];
                sample_coords(V, U0, k, U);
                const Tap tp = dense_tap(P.vol, P.mx, P.my, P.mz, U);
                const Look l = lookup(lut, P.nlut, tp.raw);
                const float Tk = T[k - k0], a = l.e.w;
                const float ga = Tk * (g.x * (l.e.x - RC0) + g.y * (l.e.y - RC1) + g.z * (l.e.z - RC2) + g.w * (1.0f - RA));
                const float ta = Tk * a;
                const float ge[4] = {g.x * ta, g.y * ta, g.z * ta, ga};
                RC0 = fmaf(a, l.e.x - RC0, RC0);
                RC1 = fmaf(a, l.e.y - RC1, RC1);
                RC2 = fmaf(a, l.e.z - RC2, RC2);
                RA = fmaf(a, 1.0f - RA, RA);
                const float4 e0 = lut[l.j], e1 = lut[l.j + 1];
                const float de[4] = {e1.x - e0.x, e1.y - e0.y, e1.z - e0.z, e1.w - e0.w};
                // LUT gradient: consecutive samples of a ray mostly fall between the
                // same two entries, so it is summed in registers until the entry pair
                // changes and only then added to the CTA's table
                if (l.j != run_j) {
                    flush_run();
                    run_j = l.j;
                }
                float gv = 0.f;
#pragma unroll
                for (int ch = 0; ch < 4; ++ch) {
                    run_lo[ch] = fmaf(1.0f - l.fl, ge[ch], run_lo[ch]);
                    run_hi[ch] = fmaf(l.fl, ge[ch], run_hi[ch]);
                    gv = fmaf(ge[ch], de[ch], gv);
                }
                gv *= nl1;
                if (gv != 0.0f && tp.raw > 0.0f && tp.raw < 1.0f) {
                    // the volume gradient is summed in registers while consecutive
                    // samples share the same eight corner voxels
                    if (tp.o000 != cell_o || tp.dx != cell_dx || tp.dy != cell_dy || tp.dz != cell_dz) {
                        flush_cell();
                        cell_o = tp.o000;
                        cell_dx = tp.dx;
                        cell_dy = tp.dy;
                        cell_dz = tp.dz;
                    }
                    const float wx1 = tp.fx, wx0 = 1.0f - tp.fx, wy1 = tp.fy, wy0 = 1.0f - tp.fy;
                    const float wz1 = tp.fz * gv, wz0 = (1.0f - tp.fz) * gv;
                    cw[0] = fmaf(wx0 * wy0, wz0, cw[0]);
                    cw[1] = fmaf(wx1 * wy0, wz0, cw[1]);
                    cw[2] = fmaf(wx0 * wy1, wz0, cw[2]);
                    cw[3] = fmaf(wx1 * wy1, wz0, cw[3]);
                    cw[4] = fmaf(wx0 * wy0, wz1, cw[4]);
                    cw[5] = fmaf(wx1 * wy0, wz1, cw[5]);
                    cw[6] = fmaf(wx0 * wy1, wz1, cw[6]);
                    cw[7] = fmaf(wx1 * wy1, wz1, cw[7]);
                }
            }
        }
        flush_run();
        flush_cell();
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 4 * P.nlut; i += blockDim.x)
        if (glut[i] != 0.0f) atomicAdd(P.grad_lut + i, glut[i]);
}

__global__ void l2_loss_kernel(const float *__restrict__ x, const float *__restrict__ t, int64_t n, float scale,
                               float *__restrict__ grad, float *__restrict__ loss)
{
    float acc = 0.f;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float d = x[i] - t[i];
        acc = fmaf(d, d, acc);
        if (grad) grad[i] = 2.0f * scale * d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(loss, scale * acc);
    }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2, float lo, float hi)
{
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float step = lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        p[i] = fminf(fmaxf(p[i] - step, lo), hi);
    }
}

// Argument checks and per-launch set-up shared by the forward and backward calls.
int dense_prepare(bool backward, const float *vol, int32_t mx, int32_t my, int32_t mz, const int64_t *src_dims,
                  const mctp_view *views, int32_t nviews, const float *lut_rgba, int32_t nlut, float alpha_stop,
                  mctp_slicemap &sm)
{
    if (!vol || !src_dims || (!views && nviews) || nviews < 0 || !lut_rgba) return MCTP_EINVAL;
    if (mx < 1 || my < 1 || mz < 1 || nlut < 2 || nlut > kMaxLut) return MCTP_EINVAL;
    if (int64_t(mx) * my * mz > (int64_t(1) << 31)) return MCTP_ESIZE;  // 32-bit voxel offsets
    if (!(alpha_stop > 0.0f && alpha_stop <= 1.0f)) return MCTP_EINVAL;
    if (reinterpret_cast<uintptr_t>(lut_rgba) & 15) return MCTP_EINVAL;
    sm = mctp_slicemap{};
    sm.nlevels = 1;
    for (int a = 0; a < 3; ++a) {
        if (src_dims[a] < 1 || src_dims[a] > (int64_t(1) << 31)) return MCTP_EINVAL;
        sm.src_dims[a] = src_dims[a];
    }
    sm.dims[0][0] = mx;
    sm.dims[0][1] = my;
    sm.dims[0][2] = mz;
    const double L = sqrt(double(src_dims[0]) * double(src_dims[0]) + double(src_dims[1]) * double(src_dims[1]) +
                          double(src_dims[2]) * double(src_dims[2]));
    const double smin = std::min(std::min(double(src_dims[0]) / mx, double(src_dims[1]) / my), double(src_dims[2]) / mz);
    for (int i = 0; i < nviews; ++i) {
        if (views[i].level != 0) return MCTP_EINVAL;
        const int rc = check_view(views[i], 1);
        if (rc != MCTP_OK) return rc;
        // a ray has at most L / Delta + 1 samples; the adjoint keeps kMaxSeg checkpoints
        if (backward && L / (double(views[i].step) * smin) * 1.0001 + 2.0 > double(kSeg) * kMaxSeg)
            return MCTP_ESIZE;
    }
    return MCTP_OK;
}

int dense_launch(bool backward, const mctp_slicemap &sm, const float *vol, const mctp_view *views, int32_t nviews,
                 const float *lut_rgba, int32_t nlut, float alpha_stop, float *out, uint64_t *samples,
                 const float *grad_out, float *grad_vol, float *grad_lut, cudaStream_t s)
{
    DenseArgs P{};
    P.samples = reinterpret_cast<unsigned long long *>(samples);
    P.vol = vol;
    P.mx = sm.dims[0][0];
    P.my = sm.dims[0][1];
    P.mz = sm.dims[0][2];
    P.lut = reinterpret_cast<const float4 *>(lut_rgba);
    P.nlut = nlut;
    P.alpha_stop = alpha_stop;
    P.out = out;
    P.grad_out = grad_out;
    P.grad_vol = grad_vol;
    P.grad_lut = grad_lut;
    const size_t smem = size_t(nlut) * sizeof(float4) * (backward ? 2 : 1);
    auto kern = backward ? dense_backward_kernel : dense_forward_kernel;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
        return MCTP_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem) != cudaSuccess) return MCTP_ECUDA;
    per_sm = std::max(per_sm, 1);
    int64_t out_off = 0;
    for (int first = 0; first < nviews; first += kDenseViews) {
        const int cnt = std::min(kDenseViews, nviews - first);
        int64_t tiles = 0;
        for (int i = 0; i < cnt; ++i) {
            const mctp_view &w = views[first + i];
            ViewParams &V = P.view[i];
            fill_view(&sm, w, V);
            V.out_offset = out_off;
            V.tile_begin = tiles;
            tiles += int64_t(V.tiles_w) * ((w.height + kTileH - 1) / kTileH);
            out_off += int64_t(w.width) * w.height * 4;
        }
        P.nviews = cnt;
        P.total_tiles = tiles;
        const int64_t grid = std::min<int64_t>(tiles, int64_t(per_sm) * num_sms());
        kern<<<unsigned(grid), kThreads, smem, s>>>(P);
        const int rc = launch_status();
        if (rc != MCTP_OK) return rc;
    }
    return MCTP_OK;
}

}  // namespace
}  // namespace mctp

extern "C" int mctp_render_dense(const float *vol, int32_t mx, int32_t my, int32_t mz, const int64_t *src_dims,
                                 const mctp_view *views, int32_t nviews, const float *lut_rgba, int32_t nlut,
                                 float alpha_stop, float *out_rgba, uint64_t *samples_taken, void *stream)
{
    using namespace mctp;
    mctp_slicemap sm;
    int rc = dense_prepare(false, vol, mx, my, mz, src_dims, views, nviews, lut_rgba, nlut, alpha_stop, sm);
    if (rc != MCTP_OK) return rc;
    if (!out_rgba || (reinterpret_cast<uintptr_t>(out_rgba) & 15)) return MCTP_EINVAL;
    cudaStream_t s = as_stream(stream);
    if (samples_taken && cudaMemsetAsync(samples_taken, 0, sizeof(uint64_t), s) != cudaSuccess) return MCTP_ECUDA;
    if (nviews == 0) return MCTP_OK;
    return dense_launch(false, sm, vol, views, nviews, lut_rgba, nlut, alpha_stop, out_rgba, samples_taken, nullptr,
                        nullptr, nullptr, s);
}

extern "C" int mctp_render_dense_backward(const float *vol, int32_t mx, int32_t my, int32_t mz,
                                          const int64_t *src_dims, const mctp_view *views, int32_t nviews,
                                          const float *lut_rgba, int32_t nlut, float alpha_stop,
                                          const float *grad_rgba, float *grad_vol, float *grad_lut, void *stream)
{
    using namespace mctp;
    mctp_slicemap sm;
    int rc = dense_prepare(true, vol, mx, my, mz, src_dims, views, nviews, lut_rgba, nlut, alpha_stop, sm);
    if (rc != MCTP_OK) return rc;
    if (!grad_rgba || !grad_vol || !grad_lut || (reinterpret_cast<uintptr_t>(grad_rgba) & 15)) return MCTP_EINVAL;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(grad_vol, 0, size_t(mx) * my * mz * sizeof(float), s) != cudaSuccess ||
        cudaMemsetAsync(grad_lut, 0, size_t(nlut) * 4 * sizeof(float), s) != cudaSuccess)
        return MCTP_ECUDA;
    if (nviews == 0) return MCTP_OK;
    return dense_launch(true, sm, vol, views, nviews, lut_rgba, nlut, alpha_stop, nullptr, nullptr, grad_rgba,
                        grad_vol, grad_lut, s);
}

extern "C" int mctp_l2_loss(const float *x, const float *target, int64_t n, float scale, float *grad, float *loss,
                            void *stream)
{
    using namespace mctp;
    if (!x || !target || !loss || n < 0) return MCTP_EINVAL;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(loss, 0, sizeof(float), s) != cudaSuccess) return MCTP_ECUDA;
    if (n == 0) return MCTP_OK;
    const int64_t grid = std::min<int64_t>((n + 255) / 256, int64_t(num_sms()) * 8);
    l2_loss_kernel<<<unsigned(grid), 256, 0, s>>>(x, target, n, scale, grad, loss);
    return launch_status();
}

extern "C" int mctp_adam_step(float *param, const float *grad, float *m, float *v, int64_t n, float lr, float beta1,
                              float beta2, float eps, int32_t step, float lo, float hi, void *stream)
{
    using namespace mctp;
    if (!param || !grad || !m || !v || n < 0 || step < 1) return MCTP_EINVAL;
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f && lo <= hi))
        return MCTP_EINVAL;
    if (n == 0) return MCTP_OK;
    const float c1 = float(1.0 / (1.0 - pow(double(beta1), double(step))));
    const float c2 = float(1.0 / (1.0 - pow(double(beta2), double(step))));
    const int64_t grid = std::min<int64_t>((n + 255) / 256, int64_t(num_sms()) * 8);
    adam_kernel<<<unsigned(grid), 256, 0, as_stream(stream)>>>(param, grad, m, v, n, lr, beta1, beta2, eps, c1, c2, lo,
                                                               hi);
    return launch_status();
}
