// entropy.cu -- information content of rendered views (Sec. III-C, optimal
// image snapshot): the Shannon entropy H = -sum_i p_i log2 p_i (Eq. 2) of each
// image's 256-bin grey-level histogram, and the view with the largest H.
//
// Grey level of a pixel: the premultiplied RGBA render shown over black, Rec.
// 709 luminance (0.2126 R + 0.7152 G) + 0.0722 B in FP32 (one rounding per
// operation, this order), clamped to [0, 1], quantised as floor(lum*255 + 0.5).
// Histograms: per-warp shared sub-histograms, one block row per view; H in
// FP64 from the counts, one block per view, then the argmax (lowest view
// index on ties).
#include <algorithm>

#include "mctp_internal.cuh"

namespace mctp {
namespace {

constexpr int kEntThreads = 256;
constexpr int kWarps = kEntThreads / 32;
constexpr int kMaxEntViews = 65535;

__device__ __forceinline__ int grey_level(float4 p)
{
    float lum = __fadd_rn(__fadd_rn(__fmul_rn(0.2126f, p.x), __fmul_rn(0.7152f, p.y)), __fmul_rn(0.0722f, p.z));
    lum = lum < 0.0f ? 0.0f : (lum > 1.0f ? 1.0f : lum);
    if (!(lum == lum)) lum = 0.0f;
    return int(floorf(__fadd_rn(__fmul_rn(lum, 255.0f), 0.5f)));
}

constexpr int kChunk = 1024;  // views per histogram launch (offsets travel as kernel parameters)

struct HistArgs {
    const float4 *rgba;
    unsigned long long *hist;  // 256 per view, view `first` first
    int32_t first, count;
    int64_t offset[kChunk + 1];  // first pixel of each view of the chunk, then the end
};

// grid (blocks per view, views of the chunk)
__global__ void __launch_bounds__(kEntThreads) image_hist_kernel(const __grid_constant__ HistArgs A)
{
    __shared__ uint32_t sh[kWarps][256];
    for (int i = threadIdx.x; i < kWarps * 256; i += blockDim.x) (&sh[0][0])[i] = 0u;
    __syncthreads();
    const int v = blockIdx.y;
    const int64_t p0 = A.offset[v], p1 = A.offset[v + 1];
    uint32_t *mine = sh[threadIdx.x >> 5];
    for (int64_t p = p0 + int64_t(blockIdx.x) * blockDim.x + threadIdx.x; p < p1; p += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(&mine[grey_level(__ldg(A.rgba + p))], 1u);
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x) {
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) sum += sh[w][b];
        if (sum) atomicAdd(&A.hist[int64_t(A.first + v) * 256 + b], (unsigned long long)sum);
    }
}

// One block per view: H in FP64 from the view's 256 counts, one bin per
// thread, reduced in a fixed order (warp shuffles, then warps in order).
__global__ void __launch_bounds__(kEntThreads) entropy_kernel(const unsigned long long *__restrict__ hist,
                                                              double *__restrict__ H)
{
    static_assert(kEntThreads == 256, "one thread per bin");
    __shared__ unsigned long long sh_t[kWarps];
    __shared__ double sh_h[kWarps];
    const int v = blockIdx.x, b = threadIdx.x, lane = b & 31, w = b >> 5;
    const unsigned long long c = hist[int64_t(v) * 256 + b];
    unsigned long long tot = c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (lane == 0) sh_t[w] = tot;
    __syncthreads();
    tot = 0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) tot += sh_t[k];
    double term = 0.0;
    if (c) {
        const double p = __ddiv_rn(double(c), double(tot));
        term = -__dmul_rn(p, log2(p));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term = __dadd_rn(term, __shfl_xor_sync(0xffffffffu, term, o));
    if (lane == 0) sh_h[w] = term;
    __syncthreads();
    if (b == 0) {
        double sum = 0.0;
#pragma unroll
        for (int k = 0; k < kWarps; ++k) sum = __dadd_rn(sum, sh_h[k]);
        H[v] = sum;
    }
}

// The view with the largest H (lowest index on ties).
__global__ void __launch_bounds__(32) best_view_kernel(const double *__restrict__ H, int nviews, int32_t *best)
{
    double bh = -1.0;
    int bv = -1;
    for (int v = threadIdx.x; v < nviews; v += 32)
        if (H[v] > bh) { bh = H[v]; bv = v; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double oh = __shfl_xor_sync(0xffffffffu, bh, o);
        const int ov = __shfl_xor_sync(0xffffffffu, bv, o);
        if (ov >= 0 && (bv < 0 || oh > bh || (oh == bh && ov < bv))) { bh = oh; bv = ov; }
    }
    if (threadIdx.x == 0) *best = bv;
}

}  // namespace
}  // namespace mctp

extern "C" int mctp_image_entropy(const float *rgba, const mctp_view *views, int32_t nviews, uint64_t *hist,
                                  double *entropy, int32_t *best, void *stream)
{
    using namespace mctp;
    if (!rgba || (!views && nviews) || nviews < 0 || nviews > kMaxEntViews || !hist || !entropy) return MCTP_EINVAL;
    if (reinterpret_cast<uintptr_t>(rgba) & 15) return MCTP_EINVAL;
    for (int i = 0; i < nviews; ++i) {
        if (views[i].width < 1 || views[i].height < 1) return MCTP_EINVAL;
        if (int64_t(views[i].width) * views[i].height > (int64_t(1) << 28)) return MCTP_ESIZE;
    }
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(hist, 0, size_t(nviews) * 256 * sizeof(uint64_t), s) != cudaSuccess) return MCTP_ECUDA;
    if (nviews == 0) {
        if (best && cudaMemsetAsync(best, 0xff, sizeof(int32_t), s) != cudaSuccess) return MCTP_ECUDA;
        return MCTP_OK;
    }
    HistArgs A{};
    A.rgba = reinterpret_cast<const float4 *>(rgba);
    A.hist = reinterpret_cast<unsigned long long *>(hist);
    int64_t base = 0;
    for (int first = 0; first < nviews; first += kChunk) {
        const int cnt = std::min(kChunk, nviews - first);
        int64_t maxpix = 1;
        A.first = first;
        A.count = cnt;
        for (int i = 0; i <= cnt; ++i) {
            A.offset[i] = base;
            if (i < cnt) {
                const int64_t n = int64_t(views[first + i].width) * views[first + i].height;
                base += n;
                maxpix = std::max(maxpix, n);
            }
        }
        const int64_t per_view = std::min<int64_t>((maxpix + kEntThreads * 16 - 1) / (kEntThreads * 16), 1024);
        image_hist_kernel<<<dim3(unsigned(per_view), unsigned(cnt)), kEntThreads, 0, s>>>(A);
        const int rc = launch_status();
        if (rc != MCTP_OK) return rc;
    }
    entropy_kernel<<<unsigned(nviews), kEntThreads, 0, s>>>(reinterpret_cast<const unsigned long long *>(hist),
                                                             entropy);
    int rc = launch_status();
    if (rc != MCTP_OK || !best) return rc;
    best_view_kernel<<<1, 32, 0, s>>>(entropy, nviews, best);
    return launch_status();
}
