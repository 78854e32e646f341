// hist.cu -- voxel histogram (the grey-value histogram that Otsu, Alg. 1, and
// ITS, Alg. 2, partition, Sec. III-A; the top-slice histogram of the
// histogram filter, Sec. III-D).
//
// One HBM pass over the slab.  Each block keeps `copies` private u32
// sub-histograms in shared memory (warp w uses copy w % copies, so warps
// rarely collide on a counter), reads the slab as 16-byte vectors with four
// loads in flight per thread, and adds its counters to the u64 global
// histogram once at the end.  With at most 256 bins the block instead keeps
// one counter per (bin, lane), which no two lanes of a warp share.  Elements before the first 16-byte boundary and
// after the last full vector are counted with scalar loads.
#include <algorithm>

#include "mctp_internal.cuh"

namespace mctp {
namespace {

constexpr int kHistThreads = 512;
constexpr int kHistUnroll = 4;

template <typename T, bool kCheckOverflow>
__device__ __forceinline__ void count_value(uint32_t v, uint32_t *sh, int shift, uint32_t limit,
                                            uint32_t &ovf)
{
    if (kCheckOverflow && v >= limit) {
        ++ovf;
        return;
    }
    atomicAdd(&sh[v >> shift], 1u);
}

template <typename T, bool kCheckOverflow>
__device__ __forceinline__ void count_vector(const uint4 &q, uint32_t *sh, int shift, uint32_t limit,
                                             uint32_t &ovf)
{
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (sizeof(T) == 1) {
#pragma unroll
            for (int b = 0; b < 4; ++b)
                count_value<T, kCheckOverflow>((w[k] >> (8 * b)) & 0xffu, sh, shift, limit, ovf);
        } else {
            count_value<T, kCheckOverflow>(w[k] & 0xffffu, sh, shift, limit, ovf);
            count_value<T, kCheckOverflow>(w[k] >> 16, sh, shift, limit, ovf);
        }
    }
}

template <typename T, bool kCheckOverflow>
__global__ void __launch_bounds__(kHistThreads)
    hist_kernel(const T *__restrict__ base, int64_t n, int64_t head, int64_t nvec, int shift,
                uint32_t limit, int nbins, int copies, unsigned long long *__restrict__ hist,
                unsigned long long *__restrict__ overflow)
{
    extern __shared__ uint32_t sh_hist[];
    for (int i = threadIdx.x; i < nbins * copies; i += blockDim.x) sh_hist[i] = 0u;
    __syncthreads();

    uint32_t *mine = sh_hist + ((threadIdx.x >> 5) % copies) * nbins;
    uint32_t ovf = 0;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthreads = int64_t(gridDim.x) * blockDim.x;
    constexpr int E = 16 / sizeof(T);

    // scalar head (before the first 16-byte boundary) and tail
    const int64_t tail0 = head + nvec * E;
    for (int64_t i = tid; i < head; i += nthreads)
        count_value<T, kCheckOverflow>(base[i], mine, shift, limit, ovf);
    for (int64_t i = tail0 + tid; i < n; i += nthreads)
        count_value<T, kCheckOverflow>(base[i], mine, shift, limit, ovf);

    // vector body
    const uint4 *body = reinterpret_cast<const uint4 *>(base + head);
    int64_t i = tid;
    for (; i + (kHistUnroll - 1) * nthreads < nvec; i += kHistUnroll * nthreads) {
        uint4 q[kHistUnroll];
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) q[u] = ld_stream_v4(body + i + u * nthreads);
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) count_vector<T, kCheckOverflow>(q[u], mine, shift, limit, ovf);
    }
    for (; i < nvec; i += nthreads) count_vector<T, kCheckOverflow>(ld_stream_v4(body + i), mine, shift, limit, ovf);

    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        uint32_t s = 0;
        for (int c = 0; c < copies; ++c) s += sh_hist[c * nbins + b];
        if (s) atomicAdd(&hist[b], (unsigned long long)s);
    }
    if (kCheckOverflow) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ovf += __shfl_xor_sync(0xffffffffu, ovf, o);
        if ((threadIdx.x & 31) == 0 && ovf) atomicAdd(overflow, (unsigned long long)ovf);
    }
}

// At most 256 bins: one counter per (bin, lane) in shared memory, bin-major
// with the lane fastest, so the 32 atomics of a warp instruction always fall
// in 32 different banks (peaked histograms, where many lanes share a bin,
// otherwise serialise).  The warps of a block share the table.
template <typename T, bool kCheckOverflow>
__global__ void __launch_bounds__(kHistThreads)
    hist_lane_kernel(const T *__restrict__ base, int64_t n, int64_t head, int64_t nvec, int shift, uint32_t limit,
                     int nbins, unsigned long long *__restrict__ hist, unsigned long long *__restrict__ overflow)
{
    extern __shared__ uint32_t sh_cols[];  // nbins * 32
    for (int i = threadIdx.x; i < nbins * 32; i += blockDim.x) sh_cols[i] = 0u;
    __syncthreads();
    uint32_t *mine = sh_cols + (threadIdx.x & 31);
    uint32_t ovf = 0;
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthreads = int64_t(gridDim.x) * blockDim.x;
    constexpr int E = 16 / sizeof(T);
    const int lane_shift = shift;  // bin = v >> shift; the column word is bin * 32
    auto count = [&](uint32_t v) {
        if (kCheckOverflow && v >= limit) {
            ++ovf;
            return;
        }
        atomicAdd(&mine[(v >> lane_shift) << 5], 1u);
    };
    const int64_t tail0 = head + nvec * E;
    for (int64_t i = tid; i < head; i += nthreads) count(base[i]);
    for (int64_t i = tail0 + tid; i < n; i += nthreads) count(base[i]);
    const uint4 *body = reinterpret_cast<const uint4 *>(base + head);
    int64_t i = tid;
    for (; i + (kHistUnroll - 1) * nthreads < nvec; i += kHistUnroll * nthreads) {
        uint4 q[kHistUnroll];
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) q[u] = ld_stream_v4(body + i + u * nthreads);
#pragma unroll
        for (int u = 0; u < kHistUnroll; ++u) {
            const uint32_t w[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (sizeof(T) == 1) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) count((w[k] >> (8 * b)) & 0xffu);
                } else {
                    count(w[k] & 0xffffu);
                    count(w[k] >> 16);
                }
            }
        }
    }
    for (; i < nvec; i += nthreads) {
        const uint4 q = ld_stream_v4(body + i);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (sizeof(T) == 1) {
#pragma unroll
                for (int b = 0; b < 4; ++b) count((w[k] >> (8 * b)) & 0xffu);
            } else {
                count(w[k] & 0xffffu);
                count(w[k] >> 16);
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) {
        unsigned long long sum = 0;  // 32 columns of up to 2^31 each
        for (int l = 0; l < 32; ++l) sum += sh_cols[b * 32 + ((l + b) & 31)];  // rotated: no bank conflicts
        if (sum) atomicAdd(&hist[b], sum);
    }
    if (kCheckOverflow) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ovf += __shfl_xor_sync(0xffffffffu, ovf, o);
        if ((threadIdx.x & 31) == 0 && ovf) atomicAdd(overflow, (unsigned long long)ovf);
    }
}

// Bins too many for shared memory (nbins > 16384): count straight into the
// global u64 histogram.
template <typename T>
__global__ void hist_global_kernel(const T *__restrict__ base, int64_t n, int shift, uint32_t limit,
                                   unsigned long long *__restrict__ hist,
                                   unsigned long long *__restrict__ overflow)
{
    const int64_t nthreads = int64_t(gridDim.x) * blockDim.x;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += nthreads) {
        uint32_t v = base[i];
        if (v >= limit) atomicAdd(overflow, 1ull);
        else atomicAdd(&hist[v >> shift], 1ull);
    }
}

template <typename T>
int launch_hist(const T *base, int64_t n, int bits, int nbins, uint64_t *hist, uint64_t *overflow,
                cudaStream_t s)
{
    const int shift = bin_shift(bits, nbins);
    const uint32_t limit = bits >= 32 ? 0xffffffffu : (1u << bits);
    const bool check = !(sizeof(T) == 1 && bits == 8) && !(sizeof(T) == 2 && bits == 16);
    auto *h = reinterpret_cast<unsigned long long *>(hist);
    auto *ov = reinterpret_cast<unsigned long long *>(overflow);
    if (nbins > 16384) {
        int grid = num_sms() * 8;
        hist_global_kernel<T><<<grid, 256, 0, s>>>(base, n, shift, limit, h, ov);
        return launch_status();
    }
    const uintptr_t addr0 = reinterpret_cast<uintptr_t>(base);
    if (nbins <= 256) {
        const size_t smem = size_t(nbins) * 32 * 4;
        int64_t head = int64_t(((16 - (addr0 & 15)) & 15) / sizeof(T));
        if (head > n) head = n;
        const int64_t nvec = (n - head) / (16 / int64_t(sizeof(T)));
        auto kern = check ? hist_lane_kernel<T, true> : hist_lane_kernel<T, false>;
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kHistThreads, smem);
        per_sm = std::max(per_sm, 1);
        int64_t want = (nvec + int64_t(kHistThreads) * kHistUnroll - 1) / (int64_t(kHistThreads) * kHistUnroll);
        int64_t grid = std::min<int64_t>(int64_t(per_sm) * num_sms(), std::max<int64_t>(want, 1));
        // every lane column stays below 2^31 counts
        grid = std::max<int64_t>(grid, (n >> 35) + 1);
        grid = std::min<int64_t>(grid, 0x7fffffff);
        kern<<<unsigned(grid), kHistThreads, smem, s>>>(base, n, head, nvec, shift, limit, nbins, h, ov);
        return launch_status();
    }
    // copies: as many private sub-histograms as fit in 32 KB, up to one per warp (more copies
    // and fewer CTAs per SM measured slower: 4096 bins, 4 copies 2.955 ms, 2 copies 2.879 ms)
    int copies = 1;
    while (copies < kHistThreads / 32 && size_t(copies * 2) * nbins * 4 <= 32768) copies *= 2;
    const size_t smem = size_t(copies) * nbins * 4;
    const uintptr_t addr = reinterpret_cast<uintptr_t>(base);
    int64_t head = int64_t(((16 - (addr & 15)) & 15) / sizeof(T));
    if (head > n) head = n;
    const int64_t nvec = (n - head) / (16 / int64_t(sizeof(T)));

    auto kern = check ? hist_kernel<T, true> : hist_kernel<T, false>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kHistThreads, smem);
    per_sm = std::max(per_sm, 1);
    int64_t want = (nvec + int64_t(kHistThreads) * kHistUnroll - 1) / (int64_t(kHistThreads) * kHistUnroll);
    int64_t grid = std::min<int64_t>(int64_t(per_sm) * num_sms(), std::max<int64_t>(want, 1));
    // keep every per-block u32 counter below 2^31
    grid = std::max<int64_t>(grid, (n >> 30) + 1);
    grid = std::min<int64_t>(grid, 0x7fffffff);
    kern<<<unsigned(grid), kHistThreads, smem, s>>>(base, n, head, nvec, shift, limit, nbins, copies, h, ov);
    return launch_status();
}

}  // namespace
}  // namespace mctp

extern "C" int mctp_build_histogram(const void *vol, const mctp_volume_desc *d, int64_t z0, int64_t z1,
                                    int32_t nbins, uint64_t *hist, uint64_t *overflow, void *stream)
{
    using namespace mctp;
    int rc = check_desc(d);
    if (rc != MCTP_OK) return rc;
    if (!vol || !hist || !overflow) return MCTP_EINVAL;
    if (z0 < 0 || z1 > d->nz || z0 > z1) return MCTP_EINVAL;
    if (bin_shift(d->bits, nbins) < 0) return MCTP_EINVAL;
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(hist, 0, size_t(nbins) * sizeof(uint64_t), s) != cudaSuccess) return MCTP_ECUDA;
    if (cudaMemsetAsync(overflow, 0, sizeof(uint64_t), s) != cudaSuccess) return MCTP_ECUDA;
    const int64_t plane = d->nx * d->ny;
    const int64_t n = (z1 - z0) * plane;
    if (n == 0) return MCTP_OK;
    if (d->dtype == MCTP_U8)
        return launch_hist(static_cast<const uint8_t *>(vol) + z0 * plane, n, d->bits, nbins, hist, overflow, s);
    return launch_hist(static_cast<const uint16_t *>(vol) + z0 * plane, n, d->bits, nbins, hist, overflow, s);
}
