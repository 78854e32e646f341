// hist.cu -- voxel histogram (the grey-value histogram that Otsu, Alg. 1, and
// ITS, Alg. 2, partition, Sec. III-A; the top-slice histogram of the
// histogram filter, Sec. III-D).
//
// One HBM pass over the slab, read as 16-byte vectors with several loads in
// flight per thread (elements before the first 16-byte boundary and after the
// last full vector with scalar loads); each block counts into shared memory
// and adds its counts to the u64 global histogram once at the end.  Shared
// atomics of a warp that hit one bank in different words wait on one another,
// so counters are laid out per lane: with at most 256 bins every (bin, lane)
// has its own counter, in the lane's bank; with more bins that holds for a
// window of 1024 bins where most values fall, and the rest share one counter
// per bin.
#include <algorithm>

#include "mctp_internal.cuh"

namespace mctp {
namespace {

constexpr int kHistThreads = 512;
constexpr int kHistUnroll = 4;

// At most 256 bins: one counter per (bin, lane) in shared memory, bin-major
// with the lane fastest, so the 32 atomics of a warp instruction always fall
// in 32 different banks (peaked histograms, where many lanes share a bin,
// otherwise serialise).  The warps of a block share the table.
// kFull8: u8 data in 256 bins (bin = value), each byte taken with one byte
// permute.
template <typename T, bool kCheckOverflow, bool kFull8 = false>
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
        if (in_range(v >> lane_shift, nbins, kFaultHistBin)) atomicAdd(&mine[(v >> lane_shift) << 5], 1u);
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
                if (sizeof(T) == 1 && kFull8) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t v = __byte_perm(w[k], 0u, 0x4440u + b);
                        if (in_range(v, nbins, kFaultHistBin)) atomicAdd(&mine[v << 5], 1u);
                    }
                } else if (sizeof(T) == 1) {
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

// Histograms of up to kHistBatch whole volumes (at most 256 bins, one dtype)
// in one launch: the volumes' 16-byte vectors, concatenated, are split evenly
// over the blocks; a block counts its share with the per-(bin, lane) counters
// above and adds them into a volume's histogram whenever its share moves on
// to the next volume.  Elements before a volume's first 16-byte boundary or
// after its last whole vector go straight to the global histogram.
constexpr int kHistBatch = 64;
struct HistBatch {
    int32_t count, nbins, shift;
    uint32_t limit;
    unsigned long long *hist;      // [count][nbins]
    unsigned long long *overflow;  // [count]
    int64_t first[kHistBatch + 1]; // vector index of volume i's first vector in the concatenation
    const void *vol[kHistBatch];
    int64_t n[kHistBatch];         // elements
    int32_t head[kHistBatch];      // elements before the first 16-byte boundary
};

template <typename T, bool kCheckOverflow, bool kFull8>
__global__ void __launch_bounds__(kHistThreads) hist_lane_batch_kernel(const __grid_constant__ HistBatch b)
{
    extern __shared__ uint32_t sh_cols[];  // nbins * 32
    for (int i = threadIdx.x; i < b.nbins * 32; i += blockDim.x) sh_cols[i] = 0u;
    constexpr int E = 16 / sizeof(T);
    // scalar head and tail elements of volumes blockIdx.x, blockIdx.x + gridDim.x, ...
    for (int u = blockIdx.x; u < b.count; u += gridDim.x) {
        const T *base = static_cast<const T *>(b.vol[u]);
        const int64_t tail0 = b.head[u] + (b.first[u + 1] - b.first[u]) * E;
        const int64_t nscal = b.head[u] + (b.n[u] - tail0);
        for (int64_t k = threadIdx.x; k < nscal; k += blockDim.x) {
            const uint32_t v = base[k < b.head[u] ? k : tail0 + (k - b.head[u])];
            if (kCheckOverflow && v >= b.limit) atomicAdd(&b.overflow[u], 1ull);
            else if (in_range(v >> b.shift, b.nbins, kFaultHistBin))
                atomicAdd(&b.hist[int64_t(u) * b.nbins + (v >> b.shift)], 1ull);
        }
    }
    __syncthreads();
    uint32_t *mine = sh_cols + (threadIdx.x & 31);
    uint32_t ovf = 0;
    auto count = [&](uint32_t v) {
        if (kCheckOverflow && v >= b.limit) {
            ++ovf;
            return;
        }
        if (in_range(v >> b.shift, b.nbins, kFaultHistBin)) atomicAdd(&mine[(v >> b.shift) << 5], 1u);
    };
    auto count_vector = [&](const uint4 &q) {
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (sizeof(T) == 1 && kFull8) {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const uint32_t v = __byte_perm(w[k], 0u, 0x4440u + j);
                    if (in_range(v, 256, kFaultHistBin)) atomicAdd(&mine[v << 5], 1u);
                }
            } else if (sizeof(T) == 1) {
#pragma unroll
                for (int j = 0; j < 4; ++j) count((w[k] >> (8 * j)) & 0xffu);
            } else {
                count(w[k] & 0xffffu);
                count(w[k] >> 16);
            }
        }
    };
    const int64_t total = b.first[b.count];
    const int64_t per = (total + gridDim.x - 1) / gridDim.x;
    const int64_t lo = min(total, int64_t(blockIdx.x) * per), hi = min(total, lo + per);
    int v = 0;
    while (v < b.count - 1 && b.first[v + 1] <= lo) ++v;
    for (int64_t pos = lo; pos < hi; ++v) {
        const int64_t vend = min(hi, b.first[v + 1]);
        const uint4 *body = reinterpret_cast<const uint4 *>(static_cast<const T *>(b.vol[v]) + b.head[v]);
        const int64_t e = vend - b.first[v];
        int64_t i = pos - b.first[v] + threadIdx.x;
        for (; i + (kHistUnroll - 1) * int64_t(blockDim.x) < e; i += kHistUnroll * int64_t(blockDim.x)) {
            uint4 q[kHistUnroll];
#pragma unroll
            for (int u = 0; u < kHistUnroll; ++u) q[u] = ld_stream_v4(body + i + u * int64_t(blockDim.x));
#pragma unroll
            for (int u = 0; u < kHistUnroll; ++u) count_vector(q[u]);
        }
        for (; i < e; i += blockDim.x) count_vector(ld_stream_v4(body + i));
        __syncthreads();
        for (int bin = threadIdx.x; bin < b.nbins; bin += blockDim.x) {
            unsigned long long sum = 0;
            for (int l = 0; l < 32; ++l) {
                const int w = bin * 32 + ((l + bin) & 31);  // rotated: no bank conflicts
                sum += sh_cols[w];
                sh_cols[w] = 0u;
            }
            if (sum) atomicAdd(&b.hist[int64_t(v) * b.nbins + bin], sum);
        }
        if (kCheckOverflow) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ovf += __shfl_xor_sync(0xffffffffu, ovf, o);
            if ((threadIdx.x & 31) == 0 && ovf) atomicAdd(&b.overflow[v], (unsigned long long)ovf);
            ovf = 0;
        }
        __syncthreads();
        pos = vend;
    }
}

// More than 256 bins: one counter per (bin, lane) does not fit in shared
// memory for all bins, so the block keeps it for a window of 1024 bins, where
// most values fall (the grey values of a scan cluster in a narrow range), and
// one counter per bin for the rest.  In the window a lane always adds to a
// word of its own bank, so a warp's atomics never wait on one another; values
// outside it share the plain table.  Every block picks the same window: the
// 1024 bins holding the most of 8192 values sampled evenly over the slab.
// Any window gives the same counts; it only changes how fast they are made.
constexpr int kWinBins = 1024;
constexpr int kWinThreads = 1024;
constexpr int kWinUnroll = 8;
constexpr int kCoarse = 64;

template <typename T, bool kCheckOverflow>
__global__ void __launch_bounds__(kWinThreads, 1)
    hist_window_kernel(const T *__restrict__ base, int64_t n, int64_t head, int64_t nvec, int shift, uint32_t limit,
                       int nbins, unsigned long long *__restrict__ hist, unsigned long long *__restrict__ overflow)
{
    extern __shared__ uint32_t sh_win[];  // kWinBins * 32 lane columns, then nbins + 1 plain counters
    __shared__ uint32_t coarse[kCoarse];
    __shared__ int sh_lo;
    uint32_t *plain = sh_win + kWinBins * 32;
    for (int i = threadIdx.x; i < kWinBins * 32 + nbins + 1; i += blockDim.x) sh_win[i] = 0u;
    if (threadIdx.x < kCoarse) coarse[threadIdx.x] = 0u;
    __syncthreads();
    constexpr int E = 16 / sizeof(T);
    const int lane = threadIdx.x & 31;
    const int cshift = __ffs(nbins) - 1 - 6;  // coarse bin = bin >> cshift (nbins = 64 << cshift)

    // ---- the window: densest run of coarse bins in an even sample
    if (nvec > 0) {
        const int64_t at = (int64_t(threadIdx.x) * nvec) / kWinThreads;
        const uint4 q = ld_stream_v4(reinterpret_cast<const uint4 *>(base + head) + at);
        const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int b = 0; b < 4 / int(sizeof(T)); ++b) {
                const uint32_t v = sizeof(T) == 1 ? (w[k] >> (8 * b)) & 0xffu : (w[k] >> (16 * b)) & 0xffffu;
                if (!kCheckOverflow || v < limit) atomicAdd(&coarse[(v >> shift) >> cshift], 1u);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        // prefix sums over the 64 coarse bins, then the best run of `wc` of them
        const int wc = min(kCoarse, (kWinBins << 6) / nbins);
        uint32_t a = coarse[2 * lane], b = coarse[2 * lane + 1];
        uint32_t s = a + b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        // inclusive prefix P[i] = coarse[0] + ... + coarse[i]
        const uint32_t p1 = s, p0 = s - b;
        __shared__ uint32_t P[kCoarse];
        P[2 * lane] = p0;
        P[2 * lane + 1] = p1;
        __syncwarp();
        uint32_t best = 0;
        int best_c = kCoarse;  // none yet
        for (int c = lane; c + wc <= kCoarse; c += 32) {
            const uint32_t m = P[c + wc - 1] - (c > 0 ? P[c - 1] : 0u);
            if (best_c == kCoarse || m > best) {
                best = m;
                best_c = c;
            }
        }
        // the lowest start among the largest sums
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const uint32_t ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oc = __shfl_xor_sync(0xffffffffu, best_c, o);
            if (ob > best || (ob == best && oc < best_c)) {
                best = ob;
                best_c = oc;
            }
        }
        if (best_c == kCoarse) best_c = 0;
        if (lane == 0) sh_lo = best_c << cshift;
    }
    __syncthreads();
    const uint32_t lo = uint32_t(sh_lo);
    // branch-free count: values >= 2^bits go to slot nbins (the overflow), a
    // value in the window to its lane's word of the window, the rest to the
    // plain table; byte offsets into shared memory
    const uint32_t nb = uint32_t(nbins);
    uint32_t *const hot_lane = sh_win + lane;
    auto count = [&](uint32_t v) {
        uint32_t bin = v >> shift;
        if (kCheckOverflow) bin = min(bin, nb);
        const uint32_t d = bin - lo;  // wraps for bins below the window
        uint32_t *const at = d < uint32_t(kWinBins) ? hot_lane + (d << 5) : plain + bin;
        if (in_range(bin, nbins + 1, kFaultHistBin)) atomicAdd(at, 1u);
    };
    auto count_vec = [&](const uint4 &q) {
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
    };

    // ---- one pass over the slab
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthreads = int64_t(gridDim.x) * blockDim.x;
    const int64_t tail0 = head + nvec * E;
    for (int64_t i = tid; i < head; i += nthreads) count(base[i]);
    for (int64_t i = tail0 + tid; i < n; i += nthreads) count(base[i]);
    const uint4 *body = reinterpret_cast<const uint4 *>(base + head);
    int64_t i = tid;
    for (; i + (kWinUnroll - 1) * nthreads < nvec; i += kWinUnroll * nthreads) {
        uint4 q[kWinUnroll];
#pragma unroll
        for (int u = 0; u < kWinUnroll; ++u) q[u] = ld_stream_v4(body + i + u * nthreads);
#pragma unroll
        for (int u = 0; u < kWinUnroll; ++u) count_vec(q[u]);
    }
    for (; i < nvec; i += nthreads) count_vec(ld_stream_v4(body + i));
    __syncthreads();

    // ---- the block's counts into the global histogram; slot nbins is the overflow
    for (int b = threadIdx.x; b <= nbins; b += blockDim.x) {
        const uint32_t d = uint32_t(b) - lo;
        unsigned long long sum = 0;
        if (d < uint32_t(kWinBins)) {
            for (int l = 0; l < 32; ++l) sum += sh_win[(d << 5) + ((l + d) & 31)];  // rotated: no bank conflicts
        } else {
            sum = plain[b];
        }
        if (sum) atomicAdd(b < nbins ? &hist[b] : overflow, sum);
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
        else if (in_range(v >> shift, limit >> shift, kFaultHistBin)) atomicAdd(&hist[v >> shift], 1ull);
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
        auto kern = check ? hist_lane_kernel<T, true>
                          : (sizeof(T) == 1 && nbins == 256 ? hist_lane_kernel<T, false, true>
                                                            : hist_lane_kernel<T, false>);
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
    if (nbins <= 16384) {
        const size_t smem = (size_t(kWinBins) * 32 + size_t(nbins) + 1) * 4;
        int64_t head = int64_t(((16 - (addr0 & 15)) & 15) / sizeof(T));
        if (head > n) head = n;
        const int64_t nvec = (n - head) / (16 / int64_t(sizeof(T)));
        auto kern = check ? hist_window_kernel<T, true> : hist_window_kernel<T, false>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)) != cudaSuccess)
            return MCTP_ECUDA;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kWinThreads, smem) != cudaSuccess)
            return MCTP_ECUDA;
        per_sm = std::max(per_sm, 1);
        const int64_t want = (nvec + int64_t(kWinThreads) * kWinUnroll - 1) / (int64_t(kWinThreads) * kWinUnroll);
        int64_t grid = std::min<int64_t>(int64_t(per_sm) * num_sms(), std::max<int64_t>(want, 1));
        // every block counts fewer than 2^31 values, so no shared counter wraps
        grid = std::max<int64_t>(grid, (n >> 31) + 1);
        grid = std::min<int64_t>(grid, 0x7fffffff);
        kern<<<unsigned(grid), kWinThreads, smem, s>>>(base, n, head, nvec, shift, limit, nbins, h, ov);
        return launch_status();
    }
    return MCTP_EINVAL;  // not reached: nbins > 16384 takes the global kernel above
}

// Whole-volume histograms of vols[0..count) (one dtype, at most 256 bins),
// kHistBatch volumes per launch.
template <typename T>
int launch_hist_batch(const void *const *vols, const mctp_volume_desc *descs, int count, int nbins,
                      uint64_t *hist, uint64_t *overflow, cudaStream_t s)
{
    const int bits = descs[0].bits;
    const int shift = bin_shift(bits, nbins);
    const bool check = !(sizeof(T) == 1 && bits == 8) && !(sizeof(T) == 2 && bits == 16);
    auto kern = check ? hist_lane_batch_kernel<T, true, false>
                      : (sizeof(T) == 1 && nbins == 256 ? hist_lane_batch_kernel<T, false, true>
                                                        : hist_lane_batch_kernel<T, false, false>);
    const size_t smem = size_t(nbins) * 32 * 4;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kHistThreads, smem) != cudaSuccess)
        return MCTP_ECUDA;
    per_sm = std::max(per_sm, 1);
    constexpr int E = 16 / sizeof(T);
    for (int base = 0; base < count; base += kHistBatch) {
        HistBatch b{};
        b.count = std::min(kHistBatch, count - base);
        b.nbins = nbins;
        b.shift = shift;
        b.limit = bits >= 32 ? 0xffffffffu : (1u << bits);
        b.hist = reinterpret_cast<unsigned long long *>(hist + int64_t(base) * nbins);
        b.overflow = reinterpret_cast<unsigned long long *>(overflow + base);
        for (int i = 0; i < b.count; ++i) {
            const mctp_volume_desc &d = descs[base + i];
            const int64_t n = d.nx * d.ny * d.nz;
            const uintptr_t addr = reinterpret_cast<uintptr_t>(vols[base + i]);
            const int64_t head = std::min<int64_t>(int64_t(((16 - (addr & 15)) & 15) / sizeof(T)), n);
            b.vol[i] = vols[base + i];
            b.n[i] = n;
            b.head[i] = int32_t(head);
            b.first[i + 1] = b.first[i] + (n - head) / E;
        }
        const int64_t total = b.first[b.count];
        int64_t grid = std::min<int64_t>(int64_t(per_sm) * num_sms(),
                                         std::max<int64_t>((total + kHistThreads * kHistUnroll - 1) /
                                                               (kHistThreads * kHistUnroll), b.count));
        // every lane counter of a block stays below 2^31
        grid = std::max<int64_t>(grid, (total >> 36) + 1);
        grid = std::min<int64_t>(std::max<int64_t>(grid, 1), 0x7fffffff);
        kern<<<unsigned(grid), kHistThreads, smem, s>>>(b);
        const int rc = launch_status();
        if (rc != MCTP_OK) return rc;
    }
    return MCTP_OK;
}

}  // namespace

MCTP_FAULT_READER(hist)

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

extern "C" int mctp_build_histogram_batch(const void *const *vols, const mctp_volume_desc *descs, int32_t count,
                                          int32_t nbins, uint64_t *hist, uint64_t *overflow, void *stream)
{
    using namespace mctp;
    if (count < 0 || (count > 0 && (!vols || !descs || !hist || !overflow))) return MCTP_EINVAL;
    for (int i = 0; i < count; ++i) {
        const int rc = check_desc(&descs[i]);
        if (rc != MCTP_OK) return rc;
        if (!vols[i]) return MCTP_EINVAL;
        if (descs[i].dtype != descs[0].dtype || descs[i].bits != descs[0].bits) return MCTP_EINVAL;
    }
    if (count == 0) return MCTP_OK;
    if (bin_shift(descs[0].bits, nbins) < 0) return MCTP_EINVAL;
    if (int64_t(count) * nbins > (int64_t(1) << 40)) return MCTP_EINVAL;
    if (nbins > 256) {  // one launch per volume (the window kernel)
        for (int i = 0; i < count; ++i) {
            const int rc = mctp_build_histogram(vols[i], &descs[i], 0, descs[i].nz, nbins, hist + int64_t(i) * nbins,
                                                overflow + i, stream);
            if (rc != MCTP_OK) return rc;
        }
        return MCTP_OK;
    }
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(hist, 0, size_t(count) * size_t(nbins) * sizeof(uint64_t), s) != cudaSuccess ||
        cudaMemsetAsync(overflow, 0, size_t(count) * sizeof(uint64_t), s) != cudaSuccess)
        return MCTP_ECUDA;
    if (descs[0].dtype == MCTP_U8) return launch_hist_batch<uint8_t>(vols, descs, count, nbins, hist, overflow, s);
    return launch_hist_batch<uint16_t>(vols, descs, count, nbins, hist, overflow, s);
}
