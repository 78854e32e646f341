// threshold.cu -- threshold selection (Otsu, Alg. 1; iterative threshold
// selection, Alg. 2; top-slice histogram filtering, Sec. III-D) and the
// binary keep/discard classification of voxels (Sec. III-A).
//
// Selection runs in one 1024-thread block.  Class sizes and grey-value sums
// are exact u64 prefix sums; every floating-point step is FP64 with explicit
// round-to-nearest intrinsics (no fused multiply-add) in a fixed order, so the
// chosen threshold does not depend on the reduction order.
#include <math.h>

#include <algorithm>

#include "mctp_internal.cuh"

namespace mctp {
namespace {

constexpr int kSelThreads = 1024;

struct BlockScratch {
    unsigned long long a[32];
    unsigned long long b[32];
    double d[32];
    int t[32];
    unsigned long long bc[4];
    double bd[4];
};

// Block-wide sum of two u64 values; every thread gets the totals.
__device__ void block_sum2(unsigned long long &x, unsigned long long &y, BlockScratch &sc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        y += __shfl_xor_sync(0xffffffffu, y, o);
    }
    __syncthreads();
    if (lane == 0) { sc.a[warp] = x; sc.b[warp] = y; }
    __syncthreads();
    if (warp == 0) {
        unsigned long long p = lane < (int)(blockDim.x >> 5) ? sc.a[lane] : 0ull;
        unsigned long long q = lane < (int)(blockDim.x >> 5) ? sc.b[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            p += __shfl_xor_sync(0xffffffffu, p, o);
            q += __shfl_xor_sync(0xffffffffu, q, o);
        }
        if (lane == 0) { sc.bc[0] = p; sc.bc[1] = q; }
    }
    __syncthreads();
    x = sc.bc[0];
    y = sc.bc[1];
}

// Block-wide exclusive prefix sum of two u64 values (thread order), plus totals.
__device__ void block_exscan2(unsigned long long &x, unsigned long long &y, unsigned long long &tx,
                              unsigned long long &ty, BlockScratch &sc)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long ix = x, iy = y;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long vx = __shfl_up_sync(0xffffffffu, ix, o);
        unsigned long long vy = __shfl_up_sync(0xffffffffu, iy, o);
        if (lane >= o) { ix += vx; iy += vy; }
    }
    __syncthreads();
    if (lane == 31) { sc.a[warp] = ix; sc.b[warp] = iy; }
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long px = lane < nw ? sc.a[lane] : 0ull;
        unsigned long long py = lane < nw ? sc.b[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long vx = __shfl_up_sync(0xffffffffu, px, o);
            unsigned long long vy = __shfl_up_sync(0xffffffffu, py, o);
            if (lane >= o) { px += vx; py += vy; }
        }
        sc.a[lane] = px;   // inclusive over warps
        sc.b[lane] = py;
    }
    __syncthreads();
    const unsigned long long wx = warp > 0 ? sc.a[warp - 1] : 0ull;
    const unsigned long long wy = warp > 0 ? sc.b[warp - 1] : 0ull;
    tx = sc.a[(blockDim.x >> 5) - 1];
    ty = sc.b[(blockDim.x >> 5) - 1];
    x = wx + ix - x;
    y = wy + iy - y;
    __syncthreads();
}

// Otsu's between-class variance for the split [0,T) | [T,nbins); the FP64
// order is part of the definition: Wa = na/N, Wb = nb/N, Ua = Sa/na,
// Ub = Sb/nb, d = Ua - Ub, sigma = ((Wa*Wb)*d)*d.
__device__ __forceinline__ double otsu_sigma(unsigned long long N, unsigned long long na,
                                             unsigned long long nb, unsigned long long Sa,
                                             unsigned long long Sb)
{
    const double Nd = __ull2double_rn(N);
    const double dna = __ull2double_rn(na), dnb = __ull2double_rn(nb);
    const double Wa = __ddiv_rn(dna, Nd);
    const double Wb = __ddiv_rn(dnb, Nd);
    const double Ua = __ddiv_rn(__ull2double_rn(Sa), dna);
    const double Ub = __ddiv_rn(__ull2double_rn(Sb), dnb);
    const double d = __dsub_rn(Ua, Ub);
    return __dmul_rn(__dmul_rn(__dmul_rn(Wa, Wb), d), d);
}

__global__ void __launch_bounds__(kSelThreads)
    select_kernel(const unsigned long long *__restrict__ hist, int nbins, mctp_thr_params p,
                  uint8_t *__restrict__ keep, int32_t *__restrict__ result)
{
    __shared__ BlockScratch sc;
    __shared__ int sh_T;
    const int tid = threadIdx.x;
    // block i selects for histogram i of a batch (a single call launches one block)
    if (hist) hist += int64_t(blockIdx.x) * nbins;
    keep += int64_t(blockIdx.x) * nbins;
    if (result) result += 4 * int64_t(blockIdx.x);
    int T = 0, iters = 0, converged = 1;

    if (p.mode == MCTP_THR_EXPLICIT) {
        T = p.explicit_T;
    } else if (p.mode == MCTP_THR_TOPSLAB) {
        for (int b = tid; b < nbins; b += blockDim.x) keep[b] = hist[b] < p.topslab_kmin ? 1 : 0;
        if (tid == 0 && result) { result[0] = -1; result[1] = 0; result[2] = 1; result[3] = 0; }
        return;
    } else {
        // totals N = sum h, S = sum b h (exact)
        unsigned long long n = 0, S = 0;
        for (int b = tid; b < nbins; b += blockDim.x) {
            const unsigned long long h = hist[b];
            n += h;
            S += (unsigned long long)b * h;
        }
        block_sum2(n, S, sc);
        const unsigned long long N = n, Stot = S;

        if (p.mode == MCTP_THR_OTSU) {
            double best = 0.0;
            int bestT = 0x7fffffff;
            unsigned long long cn = 0, cs = 0;
            for (int base = 0; base < nbins; base += blockDim.x) {
                const int b = base + tid;
                unsigned long long h = b < nbins ? hist[b] : 0ull;
                unsigned long long x = h, y = (unsigned long long)b * h, tx, ty;
                block_exscan2(x, y, tx, ty, sc);
                const unsigned long long na = cn + x, Sa = cs + y;
                if (b < nbins) {
                    const unsigned long long nb = N - na, Sb = Stot - Sa;
                    if (na != 0ull && nb != 0ull) {
                        const double sigma = otsu_sigma(N, na, nb, Sa, Sb);
                        if (sigma > best) { best = sigma; bestT = b; }
                    }
                }
                cn += tx;
                cs += ty;
            }
            // arg max, ties to the lowest T (the sweep keeps the first strict maximum)
            const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int ot = __shfl_xor_sync(0xffffffffu, bestT, o);
                if (ob > best || (ob == best && ot < bestT)) { best = ob; bestT = ot; }
            }
            if (lane == 0) { sc.d[warp] = best; sc.t[warp] = bestT; }
            __syncthreads();
            if (warp == 0) {
                const int nw = blockDim.x >> 5;
                best = lane < nw ? sc.d[lane] : 0.0;
                bestT = lane < nw ? sc.t[lane] : 0x7fffffff;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                    const int ot = __shfl_xor_sync(0xffffffffu, bestT, o);
                    if (ob > best || (ob == best && ot < bestT)) { best = ob; bestT = ot; }
                }
                if (lane == 0) sh_T = best > 0.0 ? bestT : 0;
            }
            __syncthreads();
            T = sh_T;
        } else {  // MCTP_THR_ITS
            double T_it = __ddiv_rn((double)nbins, 2.0);
            double r = T_it;
            while (r != 0.0 && iters < p.its_max_iter) {
                const double c = ceil(T_it);
                const long long m = c < 0.0 ? 0 : (c > (double)nbins ? nbins : (long long)c);
                unsigned long long n1 = 0, S1 = 0;
                for (int b = tid; b < m; b += blockDim.x) {
                    const unsigned long long h = hist[b];
                    n1 += h;
                    S1 += (unsigned long long)b * h;
                }
                block_sum2(n1, S1, sc);
                const unsigned long long n2 = N - n1, S2 = Stot - S1;
                const double mu1 = n1 ? __ddiv_rn(__ull2double_rn(S1), __ull2double_rn(n1)) : T_it;
                const double mu2 = n2 ? __ddiv_rn(__ull2double_rn(S2), __ull2double_rn(n2)) : T_it;
                const double T_tmp = __ddiv_rn(__dadd_rn(mu1, mu2), 2.0);
                r = fabs(__dsub_rn(T_it, T_tmp));
                T_it = T_tmp;
                ++iters;
            }
            converged = (r == 0.0);
            const double c = ceil(T_it);
            T = (int)(c < 0.0 ? 0.0 : (c > (double)nbins ? (double)nbins : c));
        }
    }
    for (int b = tid; b < nbins; b += blockDim.x) keep[b] = b >= T ? 1 : 0;
    if (tid == 0 && result) { result[0] = T; result[1] = iters; result[2] = converged; result[3] = 0; }
}

// ------------------------------------------------------------------ filter

template <typename T>
__device__ __forceinline__ uint32_t keep_value(uint32_t v, const uint8_t *lut, int shift, uint32_t limit)
{
    return (v < limit && in_range(v >> shift, limit >> shift, kFaultKeepRead) && lut[v >> shift]) ? v : 0u;
}

template <typename T>
__global__ void __launch_bounds__(256)
    filter_kernel(const T *in, T *out, int64_t n, int64_t head, int64_t nvec,
                  const uint8_t *__restrict__ keep, int nbins, int shift, uint32_t limit)
{
    extern __shared__ uint8_t sh_keep[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh_keep[b] = keep[b];
    __syncthreads();
    const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthreads = int64_t(gridDim.x) * blockDim.x;
    constexpr int E = 16 / sizeof(T);
    const int64_t tail0 = head + nvec * E;
    for (int64_t i = tid; i < head; i += nthreads) out[i] = (T)keep_value<T>(in[i], sh_keep, shift, limit);
    for (int64_t i = tail0 + tid; i < n; i += nthreads) out[i] = (T)keep_value<T>(in[i], sh_keep, shift, limit);
    const uint4 *src = reinterpret_cast<const uint4 *>(in + head);
    uint4 *dst = reinterpret_cast<uint4 *>(out + head);
    for (int64_t i = tid; i < nvec; i += 2 * nthreads) {
        uint4 q[2];
        const bool second = i + nthreads < nvec;
        q[0] = ld_stream_v4(src + i);
        if (second) q[1] = ld_stream_v4(src + i + nthreads);
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (u == 1 && !second) break;
            uint32_t w[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint32_t r = 0;
                if (sizeof(T) == 1) {
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        r |= keep_value<T>((w[k] >> (8 * b)) & 0xffu, sh_keep, shift, limit) << (8 * b);
                } else {
                    r = keep_value<T>(w[k] & 0xffffu, sh_keep, shift, limit) |
                        (keep_value<T>(w[k] >> 16, sh_keep, shift, limit) << 16);
                }
                w[k] = r;
            }
            st_stream_v4(dst + i + u * nthreads, make_uint4(w[0], w[1], w[2], w[3]));
        }
    }
}

template <typename T>
int launch_filter(const T *in, T *out, int64_t n, const uint8_t *keep, int nbins, int bits, cudaStream_t s)
{
    const int shift = bin_shift(bits, nbins);
    const uint32_t limit = 1u << bits;
    const uintptr_t ai = reinterpret_cast<uintptr_t>(in), ao = reinterpret_cast<uintptr_t>(out);
    int64_t head, nvec;
    if ((ai & 15) == (ao & 15)) {
        head = int64_t(((16 - (ai & 15)) & 15) / sizeof(T));
        if (head > n) head = n;
        nvec = (n - head) / (16 / int64_t(sizeof(T)));
    } else {  // different misalignment: scalar path only
        head = n;
        nvec = 0;
    }
    const size_t smem = size_t(nbins);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(filter_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    int64_t want = (std::max<int64_t>(nvec, head) + 511) / 512;
    int64_t grid = std::min<int64_t>(int64_t(num_sms()) * 8, std::max<int64_t>(want, 1));
    filter_kernel<T><<<unsigned(grid), 256, smem, s>>>(in, out, n, head, nvec, keep, nbins, shift, limit);
    return launch_status();
}

}  // namespace

MCTP_FAULT_READER(threshold)

}  // namespace mctp

namespace mctp {
namespace {
int check_select(const uint64_t *hist, int32_t nbins, const mctp_thr_params *p, const uint8_t *keep_lut,
                 bool need_buffers = true)
{
    if (!p || (need_buffers && !keep_lut)) return MCTP_EINVAL;
    if (nbins < 1 || nbins > 65536 || log2_exact(nbins) < 0) return MCTP_EINVAL;
    if (p->mode < MCTP_THR_OTSU || p->mode > MCTP_THR_EXPLICIT) return MCTP_EUNSUPPORTED;
    if (need_buffers && p->mode != MCTP_THR_EXPLICIT && !hist) return MCTP_EINVAL;
    if (p->mode == MCTP_THR_ITS && p->its_max_iter < 1) return MCTP_EINVAL;
    if (p->mode == MCTP_THR_TOPSLAB && p->topslab_kmin < 1) return MCTP_EINVAL;
    return MCTP_OK;
}
}  // namespace
}  // namespace mctp

extern "C" int mctp_select_threshold(const uint64_t *hist, int32_t nbins, const mctp_thr_params *p,
                                     uint8_t *keep_lut, int32_t *result, void *stream)
{
    return mctp_select_threshold_batch(hist, 1, nbins, p, keep_lut, result, stream);
}

extern "C" int mctp_select_threshold_batch(const uint64_t *hist, int32_t count, int32_t nbins,
                                           const mctp_thr_params *p, uint8_t *keep_lut, int32_t *result,
                                           void *stream)
{
    using namespace mctp;
    const int rc = check_select(hist, nbins, p, keep_lut, count != 0);
    if (rc != MCTP_OK) return rc;
    if (count < 0 || int64_t(count) * nbins > (int64_t(1) << 31)) return MCTP_EINVAL;
    if (count == 0) return MCTP_OK;
    select_kernel<<<unsigned(count), kSelThreads, 0, as_stream(stream)>>>(
        reinterpret_cast<const unsigned long long *>(hist), nbins, *p, keep_lut, result);
    return launch_status();
}

extern "C" int mctp_filter_threshold(const void *in, const mctp_volume_desc *d, const uint8_t *keep_lut,
                                     int32_t nbins, void *out, void *stream)
{
    using namespace mctp;
    int rc = check_desc(d);
    if (rc != MCTP_OK) return rc;
    if (!in || !out || !keep_lut) return MCTP_EINVAL;
    if (bin_shift(d->bits, nbins) < 0) return MCTP_EINVAL;
    const int64_t n = d->nx * d->ny * d->nz;
    const size_t bytes = size_t(n) * elem_size(d->dtype);
    const char *pi = static_cast<const char *>(in);
    const char *po = static_cast<const char *>(out);
    if (pi != po && pi < po + bytes && po < pi + bytes) return MCTP_EINVAL;  // partial overlap
    cudaStream_t s = as_stream(stream);
    if (d->dtype == MCTP_U8)
        return launch_filter(static_cast<const uint8_t *>(in), static_cast<uint8_t *>(out), n, keep_lut, nbins,
                             d->bits, s);
    return launch_filter(static_cast<const uint16_t *>(in), static_cast<uint16_t *>(out), n, keep_lut, nbins,
                         d->bits, s);
}
