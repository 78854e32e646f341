// container.cu -- container removal (Sec. III, Container Removal): the sample
// container's circle on one slice by a Hough circle transform, then every
// voxel outside it set to 0 in every slice.
//
// The cited transform (Ioannou, Huda and Laine 1999) votes for the centre
// along each edge pixel's gradient line and takes the radius from a histogram
// of edge distances.  Steps (integers unless stated; FP steps with one
// rounding per operation in a fixed order, so the result is reproducible):
//  1. smoothing by the separable [1 4 6 4 1]^2 filter, borders clamped;
//  2. Sobel gradient of the smoothed slice at interior pixels;
//  3. edge pixels: |g|^2 >= (256 thr)^2, unit gradient in FP32;
//  4. coarse centre: each edge pixel votes at (x, y) - t u for t = rmin..rmax
//     (against the gradient: the circle whose inside is darker than its rim,
//     the container's inner wall) into cells of s x s pixels; the fullest
//     cell is the centre;
//  5. coarse radius: histogram of the distances (FP64) of the edge pixels
//     whose gradient points away from the centre;
//  6. three least-squares circle fits (Kasa) over those edge pixels within a
//     band around the current circle (2s + 3, s + 3, 3 pixels), from exact
//     integer moment sums, solved by Cramer's rule in FP64 (the Hough cells
//     are s pixels wide; the fits bring the circle to sub-pixel accuracy).
// Everything after the edge detection is independent of the order in which
// edge pixels are visited (integer counts and sums, index-ordered argmax).
#include <algorithm>

#include "mctp_internal.cuh"

namespace mctp {
namespace {

constexpr int kThreads = 256;

struct Edge {
    int32_t x, y;
    float ux, uy;
};

struct HoughState {
    unsigned int nedge;
    int32_t rbest;
    int32_t valid;  // the refinement continues while 1
    int32_t pad;
    double cx, cy, rf;
    unsigned long long sums[9];  // n, sxx, sxy, sx, syy, sy, sz, sxz, syz (int64, two's complement)
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// workspace: state | smoothed slice (int32) | edge list
size_t ws_state() { return 0; }
size_t ws_blur() { return align256(sizeof(HoughState)); }
size_t ws_edges(int64_t nx, int64_t ny) { return ws_blur() + align256(size_t(nx) * size_t(ny) * sizeof(int32_t)); }
size_t ws_total(int64_t nx, int64_t ny) { return ws_edges(nx, ny) + align256(size_t(nx) * size_t(ny) * sizeof(Edge)); }

template <typename T>
__global__ void blur_kernel(const T *__restrict__ slice, int nx, int ny, int32_t *__restrict__ b)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x >= nx) return;
    const int w[5] = {1, 4, 6, 4, 1};
    int32_t acc = 0;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        const int yy = min(max(y + j - 2, 0), ny - 1);
        int32_t row = 0;
#pragma unroll
        for (int i = 0; i < 5; ++i) row += w[i] * int32_t(__ldg(slice + int64_t(yy) * nx + min(max(x + i - 2, 0), nx - 1)));
        acc += w[j] * row;
    }
    b[int64_t(y) * nx + x] = acc;
}

__global__ void edge_vote_kernel(const int32_t *__restrict__ b, int nx, int ny, long long t2, int rmin, int rmax,
                                 int s, int gxn, int gyn, unsigned int *__restrict__ acc, Edge *__restrict__ edges,
                                 HoughState *st)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    if (x < 1 || x >= nx - 1 || y < 1 || y >= ny - 1) return;
#define BV(xx, yy) (long long)b[int64_t(yy) * nx + (xx)]
    const long long gx = (BV(x + 1, y - 1) + 2 * BV(x + 1, y) + BV(x + 1, y + 1)) -
                         (BV(x - 1, y - 1) + 2 * BV(x - 1, y) + BV(x - 1, y + 1));
    const long long gy = (BV(x - 1, y + 1) + 2 * BV(x, y + 1) + BV(x + 1, y + 1)) -
                         (BV(x - 1, y - 1) + 2 * BV(x, y - 1) + BV(x + 1, y - 1));
#undef BV
    const long long g2 = gx * gx + gy * gy;
    if (g2 < t2) return;
    const float m = __fsqrt_rn(__ll2float_rn(g2));
    const float ux = __fdiv_rn(__ll2float_rn(gx), m), uy = __fdiv_rn(__ll2float_rn(gy), m);
    const unsigned int k = atomicAdd(&st->nedge, 1u);
    edges[k] = Edge{x, y, ux, uy};
    const float fs = float(s);
    for (int t = rmin; t <= rmax; ++t) {
        const float fx = __fsub_rn(float(x), __fmul_rn(float(t), ux));
        const float fy = __fsub_rn(float(y), __fmul_rn(float(t), uy));
        if (!(fx >= 0.0f && fy >= 0.0f)) continue;
        const long long ix = (long long)floorf(__fdiv_rn(fx, fs)), iy = (long long)floorf(__fdiv_rn(fy, fs));
        if (ix < gxn && iy < gyn) atomicAdd(&acc[iy * gxn + ix], 1u);
    }
}

// One block: index of the largest count (lowest index on ties).
__device__ long long block_argmax(const unsigned int *v, long long n)
{
    __shared__ unsigned int sv[32];
    __shared__ long long si[32];
    unsigned int best = 0;
    long long bi = n;  // "none yet"
    for (long long i = threadIdx.x; i < n; i += blockDim.x)
        if (bi == n || v[i] > best) { best = v[i]; bi = i; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned int ov = __shfl_xor_sync(0xffffffffu, best, o);
        const long long oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (oi < n && (bi == n || ov > best || (ov == best && oi < bi))) { best = ov; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = best; si[threadIdx.x >> 5] = bi; }
    __syncthreads();
    long long r = 0;
    if (threadIdx.x == 0) {
        best = 0;
        bi = n;
        for (int w = 0; w < int(blockDim.x >> 5); ++w)
            if (si[w] < n && (bi == n || sv[w] > best || (sv[w] == best && si[w] < bi))) { best = sv[w]; bi = si[w]; }
        r = bi == n ? 0 : bi;
    }
    return r;
}

__global__ void centre_kernel(const unsigned int *__restrict__ acc, int gxn, int gyn, int s, HoughState *st)
{
    const long long i = block_argmax(acc, (long long)gxn * gyn);
    if (threadIdx.x == 0) {
        st->cx = __dadd_rn(double((i % gxn) * s), double(s - 1) / 2.0);
        st->cy = __dadd_rn(double((i / gxn) * s), double(s - 1) / 2.0);
    }
}

// Outward edge test and distance from the current centre (FP64, fixed order).
__device__ __forceinline__ bool outward(const Edge &e, const HoughState *st, double &d)
{
    const double dx = __dsub_rn(double(e.x), st->cx), dy = __dsub_rn(double(e.y), st->cy);
    d = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    return __dadd_rn(__dmul_rn(dx, double(e.ux)), __dmul_rn(dy, double(e.uy))) > 0.0;
}

__global__ void radius_hist_kernel(const Edge *__restrict__ edges, const HoughState *st, int rmin, int rmax,
                                   unsigned int *__restrict__ rhist)
{
    const unsigned int ne = st->nedge;
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += gridDim.x * blockDim.x) {
        double d;
        if (!outward(edges[k], st, d)) continue;
        const long long r = (long long)floor(__dadd_rn(d, 0.5));
        if (r >= rmin && r <= rmax) atomicAdd(&rhist[r], 1u);
    }
}

__global__ void radius_kernel(const unsigned int *__restrict__ rhist, int rmin, int rmax, HoughState *st)
{
    const long long i = block_argmax(rhist + rmin, (long long)(rmax - rmin + 1));
    if (threadIdx.x == 0) {
        const int r = rmin + int(i);
        st->rbest = r;
        st->rf = double(r);
        st->valid = (st->nedge > 0 && rhist[r] > 0) ? 1 : 0;
        for (int k = 0; k < 9; ++k) st->sums[k] = 0ull;
    }
}

__device__ __forceinline__ unsigned long long warp_sum(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return (unsigned long long)v;
}

__global__ void fit_sums_kernel(const Edge *__restrict__ edges, HoughState *st, double band)
{
    if (!st->valid) return;
    const unsigned int ne = st->nedge;
    long long m[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (unsigned int k = blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += gridDim.x * blockDim.x) {
        const Edge e = edges[k];
        double d;
        if (!outward(e, st, d)) continue;
        if (!(fabs(__dsub_rn(d, st->rf)) <= band)) continue;
        const long long x = e.x, y = e.y, z = x * x + y * y;
        m[0] += 1; m[1] += x * x; m[2] += x * y; m[3] += x; m[4] += y * y; m[5] += y; m[6] += z;
        m[7] += x * z; m[8] += y * z;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const unsigned long long w = warp_sum(m[k]);
        if ((threadIdx.x & 31) == 0 && w) atomicAdd(&st->sums[k], w);
    }
}

// 3x3 determinant | a b c ; d e f ; g h i | expanded along the first row, in a fixed order.
__device__ __forceinline__ double det3(double a, double b, double c, double d, double e, double f, double g, double h,
                                       double i)
{
    const double m1 = __dsub_rn(__dmul_rn(e, i), __dmul_rn(f, h));
    const double m2 = __dsub_rn(__dmul_rn(d, i), __dmul_rn(f, g));
    const double m3 = __dsub_rn(__dmul_rn(d, h), __dmul_rn(e, g));
    return __dadd_rn(__dsub_rn(__dmul_rn(a, m1), __dmul_rn(b, m2)), __dmul_rn(c, m3));
}

__global__ void fit_solve_kernel(HoughState *st)
{
    if (!st->valid) return;
    long long S[9];
    for (int k = 0; k < 9; ++k) {
        S[k] = (long long)st->sums[k];
        st->sums[k] = 0ull;  // ready for the next fit
    }
    const long long n = S[0];
    if (n < 3) { st->valid = 0; return; }
    const double a11 = __ll2double_rn(S[1]), a12 = __ll2double_rn(S[2]), a13 = __ll2double_rn(S[3]);
    const double a22 = __ll2double_rn(S[4]), a23 = __ll2double_rn(S[5]), a33 = __ll2double_rn(n);
    const double b1 = -__ll2double_rn(S[7]), b2 = -__ll2double_rn(S[8]), b3 = -__ll2double_rn(S[6]);
    // the symmetric system [a11 a12 a13; a12 a22 a23; a13 a23 a33] (D, E, F) = (b1, b2, b3)
    const double det = det3(a11, a12, a13, a12, a22, a23, a13, a23, a33);
    if (det == 0.0) { st->valid = 0; return; }
    const double dD = det3(b1, a12, a13, b2, a22, a23, b3, a23, a33);
    const double dE = det3(a11, b1, a13, a12, b2, a23, a13, b3, a33);
    const double dF = det3(a11, a12, b1, a12, a22, b2, a13, a23, b3);
    const double D = __ddiv_rn(dD, det), E = __ddiv_rn(dE, det), F = __ddiv_rn(dF, det);
    const double ncx = __ddiv_rn(-D, 2.0), ncy = __ddiv_rn(-E, 2.0);
    const double rr2 = __dsub_rn(__dadd_rn(__dmul_rn(ncx, ncx), __dmul_rn(ncy, ncy)), F);
    if (!(rr2 > 0.0)) { st->valid = 0; return; }
    st->cx = ncx;
    st->cy = ncy;
    st->rf = __dsqrt_rn(rr2);
}

__global__ void finish_kernel(const HoughState *st, const unsigned int *__restrict__ rhist, int32_t *circle, double *fit)
{
    double cx = st->cx, cy = st->cy, rf = st->rf;
    if (st->nedge == 0 || rhist[st->rbest] == 0) { cx = 0.0; cy = 0.0; rf = -1.0; }
    circle[0] = int32_t(floor(__dadd_rn(cx, 0.5)));
    circle[1] = int32_t(floor(__dadd_rn(cy, 0.5)));
    circle[2] = int32_t(floor(rf));
    if (fit) { fit[0] = cx; fit[1] = cy; fit[2] = rf; }
}

// Mask: keep (x - cx)^2 + (y - cy)^2 <= r_keep^2, r_keep = max(r - margin, 0);
// no circle (r < 0): keep everything.  One element per thread, grid-stride.
template <typename T>
__global__ void mask_kernel(const T *__restrict__ in, T *__restrict__ out, int64_t nx, int64_t ny, int64_t n,
                            const int32_t *__restrict__ circle, int margin)
{
    const int32_t cx = circle[0], cy = circle[1], r = circle[2];
    const long long rk = r < 0 ? -1 : max(r - margin, 0);
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t row = i / nx, x = i - row * nx, y = row % ny;
        const long long dx = x - cx, dy = y - cy;
        const bool keep = rk < 0 || dx * dx + dy * dy <= rk * rk;
        out[i] = keep ? in[i] : T(0);
    }
}

// Vector form for 16-byte aligned data: each thread takes 16-byte chunks.
template <typename T>
__global__ void mask_vec_kernel(const T *__restrict__ in, T *__restrict__ out, int64_t nx, int64_t ny,
                                int64_t nvec, const int32_t *__restrict__ circle, int margin)
{
    constexpr int E = 16 / sizeof(T);
    const int32_t cx = circle[0], cy = circle[1], r = circle[2];
    const long long rk = r < 0 ? -1 : max(r - margin, 0);
    for (int64_t v = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; v < nvec; v += int64_t(gridDim.x) * blockDim.x) {
        union { uint4 q; T e[E]; } u;
        u.q = ld_stream_v4(in + v * E);
        if (rk >= 0) {
            int64_t i0 = v * E;
            int64_t row = i0 / nx, x = i0 - row * nx, y = row % ny;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const long long dx = x - cx, dy = y - cy;
                if (dx * dx + dy * dy > rk * rk) u.e[e] = T(0);
                if (++x == nx) { x = 0; if (++y == ny) y = 0; }
            }
        }
        st_stream_v4(out + v * E, u.q);
    }
}

}  // namespace
}  // namespace mctp

extern "C" size_t mctp_container_workspace(int64_t nx, int64_t ny)
{
    if (nx < 3 || ny < 3 || nx > (int64_t(1) << 20) || ny > (int64_t(1) << 20)) return 0;
    return mctp::ws_total(nx, ny);
}

extern "C" int mctp_find_container(const void *vol, const mctp_volume_desc *d, int64_t z, int64_t thr, int32_t rmin,
                                   int32_t rmax, int32_t cell, uint32_t *acc, uint32_t *rhist, void *workspace,
                                   size_t workspace_bytes, int32_t *circle, double *fit, void *stream)
{
    using namespace mctp;
    int rc = check_desc(d);
    if (rc != MCTP_OK) return rc;
    if (!vol || !acc || !rhist || !workspace || !circle) return MCTP_EINVAL;
    if (z < 0 || z >= d->nz || thr < 1 || thr > (int64_t(1) << 20) || rmin < 0 || rmax < rmin || cell < 1)
        return MCTP_EINVAL;
    if (d->nx < 3 || d->ny < 3 || d->nx > (int64_t(1) << 20) || d->ny > (int64_t(1) << 20)) return MCTP_EINVAL;
    if (int64_t(rmax) > 4 * std::max(d->nx, d->ny)) return MCTP_EINVAL;
    if (reinterpret_cast<uintptr_t>(workspace) & 255) return MCTP_EINVAL;
    const int nx = int(d->nx), ny = int(d->ny);
    if (workspace_bytes < ws_total(nx, ny)) return MCTP_ESIZE;
    const int gxn = (nx + cell - 1) / cell, gyn = (ny + cell - 1) / cell;
    uint8_t *ws = static_cast<uint8_t *>(workspace);
    HoughState *st = reinterpret_cast<HoughState *>(ws + ws_state());
    int32_t *b = reinterpret_cast<int32_t *>(ws + ws_blur());
    Edge *edges = reinterpret_cast<Edge *>(ws + ws_edges(nx, ny));
    cudaStream_t s = as_stream(stream);
    if (cudaMemsetAsync(st, 0, sizeof(HoughState), s) != cudaSuccess ||
        cudaMemsetAsync(acc, 0, size_t(gxn) * gyn * sizeof(uint32_t), s) != cudaSuccess ||
        cudaMemsetAsync(rhist, 0, (size_t(rmax) + 1) * sizeof(uint32_t), s) != cudaSuccess)
        return MCTP_ECUDA;
    const dim3 grid2((nx + kThreads - 1) / kThreads, ny);
    const int64_t plane = d->nx * d->ny;
    if (d->dtype == MCTP_U8)
        blur_kernel<uint8_t><<<grid2, kThreads, 0, s>>>(static_cast<const uint8_t *>(vol) + z * plane, nx, ny, b);
    else
        blur_kernel<uint16_t><<<grid2, kThreads, 0, s>>>(static_cast<const uint16_t *>(vol) + z * plane, nx, ny, b);
    const long long t2 = (256LL * thr) * (256LL * thr);
    edge_vote_kernel<<<grid2, kThreads, 0, s>>>(b, nx, ny, t2, rmin, rmax, cell, gxn, gyn,
                                                reinterpret_cast<unsigned int *>(acc), edges, st);
    centre_kernel<<<1, 1024, 0, s>>>(reinterpret_cast<const unsigned int *>(acc), gxn, gyn, cell, st);
    const int egrid = num_sms() * 4;
    radius_hist_kernel<<<egrid, kThreads, 0, s>>>(edges, st, rmin, rmax, reinterpret_cast<unsigned int *>(rhist));
    radius_kernel<<<1, 1024, 0, s>>>(reinterpret_cast<const unsigned int *>(rhist), rmin, rmax, st);
    const double bands[3] = {2.0 * cell + 3.0, double(cell) + 3.0, 3.0};
    for (int it = 0; it < 3; ++it) {
        fit_sums_kernel<<<egrid, kThreads, 0, s>>>(edges, st, bands[it]);
        fit_solve_kernel<<<1, 1, 0, s>>>(st);
    }
    finish_kernel<<<1, 1, 0, s>>>(st, reinterpret_cast<const unsigned int *>(rhist), circle, fit);
    return launch_status();
}

extern "C" int mctp_mask_container(const void *in, const mctp_volume_desc *d, const int32_t *circle, int32_t margin,
                                   void *out, void *stream)
{
    using namespace mctp;
    int rc = check_desc(d);
    if (rc != MCTP_OK) return rc;
    if (!in || !out || !circle || margin < 0) return MCTP_EINVAL;
    const int es = elem_size(d->dtype);
    const int64_t n = d->nx * d->ny * d->nz;
    const char *a = static_cast<const char *>(in);
    const char *o = static_cast<const char *>(out);
    if (a != o && a < o + n * es && o < a + n * es) return MCTP_EINVAL;  // partial overlap
    cudaStream_t s = as_stream(stream);
    const bool vec = ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15) == 0 &&
                     ((n * es) & 15) == 0;
    const int64_t grid = int64_t(num_sms()) * 8;
    if (vec) {
        const int64_t nvec = n * es / 16;
        if (d->dtype == MCTP_U8)
            mask_vec_kernel<uint8_t><<<unsigned(grid), kThreads, 0, s>>>(static_cast<const uint8_t *>(in),
                                                                          static_cast<uint8_t *>(out), d->nx, d->ny,
                                                                          nvec, circle, margin);
        else
            mask_vec_kernel<uint16_t><<<unsigned(grid), kThreads, 0, s>>>(static_cast<const uint16_t *>(in),
                                                                           static_cast<uint16_t *>(out), d->nx, d->ny,
                                                                           nvec, circle, margin);
    } else if (d->dtype == MCTP_U8) {
        mask_kernel<uint8_t><<<unsigned(grid), kThreads, 0, s>>>(static_cast<const uint8_t *>(in),
                                                                  static_cast<uint8_t *>(out), d->nx, d->ny, n, circle,
                                                                  margin);
    } else {
        mask_kernel<uint16_t><<<unsigned(grid), kThreads, 0, s>>>(static_cast<const uint16_t *>(in),
                                                                   static_cast<uint16_t *>(out), d->nx, d->ny, n,
                                                                   circle, margin);
    }
    return launch_status();
}
