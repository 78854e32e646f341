// render_common.cuh -- the per-ray part of slicemap rendering (Sec. III-C),
// shared by the single-call renderer (render.cu) and the batched, work-queue
// renderer (render_batch.cu), so both produce the same bits for a ray.
//
// Per ray:
//  * set-up in FP32 with one rounding per operation in a fixed order (camera
//    origin, slab intersection, sample count n = floor((t_far - t_near) /
//    Delta)), so n matches any other IEEE implementation of the same steps;
//  * the level coordinate of sample k is q0 + k dq, held as 32.32 fixed-point
//    integers: dq once per view on the host (FP64), q0 once per ray in
//    float-float arithmetic (no FP64, which runs at a small fraction of the
//    FP32 rate on this part), so stepping is exact integer arithmetic and a
//    sample position is accurate to ~1e-9 voxel;
//  * trilinear interpolation of the atlas in FP32 (corner indices clamped to
//    the level), transfer-function lookup with linear interpolation,
//    premultiplied over-compositing, exit once A >= alpha_stop.
//
// Empty-space skipping: given a bitmap of the 8^3 cells whose maximum (over
// the cell plus one voxel, i.e. every voxel a sample with its lower corner in
// the cell reads) can produce a nonzero opacity under the transfer function,
// a sample whose lower corner lies in an unmarked cell has opacity exactly 0
// and adds exactly nothing to C and A.  An exact integer DDA over the cells
// gives the index of the first sample of the next cell and the march jumps
// there, so images and sample counts equal those of a full march.
#pragma once

#include <math.h>

#include <algorithm>
#include <climits>

#include "mctp_internal.cuh"

namespace mctp {
namespace render {

constexpr int kMaxLut = 4096;

// Per-view constants of the march (computed on the host by fill_view).
struct ViewParams {
    float b[3], r[3], u[3];
    float c[3], N[3];
    float L, delta;
    int32_t W, H;
    int32_t tiles_w;  // 16 x 16 image tiles along x (single-call renderer)
    int32_t level;
    float sc_hi[3], sc_lo[3];  // M_a / N_a as an unevaluated float sum
    float inv_m[3];            // 1 / |dU| (0 when dU == 0)
    float inv_d[3];            // 1 / d_a, d = -b, correctly rounded (0 when d_a == 0)
    long long dU[3];           // fixed-point step of the level coordinate per sample
    uint32_t qq[3], rr[3];     // 8 voxels (fixed point) = qq |dU| + rr (qq capped at 2^30)
    int32_t skip_ok;           // |dU| < 2^32 on every axis: the cell DDA runs in 32 bits
    int64_t out_offset;        // in floats
    int64_t tile_begin;        // first tile of this view (single-call renderer)
};

// Level geometry of the march.
struct LevelGeom {
    int32_t m1[3];   // M_a - 1
    uint32_t pitch;  // elements per atlas row
    int32_t gy;      // bitmap: cells along y
    int32_t wpr;     // bitmap: 32-bit words per (cz, cy) row
    int64_t elems;   // atlas elements of the level's tiles (bounds of the checked build)
};

template <typename T>
__device__ __forceinline__ float texel(const T *atlas, uint32_t off)
{
    return float(__ldg(atlas + off));
}

// Error-free transformations (Knuth's TwoSum; the FMA TwoProduct): a + b and
// a * b as an unevaluated sum hi + lo of two floats.
__device__ __forceinline__ void two_sum(float a, float b, float &hi, float &lo)
{
    hi = __fadd_rn(a, b);
    const float bb = __fsub_rn(hi, a);
    lo = __fadd_rn(__fsub_rn(a, __fsub_rn(hi, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float &hi, float &lo)
{
    hi = __fmul_rn(a, b);
    lo = fmaf(a, b, -hi);
}

// Fixed-point (32.32) level coordinate (o + t0 d) * sc - 1/2 of a ray's first
// sample, t0 = tn + h, in float-float arithmetic (relative error ~2^-44).
__device__ __forceinline__ long long start_coord(float o, float d, float tn, float h, float sc_hi, float sc_lo)
{
    float t_hi, t_lo, p_hi, p_lo, s_hi, s_lo, m_hi, m_lo;
    two_sum(tn, h, t_hi, t_lo);
    two_prod(t_hi, d, p_hi, p_lo);
    p_lo = fmaf(t_lo, d, p_lo);
    two_sum(o, p_hi, s_hi, s_lo);
    s_lo = __fadd_rn(s_lo, p_lo);
    two_prod(s_hi, sc_hi, m_hi, m_lo);
    m_lo = fmaf(s_hi, sc_lo, fmaf(s_lo, sc_hi, m_lo));
    return __float2ll_rn(__fmul_rn(m_hi, 4294967296.0f)) + __float2ll_rn(__fmul_rn(m_lo, 4294967296.0f)) -
           (1LL << 31);
}

// Lookup coordinate of a raw interpolated value, as the march computes it.
__device__ __forceinline__ float lut_coord(float raw, float inv_vmax, float nl1)
{
    return __fmul_rn(fminf(__fmul_rn(raw, inv_vmax), 1.0f), nl1);
}

// Largest raw grey value S such that every sample whose corners are all <= S
// has opacity exactly 0 under a transfer function whose entries 0..zmax (and
// no more) have zero opacity; -1 when none.  Corners <= S give an
// interpolated value below S + 1, whose lookup coordinate is <= that of
// S + 1; if that coordinate is <= zmax the interpolated opacity is exactly 0.
// All-zero corners interpolate to exactly 0, which is enough when entry 0 is
// zero.
__device__ inline int skip_threshold_from(int zmax, int nlut, float inv_vmax, int vmax_int)
{
    if (zmax < 0) return -1;
    const float nl1 = float(nlut - 1), zf = float(zmax);
    int lo = -1, hi = vmax_int;  // invariant: lo satisfies (or is -1), hi + 1 fails or hi is the top
    if (lut_coord(float(vmax_int) + 1.0f, inv_vmax, nl1) <= zf) return vmax_int;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (lut_coord(float(mid) + 1.0f, inv_vmax, nl1) <= zf) lo = mid;
        else hi = mid;
    }
    return lo > 0 ? lo : 0;
}

// skip_threshold_from for the transfer function `lut` (scanned serially).
__device__ inline int skip_threshold(const float4 *lut, int nlut, float inv_vmax, int vmax_int)
{
    int zmax = -1;
    while (zmax + 1 < nlut && lut[zmax + 1].w == 0.0f) ++zmax;
    return skip_threshold_from(zmax, nlut, inv_vmax, vmax_int);
}

// Bitmap word w (rows of wpr words per (cz, cy)) of the cells whose maximum
// exceeds S, from a max grid of gx cells per row.
__device__ __forceinline__ uint32_t occupancy_word(const uint16_t *maxgrid, int gx, int wpr, int w, int S)
{
    const int r = w / wpr, wx = w - r * wpr;
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b) {
        const int cx = wx * 32 + b;
        if (cx < gx && int(__ldg(maxgrid + int64_t(r) * gx + cx)) > S) bits |= 1u << b;
    }
    return bits;
}

// Table access of the march: the transfer function, the atlas offset of each
// slice and the cell bitmap, from shared memory or through the read-only
// cache.
struct SharedTables {
    static constexpr bool kGather = false;
    const float4 *lut;
    const uint32_t *slice_off;
    const uint32_t *occ;
    __device__ __forceinline__ float4 lut_at(int j) const { return lut[j]; }
    __device__ __forceinline__ uint32_t slice_at(int z) const { return slice_off[z]; }
    __device__ __forceinline__ uint32_t occ_at(int w) const { return occ[w]; }
};

template <bool kLutShared>
struct CachedTables {
    static constexpr bool kGather = false;
    const float4 *lut;
    const uint32_t *slice_off;
    const uint32_t *occ;
    __device__ __forceinline__ float4 lut_at(int j) const { return kLutShared ? lut[j] : __ldg(lut + j); }
    __device__ __forceinline__ uint32_t slice_at(int z) const { return __ldg(slice_off + z); }
    __device__ __forceinline__ uint32_t occ_at(int w) const { return __ldg(occ + w); }
};

// Atlas texture of the level (mctp_atlas_texture_*): slice_at(z) is then the
// texel x | y << 16 where slice z's tile starts inside its padded cell (every
// tile has a one-texel border repeating its edges), and the four in-slice
// corners of a sample come from one gather.
template <bool kLutShared>
struct GatherTables {
    static constexpr bool kGather = true;
    const float4 *lut;
    const uint32_t *slice_off;
    const uint32_t *occ;
    cudaTextureObject_t tex;
    __device__ __forceinline__ float4 lut_at(int j) const { return kLutShared ? lut[j] : __ldg(lut + j); }
    __device__ __forceinline__ uint32_t slice_at(int z) const { return __ldg(slice_off + z); }
    __device__ __forceinline__ uint32_t occ_at(int w) const { return __ldg(occ + w); }
};

template <typename T> struct Quad;
template <> struct Quad<uint8_t> { using type = uchar4; };
template <> struct Quad<uint16_t> { using type = ushort4; };

// Corners (ix, iy), (ix + 1, iy), (ix, iy + 1), (ix + 1, iy + 1) of the slice
// whose tile starts at texel `origin`, for ix in [-1, mx - 1] and iy in
// [-1, my - 1]: the padded cell's border holds the clamped values.  The
// gather at texel coordinate (X + 1, Y + 1) returns the 2x2 block whose lower
// corner is (X, Y), in the order (X, Y+1), (X+1, Y+1), (X+1, Y), (X, Y) (the
// bilinear footprint order of texture gathers).
template <typename T>
__device__ __forceinline__ void gather_quad(cudaTextureObject_t tex, uint32_t origin, int ix, int iy, float &v00,
                                            float &v10, float &v01, float &v11)
{
    const float gx = float(int(origin & 0xffffu) + ix + 1), gy = float(int(origin >> 16) + iy + 1);
    const typename Quad<T>::type g = tex2Dgather<typename Quad<T>::type>(tex, gx, gy, 0);
    v00 = float(g.w);
    v10 = float(g.z);
    v01 = float(g.x);
    v11 = float(g.y);
}

// Depth range of the samples of a ray that can lie in a marked cell, from the
// per-view raster of the marked cells (render_batch.cu): lo and hi are the
// float bits of depth + L, depth = <p - centre, d> along the ray; lo > hi:
// no marked cell on the ray.  Off: every sample may.
struct DepthRange {
    bool on;
    uint32_t lo, hi;
};

// FP32 set-up of one ray: origin, direction, entry distance and sample count.
struct RaySpan {
    float o[3], d[3];
    float tmin;
    int n;  // samples of the ray; 0 when it misses the box
};

// The ray of pixel (px, py) of view V, one rounding per operation in a fixed
// order (camera origin, slab intersection, n = floor((t_far - t_near) / Delta)).
__device__ __forceinline__ RaySpan ray_span(const ViewParams &V, int px, int py)
{
    RaySpan R;
    const float sx = __fsub_rn(__fdiv_rn(__fadd_rn(float(px), 0.5f), float(V.W)), 0.5f);
    const float sy = __fsub_rn(0.5f, __fdiv_rn(__fadd_rn(float(py), 0.5f), float(V.H)));
    const float sxL = __fmul_rn(sx, V.L), syL = __fmul_rn(sy, V.L);
    float tmin = -INFINITY, tmax = INFINITY;
    bool miss = false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float t1 = __fadd_rn(V.c[a], __fmul_rn(sxL, V.r[a]));
        const float t2 = __fadd_rn(t1, __fmul_rn(syL, V.u[a]));
        R.o[a] = __fadd_rn(t2, __fmul_rn(V.L, V.b[a]));
        R.d[a] = -V.b[a];
        if (R.d[a] != 0.0f) {
            const float inv = V.inv_d[a];  // = __frcp_rn(d[a]), rounded once on the host
            const float s0 = __fmul_rn(__fsub_rn(0.0f, R.o[a]), inv);
            const float s1 = __fmul_rn(__fsub_rn(V.N[a], R.o[a]), inv);
            tmin = fmaxf(tmin, fminf(s0, s1));
            tmax = fminf(tmax, fmaxf(s0, s1));
        } else if (!(R.o[a] >= 0.0f && R.o[a] <= V.N[a])) {
            miss = true;
        }
    }
    R.tmin = tmin;
    R.n = 0;
    if (!miss && tmax > tmin) R.n = int(floorf(__fdiv_rn(__fsub_rn(tmax, tmin), V.delta)));
    if (R.n < 0) R.n = 0;
    return R;
}

// Samples [k0, kend) of a ray of n > 0 samples that can reach a marked cell;
// the others have opacity exactly 0.  Sample k sits at depth
// tmin + (k + 1/2) Delta - L, so k = (depth + L - tmin) / Delta - 1/2; two
// samples of margin cover the rounding of this estimate (the raster already
// adds a voxel).  False when the ray meets no marked cell at all.
__device__ __forceinline__ bool ray_range(const ViewParams &V, const RaySpan &R, DepthRange range, int &k0,
                                          int &kend)
{
    k0 = 0;
    kend = R.n;
    if (!range.on) return true;
    if (range.lo > range.hi) return false;
    const float inv_d = 1.0f / V.delta;
    const float klo = (__uint_as_float(range.lo) - R.tmin) * inv_d - 2.5f;
    const float khi = (__uint_as_float(range.hi) - R.tmin) * inv_d + 2.5f;
    k0 = int(fminf(fmaxf(klo, 0.0f), float(R.n)));
    kend = int(fminf(fmaxf(khi, 0.0f), float(R.n - 1))) + 1;
    return true;
}

// Fixed-point level coordinates of sample k of the ray.
__device__ __forceinline__ void ray_coords(const ViewParams &V, const RaySpan &R, int k, long long U[3])
{
#pragma unroll
    for (int a = 0; a < 3; ++a)
        U[a] = start_coord(R.o[a], R.d[a], R.tmin, 0.5f * V.delta, V.sc_hi[a], V.sc_lo[a]) + (long long)k * V.dU[a];
}

// March state of one ray from its first sample that can reach a marked cell
// to its end: the fixed-point coordinates U of sample k; the exact integer
// DDA over the 8^3 cells of each sample's lower corner (cc: current cell;
// nxt[a]: the first sample index whose corner is in the next cell along axis
// a, past the ray's end for none; ee: the slack of that crossing; kmin: the
// least nxt); the compositing sums; the current slice pair's atlas offsets.
struct RayMarch {
    long long U[3];
    int k, kend, n;
    int cc[3], nxt[3];
    uint32_t ee[3];
    int kmin;
    bool occupied;
    float C0, C1, C2, A;
    int zc;               // level slice of the cached offsets (INT_MIN: none)
    uint32_t za, zb;      // texel offsets (or texture origins) of slices zc and zc + 1, clamped
    int nev;              // samples evaluated (counted only with kCount)
};

// Cell bit of cc in the bitmap.
template <class Tab>
__device__ __forceinline__ bool cell_marked(const Tab &tab, const LevelGeom &G, const int cc[3])
{
    const int w = (cc[2] * G.gy + cc[1]) * G.wpr + (cc[0] >> 5);
    if (!in_range(w, int64_t((G.m1[2] >> 3) + 1) * G.gy * G.wpr, kFaultTableRead)) return true;
    const uint32_t word = tab.occ_at(w);
    return (word >> (cc[0] & 31)) & 1u;
}

// State at sample k0 given that sample's coordinates U; with the DDA when
// `skip` (empty cells are jumped over), else every cell counts as marked.
// With m = |dU| (< 2^32) and D = 8 voxels = q m + r, the crossing after one
// at c (slack e = c m - distance, 0 <= e < m) is at c + q + (r > e), slack
// e + (r > e ? m : 0) - r.
template <class Tab>
__device__ __forceinline__ void march_begin(RayMarch &S, const ViewParams &V, const LevelGeom &G, bool skip,
                                            const Tab &tab, const long long U[3], int k0, int kend, int n)
{
    constexpr int kInf = 0x7fffffff;
    S.k = k0;
    S.kend = kend;
    S.n = n;
    S.C0 = S.C1 = S.C2 = S.A = 0.f;
    S.zc = INT_MIN;
    S.za = S.zb = 0u;
    S.nev = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        S.U[a] = U[a];
        S.cc[a] = min(max(int(U[a] >> 32), 0), G.m1[a]) >> 3;  // cell of sample k0
        S.nxt[a] = kInf;
        S.ee[a] = 0;
        const long long dU = V.dU[a];
        const int last = G.m1[a] >> 3;
        if (skip && dU != 0 && (dU > 0 ? S.cc[a] < last : S.cc[a] > 0)) {
            const long long U0 = U[a] - (long long)k0 * dU;  // coordinates of sample 0
            const long long m = dU > 0 ? dU : -dU;
            const long long num = dU > 0 ? ((long long)(8 * S.cc[a] + 8) << 32) - U0
                                         : U0 - ((long long)(8 * S.cc[a]) << 32) + 1;
            // c = ceil(num / m): float estimate, then exact correction
            const float est = float(num) * V.inv_m[a];
            if (est < float(n) + 2.0f) {
                long long c = (long long)est;
                while (c * m < num) ++c;
                while (c > 0 && (c - 1) * m >= num) --c;
                S.nxt[a] = int(c);
                S.ee[a] = uint32_t(c * m - num);
            }
        }
    }
    S.kmin = min(min(S.nxt[0], S.nxt[1]), S.nxt[2]);
    S.occupied = skip ? cell_marked(tab, G, S.cc) : true;
}

// The DDA crosses into the next cell along every axis whose crossing is at
// sample k (= kmin), and refreshes the current cell's bit.
template <class Tab>
__device__ __forceinline__ void march_cross(RayMarch &S, const ViewParams &V, const LevelGeom &G, const Tab &tab)
{
    constexpr int kInf = 0x7fffffff;
    const int k = S.kmin;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (S.nxt[a] != k) continue;
        const bool fwd = V.dU[a] > 0;
        S.cc[a] += fwd ? 1 : -1;
        if (fwd ? S.cc[a] >= (G.m1[a] >> 3) : S.cc[a] <= 0) {
            S.nxt[a] = kInf;  // the last cell this way: clamping keeps the corner in it
            continue;
        }
        const uint32_t m = uint32_t(fwd ? V.dU[a] : -V.dU[a]);
        const bool up = V.rr[a] > S.ee[a];
        S.nxt[a] = int(min(uint32_t(S.nxt[a]) + V.qq[a] + (up ? 1u : 0u), uint32_t(kInf)));
        S.ee[a] += (up ? m : 0u) - V.rr[a];
    }
    S.kmin = min(min(S.nxt[0], S.nxt[1]), S.nxt[2]);
    S.occupied = cell_marked(tab, G, S.cc);
}

// One iteration of the march: a jump over an empty cell, or one sample
// (trilinear interpolation, transfer function, compositing).  Returns true
// when the ray is finished: past its last sample that can reach a marked
// cell, or stopped early once A >= alpha_stop.
template <typename T, bool kCount, class Tab>
__device__ __forceinline__ bool march_step(RayMarch &S, const ViewParams &V, const T *atlas, const LevelGeom &G,
                                           const Tab &tab, int nlut, float inv_vmax, float alpha_stop)
{
    if (S.k >= S.kend) return true;
    if (!S.occupied) {
        // an empty cell: its samples have opacity exactly 0; jump to the
        // first sample of the next cell
        const int kn = S.kmin;
        if (kn >= S.kend) return true;
        const long long dk = (long long)(kn - S.k);
#pragma unroll
        for (int a = 0; a < 3; ++a) S.U[a] += dk * V.dU[a];
        S.k = kn;
        march_cross(S, V, G, tab);
        return false;
    }
    const int *Mm1 = G.m1;
    const int ix = int(S.U[0] >> 32), iy = int(S.U[1] >> 32), iz = int(S.U[2] >> 32);
    const float fx = float(uint32_t(S.U[0])) * 2.3283064365386963e-10f;
    const float fy = float(uint32_t(S.U[1])) * 2.3283064365386963e-10f;
    const float fz = float(uint32_t(S.U[2])) * 2.3283064365386963e-10f;
    if (iz != S.zc) {
        // the slice pair changes only when the sample's lower corner leaves its slice
        S.zc = iz;
        const int za = min(max(iz, 0), Mm1[2]), zb = min(max(iz + 1, 0), Mm1[2]);
        S.za = in_range(za, Mm1[2] + 1, kFaultTableRead) ? tab.slice_at(za) : 0u;
        S.zb = in_range(zb, Mm1[2] + 1, kFaultTableRead) ? tab.slice_at(zb) : 0u;
    }
    float v000, v100, v010, v110, v001, v101, v011, v111;
    if constexpr (Tab::kGather) {
        // a sample inside the box has its lower corner in [-1, M - 1] per axis;
        // the clamp only keeps a rounding-level excursion inside its cell
        const int gx = min(max(ix, -1), Mm1[0]), gy = min(max(iy, -1), Mm1[1]);
        gather_quad<T>(tab.tex, S.za, gx, gy, v000, v100, v010, v110);
        gather_quad<T>(tab.tex, S.zb, gx, gy, v001, v101, v011, v111);
    } else {
        const int x0 = min(max(ix, 0), Mm1[0]), y0i = min(max(iy, 0), Mm1[1]);
        const int x1 = min(max(ix + 1, 0), Mm1[0]), y1i = min(max(iy + 1, 0), Mm1[1]);
        const uint32_t pitch = G.pitch;
        const uint32_t ya = uint32_t(y0i) * pitch, yb = uint32_t(y1i) * pitch;
        v000 = in_range(int64_t(S.za + ya + x0), G.elems, kFaultAtlasRead) ? texel(atlas, S.za + ya + x0) : 0.f;
        v100 = in_range(int64_t(S.za + ya + x1), G.elems, kFaultAtlasRead) ? texel(atlas, S.za + ya + x1) : 0.f;
        v010 = in_range(int64_t(S.za + yb + x0), G.elems, kFaultAtlasRead) ? texel(atlas, S.za + yb + x0) : 0.f;
        v110 = in_range(int64_t(S.za + yb + x1), G.elems, kFaultAtlasRead) ? texel(atlas, S.za + yb + x1) : 0.f;
        v001 = in_range(int64_t(S.zb + ya + x0), G.elems, kFaultAtlasRead) ? texel(atlas, S.zb + ya + x0) : 0.f;
        v101 = in_range(int64_t(S.zb + ya + x1), G.elems, kFaultAtlasRead) ? texel(atlas, S.zb + ya + x1) : 0.f;
        v011 = in_range(int64_t(S.zb + yb + x0), G.elems, kFaultAtlasRead) ? texel(atlas, S.zb + yb + x0) : 0.f;
        v111 = in_range(int64_t(S.zb + yb + x1), G.elems, kFaultAtlasRead) ? texel(atlas, S.zb + yb + x1) : 0.f;
    }
    const float c00 = fmaf(fx, v100 - v000, v000), c10 = fmaf(fx, v110 - v010, v010);
    const float c01 = fmaf(fx, v101 - v001, v001), c11 = fmaf(fx, v111 - v011, v011);
    const float c0 = fmaf(fy, c10 - c00, c00), c1 = fmaf(fy, c11 - c01, c01);
    const float x = lut_coord(fmaf(fz, c1 - c0, c0), inv_vmax, float(nlut - 1));
    const int j = min(int(x), nlut - 2);
    const float fl = x - float(j);
    const bool lut_ok = in_range(j, nlut - 1, kFaultTableRead);
    const float4 e0 = lut_ok ? tab.lut_at(j) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 e1 = lut_ok ? tab.lut_at(j + 1) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float ca = fmaf(fl, e1.w - e0.w, e0.w);
    const float w = (1.0f - S.A) * ca;
    S.C0 = fmaf(w, fmaf(fl, e1.x - e0.x, e0.x), S.C0);
    S.C1 = fmaf(w, fmaf(fl, e1.y - e0.y, e0.y), S.C1);
    S.C2 = fmaf(w, fmaf(fl, e1.z - e0.z, e0.z), S.C2);
    S.A += w;
    ++S.k;
    if (kCount) ++S.nev;
    if (S.A >= alpha_stop) return true;
#pragma unroll
    for (int a = 0; a < 3; ++a) S.U[a] += V.dU[a];
    if (S.k == S.kmin) march_cross(S, V, G, tab);
    return S.k >= S.kend;
}

// Samples a finished ray took: all n unless it stopped early (the samples
// after its last marked cell are empty and count as taken).
__device__ __forceinline__ int march_taken(const RayMarch &S, float alpha_stop)
{
    return S.A < alpha_stop ? S.n : S.k;
}

// March the ray of pixel (px, py) of view V through a level; returns the
// premultiplied (C, A), adds the number of samples taken to `taken` and the
// number of them evaluated (not skipped as empty) to `evaluated` (kCount;
// the count costs a register in the loop).  Each adds less than 2^31; callers
// keep their 32-bit sums below 2^31 between rays (flush_count).
template <typename T, bool kCount = false, class Tab>
__device__ __forceinline__ float4 march_ray(const ViewParams &V, const T *atlas, const LevelGeom &G, bool use_skip,
                                            const Tab &tab, int nlut, float inv_vmax, float alpha_stop, int px,
                                            int py, uint32_t &taken, uint32_t &evaluated,
                                            DepthRange range = DepthRange{false, 0u, 0u})
{
    const RaySpan R = ray_span(V, px, py);
    if (R.n <= 0) return make_float4(0.f, 0.f, 0.f, 0.f);
    int k0, kend;
    if (!ray_range(V, R, range, k0, kend)) {
        taken += uint32_t(R.n);
        return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    long long U[3];
    ray_coords(V, R, k0, U);
    RayMarch S;
    march_begin(S, V, G, use_skip && V.skip_ok, tab, U, k0, kend, R.n);
    while (!march_step<T, kCount>(S, V, atlas, G, tab, nlut, inv_vmax, alpha_stop)) {
    }
    taken += uint32_t(march_taken(S, alpha_stop));
    if (kCount) evaluated += uint32_t(S.nev);
    return make_float4(S.C0, S.C1, S.C2, S.A);
}

// A per-thread 32-bit count that reached 2^31 goes to the 64-bit total (rare).
__device__ __forceinline__ void flush_count(uint32_t &count, unsigned long long *total)
{
    if (count >= 0x80000000u) {
        if (total) atomicAdd(total, (unsigned long long)count);
        count = 0;
    }
}

// The warp's 32-bit counts added to the 64-bit total by lane 0.
__device__ __forceinline__ void warp_add_count(uint32_t count, unsigned long long *total)
{
    unsigned long long t = count;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0 && t && total) atomicAdd(total, t);
}

// ---- host side

constexpr int kTileW = 16, kTileH = 16;

// Per-view constants of `w` on level w.level of `sm` (camera basis in FP64,
// rounded once to float; fixed-point step and cell-DDA constants).
inline void fill_view(const mctp_slicemap *sm, const mctp_view &w, ViewParams &V)
{
    const double PI = 3.14159265358979323846;
    const int64_t n3[3] = {sm->src_dims[0], sm->src_dims[1], sm->src_dims[2]};
    const float L = float(sqrt(double(n3[0] * n3[0] + n3[1] * n3[1] + n3[2] * n3[2])));
    const float N[3] = {float(n3[0]), float(n3[1]), float(n3[2])};
    const double az = (double(w.azimuth_deg) * PI) / 180.0;
    const double el = (double(w.elevation_deg) * PI) / 180.0;
    V.b[0] = float(cos(el) * cos(az));
    V.b[1] = float(cos(el) * sin(az));
    V.b[2] = float(sin(el));
    V.r[0] = float(-sin(az));
    V.r[1] = float(cos(az));
    V.r[2] = 0.0f;
    V.u[0] = float(-sin(el) * cos(az));
    V.u[1] = float(-sin(el) * sin(az));
    V.u[2] = float(cos(el));
    const int *M = sm->dims[w.level];
    float sa[3];
    for (int a = 0; a < 3; ++a) {
        V.N[a] = N[a];
        V.c[a] = N[a] / 2.0f;
        sa[a] = N[a] / float(M[a]);
        const double sc = double(M[a]) / double(n3[a]);
        V.sc_hi[a] = float(sc);
        V.sc_lo[a] = float(sc - double(V.sc_hi[a]));
    }
    const float smin = fminf(sa[0], fminf(sa[1], sa[2]));
    V.delta = w.step * smin;
    bool ok32 = true;
    for (int a = 0; a < 3; ++a) {
        const double sc = double(M[a]) / double(n3[a]);
        V.dU[a] = llrint(double(V.delta) * double(-V.b[a]) * sc * 4294967296.0);
        const long long m = V.dU[a] < 0 ? -V.dU[a] : V.dU[a];
        V.inv_m[a] = m ? float(1.0 / double(m)) : 0.0f;
        const float da = -V.b[a];
        V.inv_d[a] = da != 0.0f ? 1.0f / da : 0.0f;  // IEEE single division: the device's __frcp_rn(da)
        const long long q = m ? (8LL << 32) / m : 0;
        V.qq[a] = uint32_t(std::min<long long>(q, 1LL << 30));
        V.rr[a] = uint32_t(m ? (8LL << 32) - q * m : 0);
        if (m >= (1LL << 32)) ok32 = false;
    }
    V.skip_ok = ok32 ? 1 : 0;
    V.L = L;
    V.W = w.width;
    V.H = w.height;
    V.level = w.level;
    V.tiles_w = (w.width + kTileW - 1) / kTileW;
    V.out_offset = 0;
    V.tile_begin = 0;
}

// Argument checks shared by the renderers: a view on level `w.level` of a
// slicemap with `nlevels` levels.
inline int check_view(const mctp_view &w, int nlevels)
{
    if (w.width < 1 || w.height < 1 || w.level < 0 || w.level >= nlevels) return MCTP_EINVAL;
    if (!(w.step >= 1.0f / 256.0f && w.step <= 64.0f)) return MCTP_EINVAL;
    if (int64_t(w.width) * w.height > (int64_t(1) << 28)) return MCTP_ESIZE;
    return MCTP_OK;
}

// A level's atlas must be addressable with 32-bit texel offsets.
inline bool level_fits_32bit(const mctp_slicemap *sm, int k)
{
    return int64_t(sm->tiles_x[k]) * sm->dims[k][0] * int64_t(sm->tiles_y[k]) * sm->dims[k][1] <=
           (int64_t(1) << 32);
}

}  // namespace render
}  // namespace mctp
