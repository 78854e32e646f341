// slicemap_common.cuh -- helpers shared by the slicemap kernels.
#pragma once

#include "mctp_internal.cuh"

namespace mctp {

// Keep/discard of one grey value: mode 0 = no table, 1 = table lookup,
// 2 = step table (keep iff lo <= v < limit).
template <int kMode>
__device__ __forceinline__ uint32_t kept(uint32_t v, const uint8_t *lut, int shift, uint32_t limit, uint32_t lo)
{
    if (kMode == 0) return v;
    if (kMode == 2) return (v - lo) < (limit - lo) ? v : 0u;
    return (v < limit && lut[v >> shift]) ? v : 0u;
}

// Element (x, y, z) of a level stored as an atlas of tiles_x columns.
template <typename T>
__device__ __forceinline__ T *atlas_ptr(T *atlas, int64_t pitch, int tiles_x, int m_x, int m_y, int x, int y, int z)
{
    const int row = z / tiles_x, col = z - row * tiles_x;
    return atlas + (int64_t(row) * m_y + y) * pitch + int64_t(col) * m_x + x;
}

// Copy the keep table to shared memory and classify it: returns 0 (no
// table), 1 (general lookup) or 2 (a step keep[b] = b >= T; *lo = T << shift,
// clamped to limit).  All `nthreads` threads starting at thread `t0` call it;
// `sync` is a barrier over exactly those threads.
template <typename Sync>
__device__ int load_keep_table(const uint8_t *keep, int nbins, int shift, uint32_t limit, uint8_t *lut, int *sh,
                               int t, int nthreads, uint32_t *lo, Sync sync)
{
    if (!keep) return 0;
    if (t == 0) { sh[0] = nbins; sh[1] = 0; }
    for (int b = t; b < nbins; b += nthreads) lut[b] = keep[b];
    sync();
    for (int b = t; b < nbins; b += nthreads)
        if (lut[b]) atomicMin(&sh[0], b);
    sync();
    for (int b = t; b < nbins; b += nthreads)
        if (b >= sh[0] && !lut[b]) sh[1] = 1;
    sync();
    if (sh[1]) return 1;
    const uint64_t l = uint64_t(sh[0]) << shift;
    *lo = l >= limit ? limit : uint32_t(l);
    return 2;
}

// Replicate the top bit of bytes 1 and 3 over their 16-bit lanes.
__device__ __forceinline__ uint32_t lane_sign_mask(uint32_t t)
{
    uint32_t m;
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(m) : "r"(t));
    return m;
}

// Sum of the kept values of one 16-byte vector into the thread's accumulators.
// Packed: acc[k] holds two 16-bit lane sums of word k; otherwise acc[e] is one
// element's sum.  The packed step test assumes every lane is below 2^bits
// (<= 2^15): it ORs the words into *seen so the caller can detect a lane that
// breaks the assumption and redo the vector with add_vector_exact.
template <typename T, int kMode, bool kPacked>
__device__ __forceinline__ void add_vector(const uint4 &q, uint32_t *acc, const uint8_t *lut, int shift,
                                           uint32_t limit, uint32_t lo, uint32_t k_fast, uint32_t &seen)
{
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (kPacked) {
            uint32_t v = w[k];
            if (kMode == 2) {
                // lane: v + 0x8000 - lo has its top bit set iff v >= lo (no carry for v < 2^15)
                v &= lane_sign_mask(v + k_fast);
                seen |= w[k];
            }
            acc[k] += v;
        } else if (sizeof(T) == 1) {
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[4 * k + b] += kept<kMode>((w[k] >> (8 * b)) & 0xffu, lut, shift, limit, lo);
        } else {
            acc[2 * k] += kept<kMode>(w[k] & 0xffffu, lut, shift, limit, lo);
            acc[2 * k + 1] += kept<kMode>(w[k] >> 16, lut, shift, limit, lo);
        }
    }
}

// Exact packed step test for any lane values, without carries between lanes:
// the top bit of (v | 0x8000) - lo is (v & 0x7fff) >= lo, that of
// (v | 0x8000) - limit is (v & 0x7fff) >= limit, and a lane with its own top
// bit set is >= 2^15 >= limit.
__device__ __forceinline__ void add_vector_exact(const uint4 &q, uint32_t *acc, uint32_t k_lo2, uint32_t k_lim2)
{
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t v = w[k], vh = v | 0x80008000u;
        const uint32_t keep = (vh - k_lo2) & ~(vh - k_lim2) & ~v & 0x80008000u;
        acc[k] += v & ((keep - (keep >> 15)) | keep);
    }
}

}  // namespace mctp
