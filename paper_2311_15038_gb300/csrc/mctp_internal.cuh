// mctp_internal.cuh -- helpers shared by the libmctp translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "mctp.h"

namespace mctp {

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// ---- checked build
// Compiled with MCTP_CHECKED (the second library the build makes for tests),
// the kernels test their main indices against the extent of the buffer they
// address.  An index outside records a bit in a device status word of its
// translation unit and the access is skipped: nothing traps and nothing is
// read or written out of range.  In the normal build the test is the constant
// true and costs nothing.
enum : unsigned {
    kFaultHistBin = 1u,      // a histogram bin (shared or global counters)
    kFaultAtlasWrite = 4u,   // a slicemap atlas element written
    kFaultAtlasRead = 8u,    // an atlas element read by a march
    kFaultTableRead = 16u,   // a transfer-function entry, slice offset or bitmap word
    kFaultImageWrite = 32u,  // a pixel of an output image
    kFaultKeepRead = 64u,    // a keep-table entry
    kFaultSelfTest = 0x80000000u,
};
#ifdef MCTP_CHECKED
static __device__ unsigned int g_fault_word;
__device__ __forceinline__ bool in_range(long long i, long long n, unsigned bit)
{
    if (i >= 0 && i < n) return true;
    atomicOr(&g_fault_word, bit);
    return false;
}
// This translation unit's fault word (waits for the device), cleared on request.
static inline int tu_fault_word(uint32_t *bits, bool reset)
{
    unsigned int v = 0;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpyFromSymbol(&v, g_fault_word, sizeof(v)) != cudaSuccess)
        return MCTP_ECUDA;
    *bits |= v;
    if (reset) {
        const unsigned int z = 0;
        if (cudaMemcpyToSymbol(g_fault_word, &z, sizeof(z)) != cudaSuccess) return MCTP_ECUDA;
    }
    return MCTP_OK;
}
#define MCTP_FAULT_READER(name) \
    int fault_word_##name(uint32_t *bits, bool reset) { return tu_fault_word(bits, reset); }
#else
__device__ __forceinline__ constexpr bool in_range(long long, long long, unsigned) { return true; }
#define MCTP_FAULT_READER(name) \
    int fault_word_##name(uint32_t *, bool) { return MCTP_OK; }
#endif

inline int log2_exact(int64_t v)
{
    if (v <= 0 || (v & (v - 1)) != 0) return -1;
    int k = 0;
    while ((int64_t(1) << k) < v) ++k;
    return k;
}

inline int elem_size(int32_t dtype) { return dtype == MCTP_U8 ? 1 : (dtype == MCTP_U16 ? 2 : 0); }

// MCTP_OK when dtype/bits describe a supported voxel type.
inline int check_type(int32_t dtype, int32_t bits)
{
    if (dtype == MCTP_U8) return bits == 8 ? MCTP_OK : MCTP_EUNSUPPORTED;
    if (dtype == MCTP_U16) return (bits >= 1 && bits <= 16) ? MCTP_OK : MCTP_EUNSUPPORTED;
    return MCTP_EUNSUPPORTED;
}

inline int check_desc(const mctp_volume_desc *d)
{
    if (!d) return MCTP_EINVAL;
    int rc = check_type(d->dtype, d->bits);
    if (rc != MCTP_OK) return rc;
    if (d->nx < 1 || d->ny < 1 || d->nz < 1) return MCTP_EINVAL;
    if (d->nx > (int64_t(1) << 31) || d->ny > (int64_t(1) << 31) || d->nz > (int64_t(1) << 31))
        return MCTP_EINVAL;
    return MCTP_OK;
}

// Shift from a grey value to its bin, or -1 when nbins is not allowed.
inline int bin_shift(int32_t bits, int32_t nbins)
{
    int lb = log2_exact(nbins);
    if (lb < 0 || lb > bits) return -1;
    return bits - lb;
}

inline int launch_status()
{
    return cudaGetLastError() == cudaSuccess ? MCTP_OK : MCTP_ECUDA;
}

// SMs of the current device, queried once per device (grid sizes are
// multiples of it); 1 if the query fails, which keeps every launch valid.
inline int num_sms()
{
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < 64 && cached[dev] > 0) return cached[dev];
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) return 1;
    if (dev < 64) cached[dev] = v;
    return v;
}

// Depth bounds of render_batch_impl: off, on (the workspace must hold them),
// or on when the workspace has room for them.
constexpr int kBoundsOff = 0, kBoundsOn = 1, kBoundsIfRoom = 2;

// mctp_render_batch with optional per-view output offsets (render_batch.cu).
int render_batch_impl(const mctp_slicemap *sms, int32_t nsm, const mctp_view *views, const int32_t *view_slicemap,
                      const int32_t *view_lut, int32_t nviews, const float *luts_rgba, int32_t nluts, int32_t nlut,
                      float alpha_stop, const mctp_batch_tuning *tuning, float *out_rgba, const int64_t *out_offsets,
                      uint64_t *samples_taken, void *workspace, size_t workspace_bytes, cudaStream_t s,
                      int depth_bounds);

// Upper bound of the batch workspace over batches of at most max_views views,
// with room for the depth bounds of views of up to 1024 x 1024 pixels.
size_t batch_workspace_bound(const mctp_slicemap *sms, int32_t nsm, int32_t max_views);

// 16-byte streaming load that bypasses L1 allocation (data read once).
__device__ __forceinline__ uint4 ld_stream_v4(const void *p)
{
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ void st_stream_v4(void *p, uint4 v)
{
    asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

}  // namespace mctp
