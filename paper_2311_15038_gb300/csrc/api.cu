// api.cu -- small utility entry points of libmctp (version, status strings,
// atlas geometry).
#include "mctp_internal.cuh"

extern "C" int mctp_version(void) { return MCTP_ABI_VERSION; }

extern "C" const char *mctp_status_string(int code)
{
    switch (code) {
    case MCTP_OK: return "ok";
    case MCTP_EINVAL: return "invalid argument";
    case MCTP_EUNSUPPORTED: return "unsupported dtype, bit depth, mode or size";
    case MCTP_ESIZE: return "size limit exceeded (atlas tile grid, view size)";
    case MCTP_ECUDA: return "CUDA launch or copy failed";
    case MCTP_ECANCELED: return "request cancelled before its launch";
    default: return "unknown status";
    }
}

// Atlas grid of a level with mz slices: tiles_x = 2^ceil(log2 sqrt(mz)),
// tiles_y = ceil(mz / tiles_x).
extern "C" int mctp_default_tiles(int32_t mz, int32_t *tiles_x, int32_t *tiles_y)
{
    if (mz < 1 || !tiles_x || !tiles_y) return MCTP_EINVAL;
    int64_t tx = 1;
    while (tx * tx < mz) tx *= 2;
    *tiles_x = int32_t(tx);
    *tiles_y = int32_t((mz + tx - 1) / tx);
    return MCTP_OK;
}

extern "C" size_t mctp_atlas_bytes(int32_t mx, int32_t my, int32_t tiles_x, int32_t tiles_y, int32_t dtype)
{
    const int es = mctp::elem_size(dtype);
    if (mx < 1 || my < 1 || tiles_x < 1 || tiles_y < 1 || es == 0) return 0;
    return size_t(tiles_x) * mx * size_t(tiles_y) * my * es;
}

extern "C" size_t mctp_maxgrid_bytes(int32_t mx, int32_t my, int32_t mz)
{
    if (mx < 1 || my < 1 || mz < 1) return 0;
    const size_t c = MCTP_MAXGRID_CELL;
    return ((size_t(mx) + c - 1) / c) * ((size_t(my) + c - 1) / c) * ((size_t(mz) + c - 1) / c) * sizeof(uint16_t);
}

// ---- checked build (MCTP_CHECKED): index faults recorded by the kernels
namespace mctp {
int fault_word_hist(uint32_t *bits, bool reset);
int fault_word_threshold(uint32_t *bits, bool reset);
int fault_word_slicemap(uint32_t *bits, bool reset);
int fault_word_render(uint32_t *bits, bool reset);
int fault_word_render_batch(uint32_t *bits, bool reset);
MCTP_FAULT_READER(api)
namespace {
// Records the self-test bit through the same check the kernels use (an index
// outside a 3-element extent); nothing is read or written.
__global__ void checked_selftest_kernel()
{
    if (threadIdx.x == 0 && blockIdx.x == 0) (void)in_range(5, 3, kFaultSelfTest);
}
}  // namespace
}  // namespace mctp

extern "C" int mctp_checked_build(void)
{
#ifdef MCTP_CHECKED
    return 1;
#else
    return 0;
#endif
}

extern "C" int mctp_checked_status(uint32_t *bits, int32_t reset)
{
    using namespace mctp;
    if (!bits) return MCTP_EINVAL;
    *bits = 0;
    if (!mctp_checked_build()) return MCTP_EUNSUPPORTED;
    int (*const readers[])(uint32_t *, bool) = {fault_word_hist, fault_word_threshold, fault_word_slicemap,
                                                fault_word_render, fault_word_render_batch, fault_word_api};
    for (auto f : readers) {
        const int rc = f(bits, reset != 0);
        if (rc != MCTP_OK) return rc;
    }
    return MCTP_OK;
}

extern "C" int mctp_checked_selftest(void *stream)
{
    if (!mctp_checked_build()) return MCTP_EUNSUPPORTED;
    mctp::checked_selftest_kernel<<<1, 32, 0, mctp::as_stream(stream)>>>();
    return mctp::launch_status();
}
