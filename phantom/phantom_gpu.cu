/*
 * phantom_gpu.cu -- GPU writer of the synthetic phantom (input generator
 * only; not part of the preview library).  One block writes a brick of
 * 256 x 4 x 4 voxels; it first marks the primitives whose bounding boxes touch
 * the brick, then every voxel tests only those, in index order, so the owner
 * (and the byte written) is the one phantom_cpu.c computes.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "phantom.h"

#define PH_BX 256
#define PH_BY 4
#define PH_BZ 4
#define PH_MASK_WORDS ((PH_MAX_ELL + PH_MAX_CYL + 31) / 32)

__device__ __forceinline__ bool brick_hits(const float *lo, const float *hi, int64_t bx0, int64_t by0,
                                           int64_t bz0, int64_t bx1, int64_t by1, int64_t bz1)
{
    return !(hi[0] < (float)bx0 || lo[0] > (float)bx1 || hi[1] < (float)by0 ||
             lo[1] > (float)by1 || hi[2] < (float)bz0 || lo[2] > (float)bz1);
}

__global__ void __launch_bounds__(PH_BX) ph_kernel(const ph_params *__restrict__ P, void *out,
                                                   int64_t nbx, int64_t nby)
{
    __shared__ unsigned mask[PH_MASK_WORDS];
    const int64_t b = blockIdx.x;
    const int64_t bx = (b % nbx) * PH_BX;
    const int64_t by = ((b / nbx) % nby) * PH_BY;
    const int64_t bz = (b / (nbx * nby)) * PH_BZ;
    const int64_t nx = P->nx, ny = P->ny, nz = P->nz;
    const int64_t ex = bx + PH_BX < nx ? bx + PH_BX : nx;
    const int64_t ey = by + PH_BY < ny ? by + PH_BY : ny;
    const int64_t ez = bz + PH_BZ < nz ? bz + PH_BZ : nz;
    const int n_ell = P->n_ell, nprim = P->n_ell + P->n_cyl;
    if (threadIdx.x < PH_MASK_WORDS) mask[threadIdx.x] = 0u;
    __syncthreads();
    for (int p = threadIdx.x; p < nprim; p += blockDim.x) {
        bool hit = p < n_ell ? brick_hits(P->ell[p].lo, P->ell[p].hi, bx, by, bz, ex, ey, ez)
                             : brick_hits(P->cyl[p - n_ell].lo, P->cyl[p - n_ell].hi, bx, by, bz, ex, ey, ez);
        if (hit) atomicOr(&mask[p >> 5], 1u << (p & 31));
    }
    __syncthreads();
    const int64_t x = bx + threadIdx.x;
    if (x >= ex) return;
    const float fx = (float)x + 0.5f;
    for (int64_t z = bz; z < ez; ++z)
        for (int64_t y = by; y < ey; ++y) {
            const float fy = (float)y + 0.5f, fz = (float)z + 0.5f;
            int owner = ph_in_tube(P, fx, fy) ? -2 : -1;
            for (int w = 0; w < PH_MASK_WORDS; ++w) {
                unsigned m = mask[w];
                while (m) {
                    int p = w * 32 + __ffs(m) - 1;
                    m &= m - 1u;
                    if (p < n_ell) {
                        const ph_ellipsoid *E = &P->ell[p];
                        if (ph_in_box(E->lo, E->hi, fx, fy, fz) && ph_in_ellipsoid(E, fx, fy, fz)) owner = p;
                    } else {
                        const ph_cylinder *C = &P->cyl[p - n_ell];
                        if (ph_in_box(C->lo, C->hi, fx, fy, fz) && ph_in_cylinder(C, fx, fy, fz)) owner = p;
                    }
                }
            }
            const uint32_t v = ph_grey(P, x, y, z, owner);
            const int64_t o = (z * ny + y) * nx + x;
            if (P->esize == 1) ((uint8_t *)out)[o] = (uint8_t)v;
            else ((uint16_t *)out)[o] = (uint16_t)v;
        }
}

extern "C" int ph_params_size_gpu(void) { return (int)sizeof(ph_params); }

/* Write the whole volume described by *P_host into device memory `out`
 * (nx*ny*nz elements of esize bytes) on `stream`; blocks until done.
 * Returns 0, -1 (bad arguments) or -4 (CUDA error). */
extern "C" int ph_generate_gpu(const ph_params *P_host, void *out, void *stream)
{
    if (!P_host || !out) return -1;
    cudaStream_t s = (cudaStream_t)stream;
    ph_params *P_dev = nullptr;
    if (cudaMalloc(&P_dev, sizeof(ph_params)) != cudaSuccess) return -4;
    int rc = 0;
    if (cudaMemcpyAsync(P_dev, P_host, sizeof(ph_params), cudaMemcpyHostToDevice, s) != cudaSuccess) rc = -4;
    const int64_t nbx = (P_host->nx + PH_BX - 1) / PH_BX;
    const int64_t nby = (P_host->ny + PH_BY - 1) / PH_BY;
    const int64_t nbz = (P_host->nz + PH_BZ - 1) / PH_BZ;
    const int64_t nblocks = nbx * nby * nbz;
    if (rc == 0 && (nblocks <= 0 || nblocks > 0x7fffffffLL)) rc = -1;
    if (rc == 0) {
        ph_kernel<<<(unsigned)nblocks, PH_BX, 0, s>>>(P_dev, out, nbx, nby);
        if (cudaGetLastError() != cudaSuccess) rc = -4;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = -4;
    cudaFree(P_dev);
    return rc;
}
