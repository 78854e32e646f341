/*
 * phantom.h -- seeded synthetic micro-CT volumes (input generator only).
 *
 * This module holds none of the preview method's arithmetic: it only writes
 * test and benchmark inputs.  A CPU build (phantom_cpu.c) and a GPU build
 * (phantom_gpu.cu) include the per-voxel definition below and write identical
 * bytes for the same parameters.
 *
 * Volume model (shaped like the paper's arthropod scans: an object in the
 * lower part of a container, surroundings in the top slices, narrow 8-bit
 * histograms, Table II and Sec. III-D):
 *   background   N(bg_mean, bg_sd) in 8-bit grey units
 *   ellipsoids   semi-axes U(10,60) * min(N)/256, random rotation, intensity
 *                U{80..220}, noise N(0, obj_sd), kept >= (max semi-axis + 4)
 *                from every face
 *   cylinders    "appendages": radius U(1.5,4), length U(50,400), starting on
 *                an ellipsoid surface and pointing outwards, clipped to the box
 *   container    optional: a z-aligned cylindrical shell (the sample
 *                container, Sec. III "Container Removal") around the box's
 *                centre, outer radius 0.46 min(nx, ny), wall max(3, 0.03
 *                min(nx, ny)) voxels, intensity U{60..75}; the ellipsoids are
 *                then placed inside its inner radius
 *   a voxel takes the intensity of the last primitive that contains its
 *   centre (container, then ellipsoids, then cylinders, in index order)
 *   grey values are scaled by 2^(bits-8) and clamped to [0, 2^bits - 1].
 * Randomness: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) used as a
 * counter-based generator, output k of the stream seeded with s being
 * mix(s + (k+1) * 0x9e3779b97f4a7c15).  Normal noise is an Irwin-Hall sum of
 * twelve 16-bit uniforms, evaluated in integers.
 */
#ifndef PHANTOM_H
#define PHANTOM_H

#include <stdint.h>

#define PH_MAX_ELL 16
#define PH_MAX_CYL 512

typedef struct {
    float c[3];
    float R[9];      /* world -> local rotation, row-major: q = R (p - c) */
    float inv_a[3];  /* reciprocal semi-axes */
    float lo[3], hi[3];
    int32_t intensity;
    int32_t pad;
} ph_ellipsoid;

typedef struct {
    float p0[3];
    float u[3];
    float len;
    float r2;
    float lo[3], hi[3];
    int32_t intensity;
    int32_t pad;
} ph_cylinder;

typedef struct {
    int64_t nx, ny, nz;
    uint64_t seed;
    int32_t bits, esize;
    int32_t n_ell, n_cyl;
    int32_t bg_mean, bg_sd, obj_sd, pad;
    int32_t tube, tube_intensity;   /* container shell (tube != 0) */
    float tube_c[2];                /* axis position (x, y) */
    float tube_r2_in, tube_r2_out;  /* squared inner / outer radius */
    ph_ellipsoid ell[PH_MAX_ELL];
    ph_cylinder cyl[PH_MAX_CYL];
} ph_params;

#if defined(__CUDACC__)
#define PH_HD __host__ __device__ __forceinline__
#else
#define PH_HD static inline
#endif

/* One IEEE rounding per operation on both builds (no contraction). */
PH_HD float ph_mul(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}

PH_HD float ph_add(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}

PH_HD float ph_sub(float a, float b)
{
#if defined(__CUDA_ARCH__)
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}

PH_HD uint64_t ph_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Output k (0-based) of the SplitMix64 stream seeded with s. */
PH_HD uint64_t ph_hash(uint64_t s, uint64_t k)
{
    return ph_mix64(s + (k + 1ULL) * 0x9e3779b97f4a7c15ULL);
}

PH_HD int ph_in_box(const float lo[3], const float hi[3], float x, float y, float z)
{
    return x >= lo[0] && x <= hi[0] && y >= lo[1] && y <= hi[1] && z >= lo[2] && z <= hi[2];
}

PH_HD int ph_in_ellipsoid(const ph_ellipsoid *e, float x, float y, float z)
{
    float dx = ph_sub(x, e->c[0]), dy = ph_sub(y, e->c[1]), dz = ph_sub(z, e->c[2]);
    float q0 = ph_add(ph_add(ph_mul(e->R[0], dx), ph_mul(e->R[1], dy)), ph_mul(e->R[2], dz));
    float q1 = ph_add(ph_add(ph_mul(e->R[3], dx), ph_mul(e->R[4], dy)), ph_mul(e->R[5], dz));
    float q2 = ph_add(ph_add(ph_mul(e->R[6], dx), ph_mul(e->R[7], dy)), ph_mul(e->R[8], dz));
    float s0 = ph_mul(q0, e->inv_a[0]), s1 = ph_mul(q1, e->inv_a[1]), s2 = ph_mul(q2, e->inv_a[2]);
    float ss = ph_add(ph_add(ph_mul(s0, s0), ph_mul(s1, s1)), ph_mul(s2, s2));
    return ss <= 1.0f;
}

PH_HD int ph_in_cylinder(const ph_cylinder *c, float x, float y, float z)
{
    float wx = ph_sub(x, c->p0[0]), wy = ph_sub(y, c->p0[1]), wz = ph_sub(z, c->p0[2]);
    float t = ph_add(ph_add(ph_mul(wx, c->u[0]), ph_mul(wy, c->u[1])), ph_mul(wz, c->u[2]));
    if (t < 0.0f || t > c->len) return 0;
    float ww = ph_add(ph_add(ph_mul(wx, wx), ph_mul(wy, wy)), ph_mul(wz, wz));
    float perp2 = ph_sub(ww, ph_mul(t, t));
    return perp2 <= c->r2;
}

PH_HD int ph_in_tube(const ph_params *P, float x, float y)
{
    float dx = ph_sub(x, P->tube_c[0]), dy = ph_sub(y, P->tube_c[1]);
    float d2 = ph_add(ph_mul(dx, dx), ph_mul(dy, dy));
    return P->tube && d2 >= P->tube_r2_in && d2 <= P->tube_r2_out;
}

/* Grey value of voxel (x, y, z) given the index of the primitive that owns it
 * (-1 = background, -2 = container; ellipsoids 0..n_ell-1, cylinders n_ell..). */
PH_HD uint32_t ph_grey(const ph_params *P, int64_t x, int64_t y, int64_t z, int owner)
{
    uint64_t idx = (uint64_t)((z * P->ny + y) * P->nx + x);
    int64_t S = 0;
    for (int k = 0; k < 3; ++k) {
        uint64_t h = ph_hash(P->seed, 3ULL * idx + (uint64_t)k);
        S += (int64_t)(h & 0xffff) + (int64_t)((h >> 16) & 0xffff) +
             (int64_t)((h >> 32) & 0xffff) + (int64_t)(h >> 48);
    }
    int64_t base, sd;
    if (owner == -1) { base = P->bg_mean; sd = P->bg_sd; }
    else if (owner == -2) { base = P->tube_intensity; sd = P->obj_sd; }
    else if (owner < P->n_ell) { base = P->ell[owner].intensity; sd = P->obj_sd; }
    else { base = P->cyl[owner - P->n_ell].intensity; sd = P->obj_sd; }
    int64_t scale = (int64_t)1 << (P->bits - 8);
    int64_t num = base * scale * 65536 + sd * scale * (S - 393210) + 32768;
    int64_t v = num < 0 ? 0 : (num >> 16);
    int64_t vmax = ((int64_t)1 << P->bits) - 1;
    return (uint32_t)(v > vmax ? vmax : v);
}

#ifdef __cplusplus
extern "C" {
#endif
/* Fill *P for a volume; returns 0 or -1 on bad arguments.  Implemented once,
 * in phantom_params.c, and linked into both builds. */
int ph_make_params(int64_t nx, int64_t ny, int64_t nz, int32_t bits, int32_t esize,
                   uint64_t seed, int32_t n_ell, int32_t n_cyl, int32_t tube, ph_params *P);
#ifdef __cplusplus
}
#endif

#endif
