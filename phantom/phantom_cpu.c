/*
 * phantom_cpu.c -- CPU writer of the synthetic phantom (input generator only).
 * Writes any sub-box of the volume, so a test can regenerate the few voxels it
 * needs of a volume that is too large for the host.  Bricks of 32x8x8 voxels
 * test only the primitives whose bounding boxes touch them; the per-voxel
 * value comes from phantom.h and matches the GPU writer byte for byte.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#include "phantom.h"

int ph_params_size(void) { return (int)sizeof(ph_params); }

/* The container of *P in voxel-index coordinates (voxel centres sit at index
 * + 1/2): axis (x, y), inner and outer radius; returns 0 when there is none. */
int ph_tube_info(const ph_params *P, double out[4])
{
    if (!P || !P->tube) return 0;
    out[0] = (double)P->tube_c[0] - 0.5;
    out[1] = (double)P->tube_c[1] - 0.5;
    out[2] = sqrt((double)P->tube_r2_in);
    out[3] = sqrt((double)P->tube_r2_out);
    return 1;
}

static int brick_overlaps(const float lo[3], const float hi[3], int64_t bx0, int64_t by0,
                          int64_t bz0, int64_t bx1, int64_t by1, int64_t bz1)
{
    /* voxel centres of the brick span [b0 + 0.5, b1 - 0.5] */
    return !(hi[0] < (float)bx0 || lo[0] > (float)bx1 || hi[1] < (float)by0 ||
             lo[1] > (float)by1 || hi[2] < (float)bz0 || lo[2] > (float)bz1);
}

/* Write voxels [x0,x1) x [y0,y1) x [z0,z1) of the volume described by *P into
 * out, laid out [z1-z0][y1-y0][x1-x0] with x fastest. */
int ph_generate_cpu(const ph_params *P, int64_t x0, int64_t x1, int64_t y0, int64_t y1,
                    int64_t z0, int64_t z1, void *out)
{
    if (!P || !out || x0 < 0 || y0 < 0 || z0 < 0 || x1 > P->nx || y1 > P->ny || z1 > P->nz ||
        x0 > x1 || y0 > y1 || z0 > z1)
        return -1;
    const int nprim = P->n_ell + P->n_cyl;
    int *cand = (int *)malloc(sizeof(int) * (size_t)(nprim > 0 ? nprim : 1));
    if (!cand) return -1;
    const int64_t sx = x1 - x0, sy = y1 - y0;
    for (int64_t bz = z0; bz < z1; bz += 8)
        for (int64_t by = y0; by < y1; by += 8)
            for (int64_t bx = x0; bx < x1; bx += 32) {
                int64_t ex = bx + 32 < x1 ? bx + 32 : x1;
                int64_t ey = by + 8 < y1 ? by + 8 : y1;
                int64_t ez = bz + 8 < z1 ? bz + 8 : z1;
                int nc = 0;
                for (int e = 0; e < P->n_ell; ++e)
                    if (brick_overlaps(P->ell[e].lo, P->ell[e].hi, bx, by, bz, ex, ey, ez)) cand[nc++] = e;
                for (int c = 0; c < P->n_cyl; ++c)
                    if (brick_overlaps(P->cyl[c].lo, P->cyl[c].hi, bx, by, bz, ex, ey, ez))
                        cand[nc++] = P->n_ell + c;
                for (int64_t z = bz; z < ez; ++z)
                    for (int64_t y = by; y < ey; ++y)
                        for (int64_t x = bx; x < ex; ++x) {
                            float fx = (float)x + 0.5f, fy = (float)y + 0.5f, fz = (float)z + 0.5f;
                            int owner = ph_in_tube(P, fx, fy) ? -2 : -1;
                            for (int q = 0; q < nc; ++q) {
                                int p = cand[q];
                                if (p < P->n_ell) {
                                    const ph_ellipsoid *E = &P->ell[p];
                                    if (ph_in_box(E->lo, E->hi, fx, fy, fz) && ph_in_ellipsoid(E, fx, fy, fz))
                                        owner = p;
                                } else {
                                    const ph_cylinder *C = &P->cyl[p - P->n_ell];
                                    if (ph_in_box(C->lo, C->hi, fx, fy, fz) && ph_in_cylinder(C, fx, fy, fz))
                                        owner = p;
                                }
                            }
                            uint32_t v = ph_grey(P, x, y, z, owner);
                            int64_t o = ((z - z0) * sy + (y - y0)) * sx + (x - x0);
                            if (P->esize == 1) ((uint8_t *)out)[o] = (uint8_t)v;
                            else ((uint16_t *)out)[o] = (uint16_t)v;
                        }
            }
    free(cand);
    return 0;
}
