/*
 * phantom_params.c -- seeded primitive parameters of the synthetic phantom
 * (input generator only; see phantom.h for the model).  Host code, FP64,
 * rounded to FP32 once per stored value.
 */
#include <math.h>
#include <string.h>

#include "phantom.h"

typedef struct {
    uint64_t s;
    uint64_t k;
} ph_stream;

static double uni(ph_stream *st)
{
    uint64_t h = ph_hash(st->s, st->k++);
    return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}

static void unit_vec(ph_stream *st, double v[3])
{
    const double PI = 3.14159265358979323846;
    double z = 2.0 * uni(st) - 1.0;
    double phi = 2.0 * PI * uni(st);
    double rr = sqrt(fmax(0.0, 1.0 - z * z));
    v[0] = rr * cos(phi);
    v[1] = rr * sin(phi);
    v[2] = z;
}

int ph_make_params(int64_t nx, int64_t ny, int64_t nz, int32_t bits, int32_t esize,
                   uint64_t seed, int32_t n_ell, int32_t n_cyl, int32_t tube, ph_params *P)
{
    const double PI = 3.14159265358979323846;
    if (!P || nx <= 0 || ny <= 0 || nz <= 0 || bits < 8 || bits > 16) return -1;
    if ((esize != 1 && esize != 2) || (esize == 1 && bits != 8)) return -1;
    if (n_ell < 0 || n_ell > PH_MAX_ELL || n_cyl < 0 || n_cyl > PH_MAX_CYL) return -1;
    memset(P, 0, sizeof(*P));
    P->nx = nx; P->ny = ny; P->nz = nz;
    P->seed = seed;
    P->bits = bits; P->esize = esize;
    P->bg_mean = 20; P->bg_sd = 5; P->obj_sd = 8;

    ph_stream st = {seed * 0x9e3779b97f4a7c15ULL + 0x632be59bd9b4e019ULL, 0};
    const double N[3] = {(double)nx, (double)ny, (double)nz};
    double nmin = fmin(N[0], fmin(N[1], N[2]));
    double scale = nmin / 256.0;
    double a_cap = floor(nmin / 2.0) - 5.0;   /* bounding radius that still fits */
    double tube_in = 0.0, tcx = 0.0, tcy = 0.0;
    if (tube) {
        /* its own stream, so volumes without a container keep their draws */
        ph_stream ts = {seed * 0x9e3779b97f4a7c15ULL + 0x2545f4914f6cdd1dULL, 0};
        double nxy = fmin(N[0], N[1]);
        double r_out = 0.46 * nxy, wall = fmax(3.0, 0.03 * nxy);
        tcx = N[0] / 2.0 + (uni(&ts) - 0.5) * 0.06 * nxy;
        tcy = N[1] / 2.0 + (uni(&ts) - 0.5) * 0.06 * nxy;
        tube_in = r_out - wall;
        P->tube = 1;
        P->tube_intensity = 60 + (int32_t)floor(16.0 * uni(&ts));
        P->tube_c[0] = (float)tcx;
        P->tube_c[1] = (float)tcy;
        P->tube_r2_in = (float)(tube_in * tube_in);
        P->tube_r2_out = (float)(r_out * r_out);
        a_cap = fmin(a_cap, floor(tube_in / 2.0) - 4.0);
    }

    int ne = 0;
    for (int e = 0; e < n_ell && a_cap >= 2.0; ++e) {
        double a[3];
        for (int i = 0; i < 3; ++i) a[i] = fmin((10.0 + 50.0 * uni(&st)) * scale, a_cap);
        double al = 2.0 * PI * uni(&st), be = 2.0 * PI * uni(&st), ga = 2.0 * PI * uni(&st);
        /* local -> world = Rz(al) Ry(be) Rx(ga); world -> local is its transpose */
        double ca = cos(al), sa = sin(al), cb = cos(be), sb = sin(be), cg = cos(ga), sg = sin(ga);
        double Mw[9] = {ca * cb, ca * sb * sg - sa * cg, ca * sb * cg + sa * sg,
                        sa * cb, sa * sb * sg + ca * cg, sa * sb * cg - ca * sg,
                        -sb,     cb * sg,                cb * cg};
        double rb = fmax(a[0], fmax(a[1], a[2]));
        double c[3];
        for (int i = 0; i < 3; ++i) {
            double lo = rb + 4.0, hi = N[i] - rb - 4.0;
            c[i] = hi > lo ? lo + (hi - lo) * uni(&st) : N[i] / 2.0;
        }
        if (tube) {
            /* centre the ellipsoid inside the container: a point of the disk
             * of radius tube_in - rb - 4 around the axis */
            double rr = fmax(0.0, tube_in - rb - 4.0) * sqrt(uni(&st));
            double ph = 2.0 * PI * uni(&st);
            c[0] = tcx + rr * cos(ph);
            c[1] = tcy + rr * sin(ph);
        }
        int32_t inten = 80 + (int32_t)floor(141.0 * uni(&st));
        ph_ellipsoid *E = &P->ell[ne++];
        for (int i = 0; i < 3; ++i) {
            E->c[i] = (float)c[i];
            E->inv_a[i] = (float)(1.0 / a[i]);
        }
        for (int r = 0; r < 3; ++r)
            for (int k = 0; k < 3; ++k) E->R[r * 3 + k] = (float)Mw[k * 3 + r];
        for (int j = 0; j < 3; ++j) {
            double ext = 0.0;
            for (int i = 0; i < 3; ++i) ext += (Mw[j * 3 + i] * a[i]) * (Mw[j * 3 + i] * a[i]);
            ext = sqrt(ext) + 2.0;
            E->lo[j] = (float)(c[j] - ext);
            E->hi[j] = (float)(c[j] + ext);
        }
        E->intensity = inten;
        /* keep the local->world matrix and semi-axes for the cylinders */
        (void)Mw;
    }
    P->n_ell = ne;

    int nc = 0;
    for (int k = 0; k < n_cyl && ne > 0; ++k) {
        int e = (int)floor(uni(&st) * ne);
        if (e >= ne) e = ne - 1;
        const ph_ellipsoid *E = &P->ell[e];
        double nh[3], m[3];
        unit_vec(&st, nh);
        unit_vec(&st, m);
        double r = 1.5 + 2.5 * uni(&st);
        double len = 50.0 + 350.0 * uni(&st);
        int32_t inten = 80 + (int32_t)floor(141.0 * uni(&st));
        double a[3], ql[3], g[3], p0[3], gw[3] = {0, 0, 0};
        for (int i = 0; i < 3; ++i) {
            a[i] = 1.0 / (double)E->inv_a[i];
            ql[i] = a[i] * nh[i];
            g[i] = nh[i] / a[i];
        }
        for (int j = 0; j < 3; ++j) {
            /* world = R^T local with R the stored world -> local rotation */
            p0[j] = (double)E->c[j];
            for (int i = 0; i < 3; ++i) {
                p0[j] += (double)E->R[i * 3 + j] * ql[i];
                gw[j] += (double)E->R[i * 3 + j] * g[i];
            }
        }
        double gn = sqrt(gw[0] * gw[0] + gw[1] * gw[1] + gw[2] * gw[2]);
        double u[3];
        for (int i = 0; i < 3; ++i) u[i] = gw[i] / gn + 0.5 * m[i];
        double un = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        if (un < 1e-6) { for (int i = 0; i < 3; ++i) u[i] = gw[i] / gn; un = 1.0; }
        for (int i = 0; i < 3; ++i) u[i] /= un;
        int ok = 1;
        for (int i = 0; i < 3; ++i) {
            double lo = r + (i == 2 ? 4.0 : 1.0), hi = N[i] - 1.0 - r;
            if (p0[i] < lo || p0[i] > hi) ok = 0;
            if (u[i] > 1e-12) len = fmin(len, (hi - p0[i]) / u[i]);
            else if (u[i] < -1e-12) len = fmin(len, (p0[i] - lo) / (-u[i]));
        }
        if (!ok || len < 1.0) continue;
        ph_cylinder *C = &P->cyl[nc++];
        for (int i = 0; i < 3; ++i) {
            C->p0[i] = (float)p0[i];
            C->u[i] = (float)u[i];
            double e0 = p0[i], e1 = p0[i] + len * u[i];
            C->lo[i] = (float)(fmin(e0, e1) - r - 2.0);
            C->hi[i] = (float)(fmax(e0, e1) + r + 2.0);
        }
        C->len = (float)len;
        C->r2 = (float)(r * r);
        C->intensity = inten;
    }
    P->n_cyl = nc;
    return 0;
}
