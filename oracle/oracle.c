/*
 * oracle.c -- plain, slow, CPU reference for the micro-CT preview hot path.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only tests/, __graft_entry__.smoke()
 * and bench.py's cpu_baseline / reference leg may load this library.  It shares
 * no source, header, table or helper with the CUDA library; the two meet only
 * through the seeded inputs the phantom module writes.
 *
 * Paper: "Low-latency Visual Previews of Large Synchrotron Micro-CT Datasets"
 * (arXiv 2311.15038).  Every function cites the passage it follows.  Where the
 * paper is silent or garbled the reading taken is stated beside the code.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no fused multiply-add, so each
 * float/double operation is one IEEE rounding, as written).
 *
 * Pins (tests/test_oracle_*.py, CPU only):
 *   orc_histogram   numpy.bincount, count invariant, z-range slabs
 *   orc_otsu        brute-force minimum of the within-class variance (Eq. 1),
 *                   two-delta closed form, hand-derived golden histogram
 *   orc_its         two-delta / symmetric closed forms, hand-derived golden run
 *   orc_keep_*      hand-built volumes (threshold and top-slab keep tables)
 *   orc_filter      vectorised numpy restatement on random volumes, idempotence
 *   orc_downsample  numpy block mean for integer factors (incl. identity),
 *                   constant volume, hot-voxel footprint partition, ramp
 *                   centres, sum preservation, keep table before averaging
 *   orc_atlas_pack  hand-placed golden atlas, round trip
 *   orc_maxgrid     scipy.ndimage.maximum_filter on random levels
 *   orc_render      Beer-Lambert slab closed form, axis-aligned views against a
 *                   product-form compositor over scipy map_coordinates samples,
 *                   empty volume, axis-aligned sample counts; oblique views:
 *                   camera bases against hand-derived vectors and frame
 *                   properties, sample counts against FP64 ray-box chords,
 *                   renders against the product form over FP64 positions
 *   orc_hough_circle      drawn rings of known centre and radius, the phantom
 *                         container's axis and inner radius, an image without
 *                         edges
 *   orc_mask_circle       hand-counted disks, identity for a covering circle
 *   orc_image_histogram   grey pixels land in round(v*255), primaries at their
 *                         luminance weights, counts sum to the pixel count
 *   orc_render_dense      orc_render on the same level (intensities = raw/255),
 *                         Beer-Lambert slab
 *   orc_render_dense_band its three results equal orc_render_dense stopped at
 *                         alpha_stop - eps, alpha_stop, alpha_stop + eps
 *   orc_render_dense_grad central finite differences of orc_render_dense along
 *                         random directions; closed-form dA/dalpha of a slab;
 *                         term magnitudes bound |gradient|, scale with it
 * No function here is "parity unpinned".
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)

/* ---------------------------------------------------------------- helpers */

static int orc_log2_exact(int64_t v)
{
    int k = 0;
    if (v <= 0 || (v & (v - 1)) != 0) return -1;
    while ((1LL << k) < v) ++k;
    return k;
}

static uint32_t load_voxel(const void *base, int esize, int64_t idx)
{
    if (esize == 1) return ((const uint8_t *)base)[idx];
    return ((const uint16_t *)base)[idx];
}

static void store_voxel(void *base, int esize, int64_t idx, uint32_t v)
{
    if (esize == 1) ((uint8_t *)base)[idx] = (uint8_t)v;
    else ((uint16_t *)base)[idx] = (uint16_t)v;
}

/* Shift that maps a grey value of `bits` bits onto `nbins` bins (nbins a power
 * of two, 1 <= nbins <= 2^bits).  Returns -1 when the pair is not allowed. */
static int bin_shift(int bits, int nbins)
{
    int lb = orc_log2_exact(nbins);
    if (bits < 1 || bits > 16 || lb < 0 || lb > bits) return -1;
    return bits - lb;
}

/* --------------------------------------------------------------- histogram */

/*
 * Voxel histogram: the per-grey-value counts that Alg. 1 and Alg. 2 partition
 * (Sec. III-A) and that the histogram filter inspects (Sec. III-D).
 * hist[b] = #{voxels with z in [z0,z1) and (v >> shift) == b}, shift =
 * bits - log2(nbins).  Values >= 2^bits are not grey values of the declared
 * depth; they are counted in *overflow instead of a bin.
 */
int orc_histogram(const void *vol, int esize, int64_t nx, int64_t ny, int64_t nz,
                  int bits, int64_t z0, int64_t z1, int nbins,
                  uint64_t *hist, uint64_t *overflow)
{
    int shift = bin_shift(bits, nbins);
    if (!vol || !hist || !overflow || (esize != 1 && esize != 2) || shift < 0)
        return ORC_EINVAL;
    if (esize == 1 && bits > 8) return ORC_EINVAL;
    if (nx <= 0 || ny <= 0 || nz <= 0 || z0 < 0 || z1 > nz || z0 > z1) return ORC_EINVAL;
    for (int b = 0; b < nbins; ++b) hist[b] = 0;
    *overflow = 0;
    const uint32_t limit = 1u << bits;
    for (int64_t z = z0; z < z1; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                uint32_t v = load_voxel(vol, esize, (z * ny + y) * nx + x);
                if (v >= limit) *overflow += 1;
                else hist[v >> shift] += 1;
            }
    return ORC_OK;
}

/* ------------------------------------------------------------------- Otsu */

/*
 * Otsu thresholding, Alg. 1 (Sec. III-A).  For every sweep value T the
 * histogram is split into R_a = bins [0, T) and R_b = bins [T, nbins-1]
 * (reading of the slices "[0:T]" and "[T:255]": the upper region includes the
 * last bin).  W = class weight n/N ("density"), U = mean grey value of the
 * class ("Mean"), sigma = W_a W_b (U_a - U_b)^2, the between-class variance;
 * the first T with a strictly larger sigma wins (strict ">" of Alg. 1), so
 * ties keep the lowest T.  A sweep value that leaves a class empty gives no
 * candidate (its W is 0, so sigma could not beat the initial 0 anyway).
 * Maximising this sigma is the same as minimising Eq. 1's within-class
 * variance, because the two add up to the fixed total variance.
 * Class sums are recomputed from scratch for every T, as the sweep reads.
 * The FP64 evaluation order below is part of the definition:
 *   Wa = na/N, Wb = nb/N, Ua = Sa/na, Ub = Sb/nb, d = Ua-Ub,
 *   sigma = ((Wa*Wb)*d)*d.
 * Voxels with T <= bin keep their value ("lower limit of the intensity
 * range", Sec. III-A), so T is returned as a bin index.
 */
int orc_otsu(const uint64_t *hist, int nbins, int32_t *T_out, double *sigma_out)
{
    if (!hist || !T_out || nbins < 1) return ORC_EINVAL;
    int32_t T_otsu = 0;
    double sigma_otsu = 0.0;
    uint64_t N = 0;
    for (int b = 0; b < nbins; ++b) N += hist[b];
    for (int T = 0; T < nbins; ++T) {
        uint64_t na = 0, nb = 0, Sa = 0, Sb = 0;
        for (int b = 0; b < T; ++b) { na += hist[b]; Sa += (uint64_t)b * hist[b]; }
        for (int b = T; b < nbins; ++b) { nb += hist[b]; Sb += (uint64_t)b * hist[b]; }
        if (na == 0 || nb == 0) continue;
        double Nd = (double)N;
        double Wa = (double)na / Nd;
        double Wb = (double)nb / Nd;
        double Ua = (double)Sa / (double)na;
        double Ub = (double)Sb / (double)nb;
        double d = Ua - Ub;
        double sigma = ((Wa * Wb) * d) * d;
        if (sigma > sigma_otsu) { sigma_otsu = sigma; T_otsu = T; }
    }
    *T_out = T_otsu;
    if (sigma_out) *sigma_out = sigma_otsu;
    return ORC_OK;
}

/* -------------------------------------------------------------------- ITS */

/*
 * Iterative threshold selection, Alg. 2 (Sec. III-A).
 *   T_it <- T_start = nbins/2 (the "middle" of the dynamic range).
 *   repeat: R_a = bins b < T_it, R_b = bins b >= T_it (a real T compares
 *           against integer bins, so the split index is ceil(T_it));
 *           mu1, mu2 = mean grey value of R_a, R_b (an empty region takes
 *           mu = T_it, i.e. it does not pull the threshold);
 *           T_tmp = (mu1 + mu2) / 2;  r = |T_it - T_tmp|;  T_it = T_tmp
 *   until r == 0.
 * Reading of the garbled update "r <- |r - T_tmp|": r is the change of the
 * threshold between consecutive iterations; r == 0 means mu1 and mu2 no
 * longer change (Step 5 of the prose).  At most max_iter iterations; if r is
 * still nonzero then *converged = 0 and the last T_it is used.
 * Kept voxels are those with bin >= T_it, i.e. bin >= ceil(T_it) = *T_out.
 */
int orc_its(const uint64_t *hist, int nbins, int max_iter, int32_t *T_out,
            int32_t *iters_out, int32_t *converged, double *T_real_out)
{
    if (!hist || !T_out || !iters_out || !converged || nbins < 1 || max_iter < 1)
        return ORC_EINVAL;
    double T_it = (double)nbins / 2.0;
    double r = T_it;
    int iters = 0;
    while (r != 0.0 && iters < max_iter) {
        double c = ceil(T_it);
        int64_t m = c < 0.0 ? 0 : (c > (double)nbins ? nbins : (int64_t)c);
        uint64_t n1 = 0, n2 = 0, S1 = 0, S2 = 0;
        for (int64_t b = 0; b < m; ++b) { n1 += hist[b]; S1 += (uint64_t)b * hist[b]; }
        for (int64_t b = m; b < nbins; ++b) { n2 += hist[b]; S2 += (uint64_t)b * hist[b]; }
        double mu1 = n1 ? (double)S1 / (double)n1 : T_it;
        double mu2 = n2 ? (double)S2 / (double)n2 : T_it;
        double T_tmp = (mu1 + mu2) / 2.0;
        r = fabs(T_it - T_tmp);
        T_it = T_tmp;
        ++iters;
    }
    double c = ceil(T_it);
    *T_out = (int32_t)(c < 0.0 ? 0 : (c > (double)nbins ? nbins : c));
    *iters_out = iters;
    *converged = (r == 0.0);
    if (T_real_out) *T_real_out = T_it;
    return ORC_OK;
}

/* ------------------------------------------------------------ keep tables */

/* Threshold classification (Sec. III-A, binary classification of each voxel):
 * keep[b] = 1 iff b >= T. */
int orc_keep_threshold(int nbins, int32_t T, uint8_t *keep)
{
    if (!keep || nbins < 1) return ORC_EINVAL;
    for (int b = 0; b < nbins; ++b) keep[b] = (uint8_t)(b >= T);
    return ORC_OK;
}

/* Histogram filtering (Sec. III-D): the histogram of the top slices is the
 * signature of the surroundings, and those bins are disposed of from the whole
 * volume.  keep[b] = 1 iff hist_top[b] < kmin (kmin = 1: any occurrence in the
 * top slab removes the bin). */
int orc_keep_topslab(const uint64_t *hist_top, int nbins, uint64_t kmin, uint8_t *keep)
{
    if (!hist_top || !keep || nbins < 1) return ORC_EINVAL;
    for (int b = 0; b < nbins; ++b) keep[b] = (uint8_t)(hist_top[b] < kmin);
    return ORC_OK;
}

/* ----------------------------------------------------------------- filter */

/* Binary classification applied to the volume (Sec. III-A, Sec. III-D):
 * out = v when v is a grey value of the declared depth and its bin is kept,
 * else 0 ("removed" voxels become zero). */
static uint32_t filter_one(uint32_t v, int bits, int shift, const uint8_t *keep)
{
    if (v >= (1u << bits)) return 0;
    return keep[v >> shift] ? v : 0;
}

int orc_filter(const void *in, int esize, int64_t nvox, int bits,
               const uint8_t *keep, int nbins, void *out)
{
    int shift = bin_shift(bits, nbins);
    if (!in || !out || !keep || (esize != 1 && esize != 2) || shift < 0 || nvox < 0)
        return ORC_EINVAL;
    for (int64_t i = 0; i < nvox; ++i)
        store_voxel(out, esize, i, filter_one(load_voxel(in, esize, i), bits, shift, keep));
    return ORC_OK;
}

/* ------------------------------------------------------------- downsample */

/*
 * Box downsampling of a volume to a slicemap level (slicemap conversion and
 * the coarse-then-fine multi-resolution loading, Sec. II and Sec. III; the
 * filter itself is not given by the paper).  Reading: an integer area box.
 * Output voxel i along an axis of N source and M output voxels covers the
 * source range [floor(i N / M), floor((i+1) N / M)); the output is the mean of
 * the covered (optionally keep-filtered) voxels rounded half up,
 * floor((sum + cnt/2) / cnt) with cnt the box volume.  M <= N on every axis.
 * With keep == NULL the voxels are used as stored.
 * Levels k >= 1 of a slicemap are this function applied to level k-1 with
 * M = N/2 (an exact 2x2x2 box).
 */
int orc_downsample(const void *in, int esize, int64_t nx, int64_t ny, int64_t nz,
                   int bits, const uint8_t *keep, int nbins,
                   int64_t mx, int64_t my, int64_t mz, void *out)
{
    int shift = 0;
    if (!in || !out || (esize != 1 && esize != 2)) return ORC_EINVAL;
    if (nx <= 0 || ny <= 0 || nz <= 0 || mx <= 0 || my <= 0 || mz <= 0) return ORC_EINVAL;
    if (mx > nx || my > ny || mz > nz) return ORC_EINVAL;
    if (keep) {
        shift = bin_shift(bits, nbins);
        if (shift < 0) return ORC_EINVAL;
    }
    for (int64_t k = 0; k < mz; ++k) {
        int64_t z_lo = (k * nz) / mz, z_hi = ((k + 1) * nz) / mz;
        for (int64_t j = 0; j < my; ++j) {
            int64_t y_lo = (j * ny) / my, y_hi = ((j + 1) * ny) / my;
            for (int64_t i = 0; i < mx; ++i) {
                int64_t x_lo = (i * nx) / mx, x_hi = ((i + 1) * nx) / mx;
                uint64_t sum = 0;
                uint64_t cnt = (uint64_t)((z_hi - z_lo) * (y_hi - y_lo) * (x_hi - x_lo));
                for (int64_t z = z_lo; z < z_hi; ++z)
                    for (int64_t y = y_lo; y < y_hi; ++y)
                        for (int64_t x = x_lo; x < x_hi; ++x) {
                            uint32_t v = load_voxel(in, esize, (z * ny + y) * nx + x);
                            if (keep) v = filter_one(v, bits, shift, keep);
                            sum += v;
                        }
                store_voxel(out, esize, (k * my + j) * mx + i,
                            (uint32_t)((sum + cnt / 2) / cnt));
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ atlas */

/*
 * Slicemap atlas (the 2D grid of tiled slices the paper's previews load,
 * Sec. III).  Slice z of an mx*my*mz level goes to tile row z / tiles_x, tile
 * column z % tiles_x; its pixel (x, y) sits at
 *   atlas[(row*my + y) * (tiles_x*mx) + col*mx + x].
 * Tiles past the last slice are zero.  tiles_x * tiles_y >= mz.
 */
int orc_atlas_pack(const void *level, int esize, int64_t mx, int64_t my, int64_t mz,
                   int64_t tiles_x, int64_t tiles_y, void *atlas)
{
    if (!level || !atlas || (esize != 1 && esize != 2)) return ORC_EINVAL;
    if (mx <= 0 || my <= 0 || mz <= 0 || tiles_x <= 0 || tiles_y <= 0 || tiles_x * tiles_y < mz)
        return ORC_EINVAL;
    int64_t aw = tiles_x * mx, ah = tiles_y * my;
    memset(atlas, 0, (size_t)(aw * ah * esize));
    for (int64_t z = 0; z < mz; ++z) {
        int64_t row = z / tiles_x, col = z % tiles_x;
        for (int64_t y = 0; y < my; ++y)
            for (int64_t x = 0; x < mx; ++x)
                store_voxel(atlas, esize, (row * my + y) * aw + col * mx + x,
                            load_voxel(level, esize, (z * my + y) * mx + x));
    }
    return ORC_OK;
}

/* ----------------------------------------------------------------- render */

/*
 * Server-side rendering of a slicemap level to a 2D image (Sec. III-C).  The
 * paper names the step but not the renderer; this is orthographic
 * emission-absorption direct volume rendering, front to back:
 *
 * Camera (world unit = one source voxel, box [0,Nx]x[0,Ny]x[0,Nz], centre c):
 *   az, el in radians = (deg * pi) / 180 in FP64;
 *   b  = (cos el cos az, cos el sin az, sin el)   (towards the viewer)
 *   r  = (-sin az, cos az, 0)                      (image right)
 *   u  = (-sin el cos az, -sin el sin az, cos el)  (image up, = b x r)
 *   each component evaluated in FP64 and rounded to FP32.
 *   L = FP32(sqrt(Nx^2 + Ny^2 + Nz^2)), the side of the square image plane.
 * Ray of pixel (i, j), row j counted from the top, all in FP32 with one
 * rounding per operation, in exactly this order:
 *   sx = (i + 0.5) / W - 0.5;   sy = 0.5 - (j + 0.5) / H
 *   o_a = ((c_a + (sx*L)*r_a) + (sy*L)*u_a) + L*b_a;   d_a = -b_a
 *   slab per axis: d_a != 0: inv = 1/d_a, t0 = (0 - o_a)*inv,
 *                  t1 = (N_a - o_a)*inv, [min, max];
 *                  d_a == 0: whole line if 0 <= o_a <= N_a, else no hit
 *   t_near = max of the mins, t_far = min of the maxes
 *   s_a = N_a / M_a,  Delta = step * min(s_x, s_y, s_z)
 *   n = floor((t_far - t_near) / Delta) if t_far > t_near, else 0
 * Samples (FP64 from here on): t_k = t_near + (k + 1/2) Delta, k < n;
 *   p = o + t_k d;  level coordinate q_a = (p_a * M_a) / N_a - 1/2;
 *   trilinear interpolation of the level with corner indices clamped to
 *   [0, M_a - 1]; value v = min(raw / (2^bits - 1), 1).
 * Transfer function: nlut >= 2 RGBA entries, x = v (nlut - 1),
 *   j = min(floor(x), nlut - 2), f = x - j, rgba = lut[j](1-f) + lut[j+1] f.
 * Compositing (colour in the LUT is straight, the output premultiplied):
 *   w = (1 - A) alpha;  C += w c;  A += w;  stop once A >= alpha_stop.
 *
 * Several results are correct when A lands near alpha_stop, because an FP32
 * march may stop one sample earlier or later than this FP64 one.  The march
 * therefore records the state at three stop levels, alpha_stop - eps,
 * alpha_stop and alpha_stop + eps (rgba_lo, rgba, rgba_hi; nsamp gives the
 * sample counts at the three levels).  A ray whose lo and hi results differ is
 * ambiguous; any stop between them is a correct result.
 */
typedef struct {
    float az_deg, el_deg;
    int32_t width, height;
    float step;
} orc_view;

typedef struct {
    float o[3], d[3];
    float t_near, delta;
    int64_t n;
} orc_ray;

static void ray_setup(const float b[3], const float r[3], const float u[3], float L,
                      const float c[3], const float N[3], float delta,
                      int32_t W, int32_t H, int64_t i, int64_t j, orc_ray *ray)
{
    float sx = ((float)i + 0.5f) / (float)W - 0.5f;
    float sy = 0.5f - ((float)j + 0.5f) / (float)H;
    float sxL = sx * L, syL = sy * L;
    float tmin = -INFINITY, tmax = INFINITY;
    int miss = 0;
    for (int a = 0; a < 3; ++a) {
        float t1 = c[a] + sxL * r[a];
        float t2 = t1 + syL * u[a];
        float oa = t2 + L * b[a];
        float da = -b[a];
        ray->o[a] = oa;
        ray->d[a] = da;
        if (da != 0.0f) {
            float inv = 1.0f / da;
            float s0 = (0.0f - oa) * inv;
            float s1 = (N[a] - oa) * inv;
            tmin = fmaxf(tmin, fminf(s0, s1));
            tmax = fminf(tmax, fmaxf(s0, s1));
        } else if (!(oa >= 0.0f && oa <= N[a])) {
            miss = 1;
        }
    }
    ray->t_near = tmin;
    ray->delta = delta;
    ray->n = 0;
    if (!miss && tmax > tmin) {
        float fn = floorf((tmax - tmin) / delta);
        ray->n = (int64_t)fn;
    }
}

static double level_fetch(const void *lv, int esize, int64_t mx, int64_t my,
                          int64_t x, int64_t y, int64_t z)
{
    return (double)load_voxel(lv, esize, (z * my + y) * mx + x);
}

static int64_t clampi(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

static double sample_level(const void *lv, int esize, const int64_t M[3], const double q[3],
                           double vmax)
{
    int64_t i0[3], i1[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(q[a]);
        f[a] = q[a] - fl;
        i0[a] = clampi((int64_t)fl, 0, M[a] - 1);
        i1[a] = clampi((int64_t)fl + 1, 0, M[a] - 1);
    }
    double c00 = level_fetch(lv, esize, M[0], M[1], i0[0], i0[1], i0[2]) * (1.0 - f[0]) +
                 level_fetch(lv, esize, M[0], M[1], i1[0], i0[1], i0[2]) * f[0];
    double c10 = level_fetch(lv, esize, M[0], M[1], i0[0], i1[1], i0[2]) * (1.0 - f[0]) +
                 level_fetch(lv, esize, M[0], M[1], i1[0], i1[1], i0[2]) * f[0];
    double c01 = level_fetch(lv, esize, M[0], M[1], i0[0], i0[1], i1[2]) * (1.0 - f[0]) +
                 level_fetch(lv, esize, M[0], M[1], i1[0], i0[1], i1[2]) * f[0];
    double c11 = level_fetch(lv, esize, M[0], M[1], i0[0], i1[1], i1[2]) * (1.0 - f[0]) +
                 level_fetch(lv, esize, M[0], M[1], i1[0], i1[1], i1[2]) * f[0];
    double c0 = c00 * (1.0 - f[1]) + c10 * f[1];
    double c1 = c01 * (1.0 - f[1]) + c11 * f[1];
    double v = (c0 * (1.0 - f[2]) + c1 * f[2]) / vmax;
    return v > 1.0 ? 1.0 : v;
}

int orc_render(const void *level, int esize, int bits, int64_t mx, int64_t my, int64_t mz,
               int64_t nx, int64_t ny, int64_t nz, const float *lut, int nlut,
               float alpha_stop, double eps, const orc_view *view,
               const int64_t *pixels, int64_t npix,
               double *rgba, double *rgba_lo, double *rgba_hi, uint64_t *nsamp)
{
    if (!level || !lut || !view || !rgba || (esize != 1 && esize != 2) || nlut < 2) return ORC_EINVAL;
    if (bits < 1 || bits > 16 || (esize == 1 && bits > 8)) return ORC_EINVAL;
    if (mx <= 0 || my <= 0 || mz <= 0 || nx <= 0 || ny <= 0 || nz <= 0) return ORC_EINVAL;
    if (view->width <= 0 || view->height <= 0 || !(view->step > 0.0f)) return ORC_EINVAL;
    const double PI = 3.14159265358979323846;
    double az = ((double)view->az_deg * PI) / 180.0;
    double el = ((double)view->el_deg * PI) / 180.0;
    float b[3] = {(float)(cos(el) * cos(az)), (float)(cos(el) * sin(az)), (float)sin(el)};
    float r[3] = {(float)(-sin(az)), (float)cos(az), 0.0f};
    float u[3] = {(float)(-sin(el) * cos(az)), (float)(-sin(el) * sin(az)), (float)cos(el)};
    float L = (float)sqrt((double)(nx * nx + ny * ny + nz * nz));
    float N[3] = {(float)nx, (float)ny, (float)nz};
    float c[3] = {N[0] / 2.0f, N[1] / 2.0f, N[2] / 2.0f};
    float s[3] = {N[0] / (float)mx, N[1] / (float)my, N[2] / (float)mz};
    float smin = fminf(s[0], fminf(s[1], s[2]));
    float delta = view->step * smin;
    const int64_t M[3] = {mx, my, mz};
    const double Nd[3] = {(double)nx, (double)ny, (double)nz};
    const double vmax = (double)((1u << bits) - 1u);
    const int64_t W = view->width, H = view->height;
    const int64_t total = npix >= 0 && pixels ? npix : W * H;
    const double stops[3] = {(double)alpha_stop - eps, (double)alpha_stop, (double)alpha_stop + eps};

    for (int64_t p = 0; p < total; ++p) {
        int64_t lin = pixels ? pixels[p] : p;
        if (lin < 0 || lin >= W * H) return ORC_EINVAL;
        orc_ray ray;
        ray_setup(b, r, u, L, c, N, delta, view->width, view->height, lin % W, lin / W, &ray);
        double C[3] = {0, 0, 0}, A = 0.0;
        double out[3][4];
        uint64_t cnt[3];
        int done[3] = {0, 0, 0};
        int64_t k = 0;
        for (; k < ray.n && !done[2]; ++k) {
            double t = (double)ray.t_near + ((double)k + 0.5) * (double)ray.delta;
            double q[3];
            for (int a = 0; a < 3; ++a) {
                double pa = (double)ray.o[a] + t * (double)ray.d[a];
                q[a] = (pa * (double)M[a]) / Nd[a] - 0.5;
            }
            double v = sample_level(level, esize, M, q, vmax);
            double x = v * (double)(nlut - 1);
            double fl = floor(x);
            int64_t jj = (int64_t)fl;
            if (jj > nlut - 2) jj = nlut - 2;
            double f = x - (double)jj;
            double col[4];
            for (int ch = 0; ch < 4; ++ch)
                col[ch] = (double)lut[jj * 4 + ch] * (1.0 - f) + (double)lut[(jj + 1) * 4 + ch] * f;
            double w = (1.0 - A) * col[3];
            C[0] += w * col[0];
            C[1] += w * col[1];
            C[2] += w * col[2];
            A += w;
            for (int s2 = 0; s2 < 3; ++s2) {
                if (!done[s2] && A >= stops[s2]) {
                    done[s2] = 1;
                    out[s2][0] = C[0]; out[s2][1] = C[1]; out[s2][2] = C[2]; out[s2][3] = A;
                    cnt[s2] = (uint64_t)(k + 1);
                }
            }
        }
        for (int s2 = 0; s2 < 3; ++s2) {
            if (!done[s2]) {
                out[s2][0] = C[0]; out[s2][1] = C[1]; out[s2][2] = C[2]; out[s2][3] = A;
                cnt[s2] = (uint64_t)k;
            }
        }
        for (int ch = 0; ch < 4; ++ch) {
            rgba[p * 4 + ch] = out[1][ch];
            if (rgba_lo) rgba_lo[p * 4 + ch] = out[0][ch];
            if (rgba_hi) rgba_hi[p * 4 + ch] = out[2][ch];
        }
        if (nsamp) { nsamp[p * 3 + 0] = cnt[0]; nsamp[p * 3 + 1] = cnt[1]; nsamp[p * 3 + 2] = cnt[2]; }
    }
    return ORC_OK;
}

/* Ray parameters of one pixel, exposed so the tests can pin the FP32 setup
 * against closed forms for axis-aligned views. */
int orc_ray_params(int64_t mx, int64_t my, int64_t mz, int64_t nx, int64_t ny, int64_t nz,
                   const orc_view *view, int64_t i, int64_t j, float *o, float *d,
                   float *t_near, float *delta, int64_t *n)
{
    if (!view || !o || !d || !t_near || !delta || !n) return ORC_EINVAL;
    const double PI = 3.14159265358979323846;
    double az = ((double)view->az_deg * PI) / 180.0;
    double el = ((double)view->el_deg * PI) / 180.0;
    float b[3] = {(float)(cos(el) * cos(az)), (float)(cos(el) * sin(az)), (float)sin(el)};
    float r[3] = {(float)(-sin(az)), (float)cos(az), 0.0f};
    float u[3] = {(float)(-sin(el) * cos(az)), (float)(-sin(el) * sin(az)), (float)cos(el)};
    float L = (float)sqrt((double)(nx * nx + ny * ny + nz * nz));
    float N[3] = {(float)nx, (float)ny, (float)nz};
    float c[3] = {N[0] / 2.0f, N[1] / 2.0f, N[2] / 2.0f};
    float s[3] = {N[0] / (float)mx, N[1] / (float)my, N[2] / (float)mz};
    float smin = fminf(s[0], fminf(s[1], s[2]));
    orc_ray ray;
    ray_setup(b, r, u, L, c, N, view->step * smin, view->width, view->height, i, j, &ray);
    for (int a = 0; a < 3; ++a) { o[a] = ray.o[a]; d[a] = ray.d[a]; }
    *t_near = ray.t_near;
    *delta = ray.delta;
    *n = ray.n;
    return ORC_OK;
}

/* ---------------------------------------------------------------- max grid */

/*
 * Per-cell maximum of a slicemap level, the occupancy data that lets a
 * renderer skip samples whose transfer-function opacity is exactly zero (an
 * acceleration structure of this library; the paper has none).  Cell
 * (cx, cy, cz) of edge `cell` covers level voxels [cell*c, cell*c + cell] per
 * axis (one voxel beyond the cell, clamped to the level): every voxel a
 * trilinear sample whose lower corner lies in the cell can touch.
 * grid is [ceil(mz/cell)][ceil(my/cell)][ceil(mx/cell)] uint16.
 */
int orc_maxgrid(const void *level, int esize, int64_t mx, int64_t my, int64_t mz, int cell, uint16_t *grid)
{
    if (!level || !grid || (esize != 1 && esize != 2) || cell < 1) return ORC_EINVAL;
    if (mx <= 0 || my <= 0 || mz <= 0) return ORC_EINVAL;
    int64_t gx = (mx + cell - 1) / cell, gy = (my + cell - 1) / cell, gz = (mz + cell - 1) / cell;
    for (int64_t cz = 0; cz < gz; ++cz)
        for (int64_t cy = 0; cy < gy; ++cy)
            for (int64_t cx = 0; cx < gx; ++cx) {
                uint32_t m = 0;
                for (int64_t z = cz * cell; z <= cz * cell + cell && z < mz; ++z)
                    for (int64_t y = cy * cell; y <= cy * cell + cell && y < my; ++y)
                        for (int64_t x = cx * cell; x <= cx * cell + cell && x < mx; ++x) {
                            uint32_t v = load_voxel(level, esize, (z * my + y) * mx + x);
                            if (v > m) m = v;
                        }
                grid[(cz * gy + cy) * gx + cx] = (uint16_t)m;
            }
    return ORC_OK;
}

/* ---------------------------------------------------------------- entropy */

/*
 * Shannon entropy of an image histogram, Eq. 2 (Sec. III-C):
 * H = -sum_i p_i log2 p_i with p_i the normalised counts; empty bins add 0.
 */
int orc_entropy(const uint64_t *counts, int m, double *H_out)
{
    if (!counts || !H_out || m < 1) return ORC_EINVAL;
    uint64_t tot = 0;
    for (int i = 0; i < m; ++i) tot += counts[i];
    double H = 0.0;
    if (tot > 0)
        for (int i = 0; i < m; ++i)
            if (counts[i]) {
                double p = (double)counts[i] / (double)tot;
                H -= p * log2(p);
            }
    *H_out = H;
    return ORC_OK;
}

/* ------------------------------------------- differentiable dense render */

/*
 * Rendering of a dense FP64 volume of intensities (the reduced volume that is
 * fitted so that its renders match renders of the full-resolution source,
 * the reduction goal of the previews, Sec. I / Sec. III).  Geometry, sample
 * positions, trilinear interpolation, the transfer-function lookup and the
 * compositing are those of orc_render, with the raw value already an
 * intensity: v = min(max(raw, 0), 1); vol is [mz][my][mx], lut is double
 * [nlut][4] (straight colour).  rgba gets the premultiplied (C, A) of every
 * listed pixel (all pixels when pixels is NULL), nsamp the samples taken.
 */
typedef struct {
    int64_t idx[8];  /* corner voxel indices (clamped), order (x,y,z) bits 0,1,2 */
    double w[8];     /* trilinear weights */
    double raw;      /* interpolated value before the clamp */
} orc_tap;

static void dense_tap(const double *vol, const int64_t M[3], const double q[3], orc_tap *tp)
{
    int64_t i0[3], i1[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double fl = floor(q[a]);
        f[a] = q[a] - fl;
        i0[a] = clampi((int64_t)fl, 0, M[a] - 1);
        i1[a] = clampi((int64_t)fl + 1, 0, M[a] - 1);
    }
    double raw = 0.0;
    for (int c = 0; c < 8; ++c) {
        int64_t x = (c & 1) ? i1[0] : i0[0], y = (c & 2) ? i1[1] : i0[1], z = (c & 4) ? i1[2] : i0[2];
        double w = ((c & 1) ? f[0] : 1.0 - f[0]) * ((c & 2) ? f[1] : 1.0 - f[1]) * ((c & 4) ? f[2] : 1.0 - f[2]);
        tp->idx[c] = (z * M[1] + y) * M[0] + x;
        tp->w[c] = w;
        raw += w * vol[tp->idx[c]];
    }
    tp->raw = raw;
}

typedef struct {
    double b[3];
    float bf[3], rf[3], uf[3], L, c[3], N[3], delta;
} orc_cam;

static void dense_camera(int64_t mx, int64_t my, int64_t mz, int64_t nx, int64_t ny, int64_t nz,
                         const orc_view *view, orc_cam *cam)
{
    const double PI = 3.14159265358979323846;
    double az = ((double)view->az_deg * PI) / 180.0;
    double el = ((double)view->el_deg * PI) / 180.0;
    cam->bf[0] = (float)(cos(el) * cos(az));
    cam->bf[1] = (float)(cos(el) * sin(az));
    cam->bf[2] = (float)sin(el);
    cam->rf[0] = (float)(-sin(az));
    cam->rf[1] = (float)cos(az);
    cam->rf[2] = 0.0f;
    cam->uf[0] = (float)(-sin(el) * cos(az));
    cam->uf[1] = (float)(-sin(el) * sin(az));
    cam->uf[2] = (float)cos(el);
    cam->L = (float)sqrt((double)(nx * nx + ny * ny + nz * nz));
    cam->N[0] = (float)nx;
    cam->N[1] = (float)ny;
    cam->N[2] = (float)nz;
    for (int a = 0; a < 3; ++a) cam->c[a] = cam->N[a] / 2.0f;
    float s[3] = {cam->N[0] / (float)mx, cam->N[1] / (float)my, cam->N[2] / (float)mz};
    cam->delta = view->step * fminf(s[0], fminf(s[1], s[2]));
}

/* Transfer function at intensity v: rgba, entry j and fraction f. */
static void dense_lookup(const double *lut, int nlut, double v, double rgba[4], int64_t *j, double *f)
{
    double x = v * (double)(nlut - 1);
    int64_t jj = (int64_t)floor(x);
    if (jj > nlut - 2) jj = nlut - 2;
    double ff = x - (double)jj;
    for (int ch = 0; ch < 4; ++ch) rgba[ch] = lut[jj * 4 + ch] * (1.0 - ff) + lut[(jj + 1) * 4 + ch] * ff;
    *j = jj;
    *f = ff;
}

static int dense_args_ok(const double *vol, int64_t mx, int64_t my, int64_t mz, int64_t nx, int64_t ny,
                         int64_t nz, const double *lut, int nlut, const orc_view *view)
{
    if (!vol || !lut || !view || nlut < 2) return 0;
    if (mx <= 0 || my <= 0 || mz <= 0 || nx <= 0 || ny <= 0 || nz <= 0) return 0;
    if (view->width <= 0 || view->height <= 0 || !(view->step > 0.0f)) return 0;
    return 1;
}

/* One ray of the dense render, marched until its opacity reaches the highest
 * of the three stop levels stops[0] <= stops[1] <= stops[2]; out[s] and cnt[s]
 * hold (C, A) and the number of samples at the first sample where A >= stops[s]
 * (the last sample when A never gets there). */
static void dense_ray(const double *vol, const int64_t M[3], const double Nd[3], const double *lut, int nlut,
                      const orc_ray *ray, const double stops[3], double out[3][4], uint64_t cnt[3])
{
    double C[3] = {0, 0, 0}, A = 0.0;
    int done[3] = {0, 0, 0};
    int64_t k = 0;
    while (k < ray->n && !done[2]) {
        double t = (double)ray->t_near + ((double)k + 0.5) * (double)ray->delta;
        double q[3];
        for (int a = 0; a < 3; ++a) q[a] = (((double)ray->o[a] + t * (double)ray->d[a]) * (double)M[a]) / Nd[a] - 0.5;
        orc_tap tp;
        dense_tap(vol, M, q, &tp);
        double v = tp.raw < 0.0 ? 0.0 : (tp.raw > 1.0 ? 1.0 : tp.raw);
        double e[4];
        int64_t j;
        double f;
        dense_lookup(lut, nlut, v, e, &j, &f);
        double w = (1.0 - A) * e[3];
        C[0] += w * e[0];
        C[1] += w * e[1];
        C[2] += w * e[2];
        A += w;
        ++k;
        for (int s2 = 0; s2 < 3; ++s2) {
            if (!done[s2] && A >= stops[s2]) {
                done[s2] = 1;
                out[s2][0] = C[0]; out[s2][1] = C[1]; out[s2][2] = C[2]; out[s2][3] = A;
                cnt[s2] = (uint64_t)k;
            }
        }
    }
    for (int s2 = 0; s2 < 3; ++s2) {
        if (!done[s2]) {
            out[s2][0] = C[0]; out[s2][1] = C[1]; out[s2][2] = C[2]; out[s2][3] = A;
            cnt[s2] = (uint64_t)k;
        }
    }
}

/*
 * The dense render with the early-exit band of orc_render: rgba (stop at
 * alpha_stop), rgba_lo (at alpha_stop - eps) and rgba_hi (at alpha_stop + eps),
 * nsamp[p][3] the three sample counts; rgba_lo, rgba_hi and nsamp may be NULL.
 * A ray whose lo and hi results differ may stop anywhere between them in an
 * FP32 march (several results are correct).
 */
int orc_render_dense_band(const double *vol, int64_t mx, int64_t my, int64_t mz, int64_t nx, int64_t ny,
                          int64_t nz, const double *lut, int nlut, double alpha_stop, double eps,
                          const orc_view *view, const int64_t *pixels, int64_t npix, double *rgba,
                          double *rgba_lo, double *rgba_hi, uint64_t *nsamp)
{
    if (!dense_args_ok(vol, mx, my, mz, nx, ny, nz, lut, nlut, view) || !rgba || !(eps >= 0.0)) return ORC_EINVAL;
    orc_cam cam;
    dense_camera(mx, my, mz, nx, ny, nz, view, &cam);
    const int64_t M[3] = {mx, my, mz};
    const double Nd[3] = {(double)nx, (double)ny, (double)nz};
    const double stops[3] = {alpha_stop - eps, alpha_stop, alpha_stop + eps};
    const int64_t W = view->width, H = view->height;
    const int64_t total = pixels ? npix : W * H;
    for (int64_t p = 0; p < total; ++p) {
        int64_t lin = pixels ? pixels[p] : p;
        if (lin < 0 || lin >= W * H) return ORC_EINVAL;
        orc_ray ray;
        ray_setup(cam.bf, cam.rf, cam.uf, cam.L, cam.c, cam.N, cam.delta, view->width, view->height, lin % W,
                  lin / W, &ray);
        double out[3][4];
        uint64_t cnt[3];
        dense_ray(vol, M, Nd, lut, nlut, &ray, stops, out, cnt);
        for (int ch = 0; ch < 4; ++ch) {
            rgba[p * 4 + ch] = out[1][ch];
            if (rgba_lo) rgba_lo[p * 4 + ch] = out[0][ch];
            if (rgba_hi) rgba_hi[p * 4 + ch] = out[2][ch];
        }
        if (nsamp) { nsamp[p * 3 + 0] = cnt[0]; nsamp[p * 3 + 1] = cnt[1]; nsamp[p * 3 + 2] = cnt[2]; }
    }
    return ORC_OK;
}

int orc_render_dense(const double *vol, int64_t mx, int64_t my, int64_t mz, int64_t nx, int64_t ny, int64_t nz,
                     const double *lut, int nlut, double alpha_stop, const orc_view *view,
                     const int64_t *pixels, int64_t npix, double *rgba, uint64_t *nsamp)
{
    if (!dense_args_ok(vol, mx, my, mz, nx, ny, nz, lut, nlut, view) || !rgba) return ORC_EINVAL;
    orc_cam cam;
    dense_camera(mx, my, mz, nx, ny, nz, view, &cam);
    const int64_t M[3] = {mx, my, mz};
    const double Nd[3] = {(double)nx, (double)ny, (double)nz};
    const double stops[3] = {alpha_stop, alpha_stop, alpha_stop};
    const int64_t W = view->width, H = view->height;
    const int64_t total = pixels ? npix : W * H;
    for (int64_t p = 0; p < total; ++p) {
        int64_t lin = pixels ? pixels[p] : p;
        if (lin < 0 || lin >= W * H) return ORC_EINVAL;
        orc_ray ray;
        ray_setup(cam.bf, cam.rf, cam.uf, cam.L, cam.c, cam.N, cam.delta, view->width, view->height, lin % W,
                  lin / W, &ray);
        double out[3][4];
        uint64_t cnt[3];
        dense_ray(vol, M, Nd, lut, nlut, &ray, stops, out, cnt);
        for (int ch = 0; ch < 4; ++ch) rgba[p * 4 + ch] = out[1][ch];
        if (nsamp) nsamp[p] = cnt[1];
    }
    return ORC_OK;
}

/*
 * Gradient of sum_p g_rgba[p] . rgba[p] of orc_render_dense with respect to
 * the volume and the transfer function (accumulated into g_vol, g_lut).
 * Reverse-mode differentiation of the compositing recurrence
 *   w_k = (1 - A_k) alpha_k,  C_{k+1} = C_k + w_k c_k,  A_{k+1} = A_k + w_k,
 * over each ray's stored list of samples (the stop index is held fixed):
 * with adjoints gC (constant along the ray) and gA_{k+1},
 *   gw = gC . c_k + gA_{k+1};   g c_k = gC w_k;   g alpha_k = gw (1 - A_k);
 *   gA_k = gA_{k+1} - gw alpha_k.
 * Then the lookup: g lut[j] += (1-f) g e, g lut[j+1] += f g e, and
 * g v = (nlut-1) sum_ch g e_ch (lut[j+1]_ch - lut[j]_ch) inside 0 < raw < 1
 * (0 where the clamp is active); g vol[corner] += w_corner g v.
 * g_vol_mag / g_lut_mag (may be NULL) receive, per element, the sum of the
 * absolute values of the terms added into it: the scale against which the
 * rounding error of any order of summing those terms is measured.
 */
int orc_render_dense_grad(const double *vol, int64_t mx, int64_t my, int64_t mz, int64_t nx, int64_t ny,
                          int64_t nz, const double *lut, int nlut, double alpha_stop, const orc_view *view,
                          const double *g_rgba, double *g_vol, double *g_lut, double *g_vol_mag,
                          double *g_lut_mag)
{
    if (!dense_args_ok(vol, mx, my, mz, nx, ny, nz, lut, nlut, view) || !g_rgba || !g_vol || !g_lut)
        return ORC_EINVAL;
    orc_cam cam;
    dense_camera(mx, my, mz, nx, ny, nz, view, &cam);
    const int64_t M[3] = {mx, my, mz};
    const double Nd[3] = {(double)nx, (double)ny, (double)nz};
    const int64_t W = view->width, H = view->height;
    /* per-ray sample list: tap, A before the sample, rgba, j, f */
    int64_t cap = 0;
    orc_tap *taps = NULL;
    double *Ak = NULL, *E = NULL, *F = NULL;
    int64_t *J = NULL;
    int rc = ORC_OK;
    for (int64_t lin = 0; lin < W * H && rc == ORC_OK; ++lin) {
        orc_ray ray;
        ray_setup(cam.bf, cam.rf, cam.uf, cam.L, cam.c, cam.N, cam.delta, view->width, view->height, lin % W,
                  lin / W, &ray);
        if (ray.n > cap) {
            cap = ray.n;
            free(taps); free(Ak); free(E); free(F); free(J);
            taps = (orc_tap *)malloc((size_t)cap * sizeof(orc_tap));
            Ak = (double *)malloc((size_t)cap * sizeof(double));
            E = (double *)malloc((size_t)cap * 4 * sizeof(double));
            F = (double *)malloc((size_t)cap * sizeof(double));
            J = (int64_t *)malloc((size_t)cap * sizeof(int64_t));
            if (!taps || !Ak || !E || !F || !J) { rc = ORC_EINVAL; break; }
        }
        double A = 0.0;
        int64_t n = 0;
        while (n < ray.n) {
            double t = (double)ray.t_near + ((double)n + 0.5) * (double)ray.delta;
            double q[3];
            for (int a = 0; a < 3; ++a) q[a] = (((double)ray.o[a] + t * (double)ray.d[a]) * (double)M[a]) / Nd[a] - 0.5;
            dense_tap(vol, M, q, &taps[n]);
            double raw = taps[n].raw;
            double v = raw < 0.0 ? 0.0 : (raw > 1.0 ? 1.0 : raw);
            dense_lookup(lut, nlut, v, &E[n * 4], &J[n], &F[n]);
            Ak[n] = A;
            A += (1.0 - A) * E[n * 4 + 3];
            ++n;
            if (A >= alpha_stop) break;
        }
        const double *g = &g_rgba[lin * 4];
        double gA = g[3];
        for (int64_t k = n - 1; k >= 0; --k) {
            const double *e = &E[k * 4];
            double w = (1.0 - Ak[k]) * e[3];
            double gw = g[0] * e[0] + g[1] * e[1] + g[2] * e[2] + gA;
            double ge[4] = {g[0] * w, g[1] * w, g[2] * w, gw * (1.0 - Ak[k])};
            gA = gA - gw * e[3];
            int64_t j = J[k];
            double f = F[k];
            double gv = 0.0;
            for (int ch = 0; ch < 4; ++ch) {
                g_lut[j * 4 + ch] += (1.0 - f) * ge[ch];
                g_lut[(j + 1) * 4 + ch] += f * ge[ch];
                if (g_lut_mag) {
                    g_lut_mag[j * 4 + ch] += fabs((1.0 - f) * ge[ch]);
                    g_lut_mag[(j + 1) * 4 + ch] += fabs(f * ge[ch]);
                }
                gv += ge[ch] * (lut[(j + 1) * 4 + ch] - lut[j * 4 + ch]);
            }
            gv *= (double)(nlut - 1);
            if (!(taps[k].raw > 0.0 && taps[k].raw < 1.0)) gv = 0.0;
            for (int c = 0; c < 8; ++c) {
                g_vol[taps[k].idx[c]] += taps[k].w[c] * gv;
                if (g_vol_mag) g_vol_mag[taps[k].idx[c]] += fabs(taps[k].w[c] * gv);
            }
        }
    }
    free(taps); free(Ak); free(E); free(F); free(J);
    return rc;
}

/*
 * 256-bin grey-level histogram of a rendered image, the p_i of Eq. 2
 * (Sec. III-C).  Reading: the image is the premultiplied RGBA render shown
 * over a black background; its grey level is the Rec. 709 luminance
 * lum = (0.2126 R + 0.7152 G) + 0.0722 B, computed in FP32 in this order
 * (one rounding per operation), clamped to [0, 1] and quantised to 8 bits
 * as floor(lum * 255 + 0.5).
 */
int orc_image_histogram(const float *rgba, int64_t npix, uint64_t *hist)
{
    if ((!rgba && npix) || !hist || npix < 0) return ORC_EINVAL;
    for (int i = 0; i < 256; ++i) hist[i] = 0;
    for (int64_t p = 0; p < npix; ++p) {
        float lum = (0.2126f * rgba[p * 4 + 0] + 0.7152f * rgba[p * 4 + 1]) + 0.0722f * rgba[p * 4 + 2];
        lum = lum < 0.0f ? 0.0f : (lum > 1.0f ? 1.0f : lum);
        if (!(lum == lum)) lum = 0.0f; /* NaN counts as black */
        int q = (int)floorf(lum * 255.0f + 0.5f);
        hist[q] += 1;
    }
    return ORC_OK;
}

/* ------------------------------------------------------ container removal */

/*
 * Container circle of one slice (Sec. III, Container Removal: a Hough circle
 * transform on the top slice; everything outside the circle is then dropped
 * from every slice).  The cited transform (Ioannou, Huda and Laine 1999) finds
 * the centre by a 2D vote along each edge pixel's gradient line and the radius
 * from a histogram of edge distances; the paper gives no further detail.
 * Reading, step by step (integers unless stated):
 *  1. Smooth: b = separable [1 4 6 4 1] x [1 4 6 4 1] filter of the slice,
 *     indices clamped at the borders (b is 256 x the grey scale).
 *  2. Sobel gradient of b at interior pixels 1..nx-2, 1..ny-2:
 *     gx = (b[y-1][x+1] + 2 b[y][x+1] + b[y+1][x+1]) - (same at x-1), gy likewise.
 *  3. Edge pixel: gx^2 + gy^2 >= (256 thr)^2.
 *  4. Unit gradient in FP32, one rounding per operation:
 *     m = sqrt((float)(gx^2 + gy^2)), ux = (float)gx / m, uy = (float)gy / m.
 *  5. Coarse centre: for t = rmin..rmax the point (x - t ux, y - t uy) (FP32)
 *     votes for its cell (floor(fx / s), floor(fy / s)) of a grid of s x s
 *     pixel cells (votes against the gradient: the circle whose inside is
 *     darker than its rim, the container's inner wall around the air inside);
 *     the cell with most votes (lowest row, then column, on ties) gives the
 *     centre (cx, cy) = (cell * s + (s - 1) / 2) in FP64.
 *  6. Coarse radius: over edge pixels whose gradient points away from the
 *     centre ((x - cx) ux + (y - cy) uy > 0, FP64), r = floor(d + 1/2),
 *     d = sqrt((x - cx)^2 + (y - cy)^2) (FP64), counted for rmin <= r <= rmax;
 *     the most frequent r (smallest on ties).
 *  7. Refinement (an addition: the Hough cells are s pixels wide): three
 *     least-squares circle fits (Kasa) over the outward edge pixels with
 *     |d - r| <= w, w = 2s + 3, s + 3, 3: minimise sum (x^2 + y^2 + D x + E y
 *     + F)^2 from exact integer moment sums, solved by Cramer's rule in FP64;
 *     centre (-D/2, -E/2), radius sqrt(cx^2 + cy^2 - F).  A fit with fewer
 *     than 3 pixels or a zero determinant keeps the previous circle.
 *  8. Result: centre (floor(cx + 1/2), floor(cy + 1/2)), radius floor(r); when
 *     no outward edge pixel falls in [rmin, rmax] there is no circle: (0, 0, -1).
 * acc (ceil(ny/s) * ceil(nx/s)) and rhist (rmax + 1) receive the vote counts,
 * fit (3 doubles) the refined circle, when not NULL.
 */
typedef struct {
    int64_t x, y;
    float ux, uy;
} orc_edge;

static int64_t clamp64(int64_t v, int64_t hi) { return v < 0 ? 0 : (v > hi ? hi : v); }

int orc_hough_circle(const void *slice, int esize, int64_t nx, int64_t ny, int64_t thr, int rmin, int rmax, int s,
                     uint32_t *acc, uint32_t *rhist, double *fit, int32_t *cx_out, int32_t *cy_out, int32_t *r_out)
{
    if (!slice || (esize != 1 && esize != 2) || nx < 3 || ny < 3 || thr < 1 || rmin < 0 || rmax < rmin || s < 1 ||
        !cx_out || !cy_out || !r_out)
        return ORC_EINVAL;
    const int64_t k5[5] = {1, 4, 6, 4, 1};
    int64_t *tmp = (int64_t *)malloc((size_t)(nx * ny) * sizeof(int64_t));
    int64_t *b = (int64_t *)malloc((size_t)(nx * ny) * sizeof(int64_t));
    orc_edge *E = (orc_edge *)malloc((size_t)(nx * ny) * sizeof(orc_edge));
    const int64_t gxn = (nx + s - 1) / s, gyn = (ny + s - 1) / s;
    uint32_t *A = acc ? acc : (uint32_t *)malloc((size_t)(gxn * gyn) * sizeof(uint32_t));
    uint32_t *R = rhist ? rhist : (uint32_t *)malloc(((size_t)rmax + 1) * sizeof(uint32_t));
    if (!tmp || !b || !E || !A || !R) {
        free(tmp); free(b); free(E);
        if (!acc) free(A);
        if (!rhist) free(R);
        return ORC_EINVAL;
    }
    memset(A, 0, (size_t)(gxn * gyn) * sizeof(uint32_t));
    memset(R, 0, ((size_t)rmax + 1) * sizeof(uint32_t));
    /* 1. smoothing, x then y */
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            int64_t v = 0;
            for (int i = 0; i < 5; ++i) v += k5[i] * (int64_t)load_voxel(slice, esize, y * nx + clamp64(x + i - 2, nx - 1));
            tmp[y * nx + x] = v;
        }
    for (int64_t y = 0; y < ny; ++y)
        for (int64_t x = 0; x < nx; ++x) {
            int64_t v = 0;
            for (int i = 0; i < 5; ++i) v += k5[i] * tmp[clamp64(y + i - 2, ny - 1) * nx + x];
            b[y * nx + x] = v;
        }
    /* 2-4. edges and their unit gradients */
    const int64_t t2 = (256 * thr) * (256 * thr);
    int64_t ne = 0;
    for (int64_t y = 1; y < ny - 1; ++y)
        for (int64_t x = 1; x < nx - 1; ++x) {
#define B(xx, yy) b[(yy) * nx + (xx)]
            int64_t gx = (B(x + 1, y - 1) + 2 * B(x + 1, y) + B(x + 1, y + 1)) - (B(x - 1, y - 1) + 2 * B(x - 1, y) + B(x - 1, y + 1));
            int64_t gy = (B(x - 1, y + 1) + 2 * B(x, y + 1) + B(x + 1, y + 1)) - (B(x - 1, y - 1) + 2 * B(x, y - 1) + B(x + 1, y - 1));
#undef B
            int64_t g2 = gx * gx + gy * gy;
            if (g2 < t2) continue;
            float m = sqrtf((float)g2);
            E[ne].x = x;
            E[ne].y = y;
            E[ne].ux = (float)gx / m;
            E[ne].uy = (float)gy / m;
            ++ne;
        }
    /* 5. coarse centre */
    for (int64_t e = 0; e < ne; ++e)
        for (int t = rmin; t <= rmax; ++t) {
            float fx = (float)E[e].x - (float)t * E[e].ux, fy = (float)E[e].y - (float)t * E[e].uy;
            if (!(fx >= 0.0f && fy >= 0.0f)) continue;
            int64_t ix = (int64_t)floorf(fx / (float)s), iy = (int64_t)floorf(fy / (float)s);
            if (ix < gxn && iy < gyn) A[iy * gxn + ix] += 1;
        }
    int64_t best = 0;
    for (int64_t i = 1; i < gxn * gyn; ++i)
        if (A[i] > A[best]) best = i;
    double cx = (double)((best % gxn) * s) + (double)(s - 1) / 2.0;
    double cy = (double)((best / gxn) * s) + (double)(s - 1) / 2.0;
    /* 6. coarse radius */
    for (int64_t e = 0; e < ne; ++e) {
        double dx = (double)E[e].x - cx, dy = (double)E[e].y - cy;
        if (!(dx * (double)E[e].ux + dy * (double)E[e].uy > 0.0)) continue;
        int64_t r = (int64_t)floor(sqrt(dx * dx + dy * dy) + 0.5);
        if (r >= rmin && r <= rmax) R[r] += 1;
    }
    int rbest = rmin;
    for (int r = rmin + 1; r <= rmax; ++r)
        if (R[r] > R[rbest]) rbest = r;
    double rf = (double)rbest;
    /* 7. refinement */
    const double bands[3] = {2.0 * s + 3.0, (double)s + 3.0, 3.0};
    for (int it = 0; it < 3 && ne > 0 && R[rbest] > 0; ++it) {
        int64_t n = 0, sxx = 0, sxy = 0, sx = 0, syy = 0, sy = 0, sz = 0, sxz = 0, syz = 0;
        for (int64_t e = 0; e < ne; ++e) {
            double dx = (double)E[e].x - cx, dy = (double)E[e].y - cy;
            if (!(dx * (double)E[e].ux + dy * (double)E[e].uy > 0.0)) continue;
            if (!(fabs(sqrt(dx * dx + dy * dy) - rf) <= bands[it])) continue;
            int64_t x = E[e].x, y = E[e].y, z = x * x + y * y;
            ++n; sxx += x * x; sxy += x * y; sx += x; syy += y * y; sy += y; sz += z; sxz += x * z; syz += y * z;
        }
        if (n < 3) break;
        double a11 = (double)sxx, a12 = (double)sxy, a13 = (double)sx, a22 = (double)syy, a23 = (double)sy;
        double a33 = (double)n, b1 = -(double)sxz, b2 = -(double)syz, b3 = -(double)sz;
        double det = a11 * (a22 * a33 - a23 * a23) - a12 * (a12 * a33 - a23 * a13) + a13 * (a12 * a23 - a22 * a13);
        if (det == 0.0) break;
        double dD = b1 * (a22 * a33 - a23 * a23) - a12 * (b2 * a33 - a23 * b3) + a13 * (b2 * a23 - a22 * b3);
        double dE = a11 * (b2 * a33 - b3 * a23) - b1 * (a12 * a33 - a23 * a13) + a13 * (a12 * b3 - b2 * a13);
        double dF = a11 * (a22 * b3 - a23 * b2) - a12 * (a12 * b3 - b2 * a13) + b1 * (a12 * a23 - a22 * a13);
        double D = dD / det, Ee = dE / det, F = dF / det;
        double ncx = -D / 2.0, ncy = -Ee / 2.0, rr2 = ncx * ncx + ncy * ncy - F;
        if (!(rr2 > 0.0)) break;
        cx = ncx;
        cy = ncy;
        rf = sqrt(rr2);
    }
    if (ne == 0 || R[rbest] == 0) {
        cx = 0.0;
        cy = 0.0;
        rf = -1.0;
    }
    *cx_out = (int32_t)floor(cx + 0.5);
    *cy_out = (int32_t)floor(cy + 0.5);
    *r_out = (int32_t)floor(rf);
    if (fit) { fit[0] = cx; fit[1] = cy; fit[2] = rf; }
    free(tmp); free(b); free(E);
    if (!acc) free(A);
    if (!rhist) free(R);
    return ORC_OK;
}

/* Drop everything outside the container (Sec. III, Container Removal): voxel
 * (x, y, z) keeps its value when (x - cx)^2 + (y - cy)^2 <= r_keep^2, else 0
 * (the keep/discard sense of Sec. III-A: "removed" means zero).  r_keep < 0
 * means no container was found: everything is kept. */
int orc_mask_circle(const void *in, int esize, int64_t nx, int64_t ny, int64_t nz, int32_t cx, int32_t cy,
                    int32_t r_keep, void *out)
{
    if (!in || !out || (esize != 1 && esize != 2) || nx < 1 || ny < 1 || nz < 1) return ORC_EINVAL;
    const int64_t rk2 = (int64_t)r_keep * r_keep;
    for (int64_t z = 0; z < nz; ++z)
        for (int64_t y = 0; y < ny; ++y)
            for (int64_t x = 0; x < nx; ++x) {
                int64_t i = (z * ny + y) * nx + x;
                int64_t d2 = (x - cx) * (x - cx) + (y - cy) * (y - cy);
                store_voxel(out, esize, i, (r_keep < 0 || d2 <= rk2) ? load_voxel(in, esize, i) : 0u);
            }
    return ORC_OK;
}
