/*
 * mctp.h -- C ABI of libmctp, the GB300 (sm_103a) micro-CT preview library.
 *
 * The library computes the data-parallel hot path of the preview pipeline of
 * "Low-latency Visual Previews of Large Synchrotron Micro-CT Datasets"
 * (arXiv 2311.15038): a voxel histogram, threshold selection (Otsu, Alg. 1;
 * iterative threshold selection, Alg. 2; top-slice histogram filtering,
 * Sec. III-D), the binary keep/discard classification of voxels (Sec. III-A),
 * box-filtered multi-resolution slicemap atlases (Sec. II "Interactive
 * Preview", Sec. III), and server-side direct volume rendering of a slicemap
 * (Sec. III-C).
 *
 * Conventions for every call:
 *  - Pointers named "device" are CUDA device pointers owned by the caller;
 *    descriptor structs are host memory read during the call only.  The
 *    library never keeps a pointer after a call returns and allocates no
 *    device memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on it and the call returns without waiting;
 *    outputs are valid once the stream has been synchronised.
 *  - Return value: MCTP_OK, or a negative code from the list below, detected
 *    on the host before anything is enqueued (MCTP_ECUDA: a launch failed).
 *  - Volumes are dense [nz][ny][nx] arrays, x fastest:
 *    voxel (x,y,z) at index (z*ny + y)*nx + x.
 *  - A grey value has `bits` significant bits; values >= 2^bits are outside
 *    the declared depth (counted as overflow, never kept by a filter).
 *  - Histogram bins: nbins is a power of two with 1 <= nbins <= 2^bits, and
 *    value v falls in bin v >> (bits - log2(nbins)).
 *  - No call faults or traps on bad input it can see: host checks return an
 *    error code instead.
 */
#ifndef MCTP_H
#define MCTP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCTP_ABI_VERSION 1

/* status codes */
#define MCTP_OK 0
#define MCTP_EINVAL (-1)       /* null pointer, bad size, bad nbins, bad level chain */
#define MCTP_EUNSUPPORTED (-2) /* dtype / bits / mode not supported */
#define MCTP_ESIZE (-3)        /* atlas tile grid too small, too many views */
#define MCTP_ECUDA (-4)        /* a CUDA launch or copy failed */
#define MCTP_ECANCELED (-6)    /* serving: the request was cancelled before its launch */

/* voxel types */
#define MCTP_U8 1
#define MCTP_U16 2

typedef struct {
    int64_t nx, ny, nz; /* voxels per axis, each >= 1 */
    int32_t dtype;      /* MCTP_U8 (bits must be 8) or MCTP_U16 (bits 1..16) */
    int32_t bits;
} mctp_volume_desc;

/* threshold selection modes */
#define MCTP_THR_OTSU 0     /* Alg. 1: keep bins >= T_otsu */
#define MCTP_THR_ITS 1      /* Alg. 2: keep bins >= ceil(T_it) */
#define MCTP_THR_TOPSLAB 2  /* Sec. III-D: keep bins absent from the top slices */
#define MCTP_THR_EXPLICIT 3 /* keep bins >= explicit_T */

typedef struct {
    int32_t mode;         /* one of MCTP_THR_* */
    int32_t explicit_T;   /* MCTP_THR_EXPLICIT: first kept bin */
    int32_t its_max_iter; /* MCTP_THR_ITS: iteration cap, >= 1 (256 is a good default) */
    int32_t reserved;
    uint64_t topslab_kmin;/* MCTP_THR_TOPSLAB: a bin is removed once its top-slab count >= kmin (>= 1) */
} mctp_thr_params;

#define MCTP_MAX_LEVELS 8

/*
 * A multi-resolution slicemap: level k is an mx*my*mz volume stored as a 2D
 * atlas of tiles_x * tiles_y tiles of mx*my voxels, one tile per z slice.
 * Slice z sits in tile row z / tiles_x, column z % tiles_x; voxel (x,y,z) at
 *   atlas[k][(row*my + y) * (tiles_x*mx) + col*mx + x]
 * (elements of the source dtype).  Tiles past the last slice are zero.
 * Level 0 is an area-box reduction of the source volume; level k >= 1 is the
 * exact 2x2x2 box reduction of level k-1, so its dims are exactly half.
 * The world box of every level is the source box [0,nx]x[0,ny]x[0,nz].
 */
typedef struct {
    int32_t nlevels;                  /* 1..MCTP_MAX_LEVELS */
    int32_t dtype;                    /* element type of the atlases (= source dtype) */
    int32_t bits;                     /* grey-value depth (= source bits) */
    int32_t reserved;
    int64_t src_dims[3];              /* nx, ny, nz of the source volume */
    int32_t dims[MCTP_MAX_LEVELS][3]; /* mx, my, mz of each level */
    int32_t tiles_x[MCTP_MAX_LEVELS];
    int32_t tiles_y[MCTP_MAX_LEVELS];
    void *atlas[MCTP_MAX_LEVELS];     /* device, (tiles_y*my) x (tiles_x*mx) elements each */
    void *maxgrid[MCTP_MAX_LEVELS];   /* device or NULL: per-cell maxima of the level (below) */
    uint64_t texture[MCTP_MAX_LEVELS];/* 0 or the handle of an atlas texture of level k (below) */
} mctp_slicemap;

/* Occupancy data of a level (an acceleration structure of this library; the
 * paper has none): maxgrid[k] holds, for every cell of MCTP_MAXGRID_CELL^3
 * voxels, the maximum over the voxels [c*8, c*8 + 8] per axis (the cell plus
 * one voxel, clamped to the level) as uint16, cells laid out
 * [ceil(mz/8)][ceil(my/8)][ceil(mx/8)].  build_slicemap fills it when the
 * pointer is not NULL; render_views then evaluates only samples whose cell
 * can reach a transfer-function opacity above zero.  Skipped samples have
 * opacity exactly zero, so images and sample counts are unchanged. */
#define MCTP_MAXGRID_CELL 8

/*
 * Atlas textures (an option of this library's renderers).  The paper's
 * client samples each atlas as a 2D texture (Sec. III-B/C); here a level's
 * atlas can be copied into a 2D CUDA array with a texture object, and when
 * sm->texture[k] holds its handle, mctp_render_batch (and the server) fetch
 * a sample's four in-slice corners with one texture gather per slice instead
 * of four loads.  The gathered values are the atlas values, so images and
 * sample counts are bit-identical with and without a texture.
 *   mctp_atlas_texture_create  allocates the array for level `level` of *sm
 *       ((tiles_y*my) x (tiles_x*mx) elements of its dtype) and its texture
 *       object; *out owns both, *handle receives the value for
 *       sm->texture[level].  The contents are undefined until an update.
 *   mctp_atlas_texture_update  copies atlas[level] into the array (device to
 *       device, on `stream`); call it after every mctp_build_slicemap of
 *       that slicemap, before rendering.  The slicemap must have the same
 *       level geometry and dtype as at creation.
 *   mctp_atlas_texture_destroy frees both (NULL is allowed); the caller
 *       makes sure no launch that uses the handle is still running.
 * Errors: MCTP_EINVAL (null pointers, bad slicemap or level, geometry
 *         differing from creation), MCTP_ESIZE (atlas wider or taller than
 *         the device's texture-gather limit, 32768 on this part),
 *         MCTP_ECUDA (allocation or copy failed).
 */
typedef struct mctp_atlas_texture mctp_atlas_texture;
int mctp_atlas_texture_create(const mctp_slicemap *sm, int32_t level, mctp_atlas_texture **out, uint64_t *handle);
int mctp_atlas_texture_update(mctp_atlas_texture *t, const mctp_slicemap *sm, int32_t level, void *stream);
/* mctp_atlas_texture_update for `count` textures in one launch: textures[i]
 * receives level levels[i] of sms[i] (host arrays of count entries; every
 * slicemap of one dtype).  Errors as mctp_atlas_texture_update, MCTP_EINVAL
 * also for count < 0 or mixed dtypes; count == 0 launches nothing. */
int mctp_atlas_texture_update_batch(mctp_atlas_texture *const *textures, const mctp_slicemap *sms,
                                    const int32_t *levels, int32_t count, void *stream);
int mctp_atlas_texture_destroy(mctp_atlas_texture *t);

/* One orthographic view of a slicemap level.  The camera looks at the centre
 * of the source box from azimuth az (about +z, from +x) and elevation el;
 * image right = (-sin az, cos az, 0), image up = (-sin el cos az,
 * -sin el sin az, cos el); the square image plane has the side of the box
 * diagonal.  step is the sample spacing in units of the smallest voxel edge
 * of the level. */
typedef struct {
    float azimuth_deg;
    float elevation_deg;
    int32_t width, height; /* pixels, >= 1 */
    int32_t level;         /* slicemap level to render */
    float step;            /* > 0; 0.5 = half a level voxel */
} mctp_view;

/*
 * Voxel histogram (Sec. III-A: the grey-value histogram that Alg. 1 and
 * Alg. 2 partition; Sec. III-D: the histogram of the top slices).
 *   vol       device, the volume described by *d
 *   z0, z1    slab of slices counted, 0 <= z0 <= z1 <= nz (z1 == z0: empty)
 *   hist      device uint64[nbins], overwritten with the counts
 *   overflow  device uint64[1], overwritten with the number of values >= 2^bits
 * Errors: MCTP_EINVAL (null pointers, dims < 1, bad slab, bad nbins),
 *         MCTP_EUNSUPPORTED (dtype/bits).
 */
int mctp_build_histogram(const void *vol, const mctp_volume_desc *d, int64_t z0, int64_t z1,
                         int32_t nbins, uint64_t *hist, uint64_t *overflow, void *stream);

/*
 * Histograms of `count` whole volumes in one launch (the batched form of
 * mctp_build_histogram over z in [0, nz)): vols[i] described by descs[i]
 * (host arrays of count entries, every volume with the same dtype and bits)
 * counts into hist[i nbins .. (i + 1) nbins) and overflow[i] (device uint64
 * arrays, overwritten).  With at most 256 bins the volumes share one
 * launch, which splits their concatenated 16-byte vectors evenly over the
 * blocks; with more bins each volume takes its own launch.
 * Errors: as mctp_build_histogram; MCTP_EINVAL also for count < 0 or mixed
 *         dtype/bits.
 */
int mctp_build_histogram_batch(const void *const *vols, const mctp_volume_desc *descs, int32_t count,
                               int32_t nbins, uint64_t *hist, uint64_t *overflow, void *stream);

/*
 * Threshold selection -> keep table (Sec. III-A, Alg. 1 and Alg. 2;
 * Sec. III-D histogram filtering).  Computed on the device in FP64 with a
 * fixed evaluation order:
 *   OTSU      T = first bin maximising W_a W_b (U_a - U_b)^2 over the split
 *             [0,T) | [T,nbins); keep[b] = b >= T
 *   ITS       T_it from nbins/2, T_it <- (mu1 + mu2)/2 until it no longer
 *             changes (empty side: mu = T_it) or its_max_iter iterations;
 *             keep[b] = b >= ceil(T_it)
 *   TOPSLAB   `hist` is the histogram of the top slices; keep[b] =
 *             hist[b] < topslab_kmin
 *   EXPLICIT  keep[b] = b >= explicit_T (`hist` may be NULL)
 *   hist      device uint64[nbins]
 *   keep_lut  device uint8[nbins], overwritten with 0/1
 *   result    device int32[4] or NULL: {T (-1 for TOPSLAB), iterations,
 *             converged (1/0), 0}
 * Errors: MCTP_EINVAL (null pointers, nbins < 1 or not a power of two,
 *         nbins > 65536, its_max_iter < 1, kmin < 1), MCTP_EUNSUPPORTED (mode).
 */
int mctp_select_threshold(const uint64_t *hist, int32_t nbins, const mctp_thr_params *p,
                          uint8_t *keep_lut, int32_t *result, void *stream);

/*
 * Threshold selection for `count` histograms in one launch (one block per
 * histogram; the batched form of mctp_select_threshold, for many volumes
 * previewed together).  Histogram i is hist[i nbins .. (i + 1) nbins), its
 * keep table keep_lut[i nbins ..] and its result result[4 i .. 4 i + 3]; each
 * is computed exactly as mctp_select_threshold computes it, with the same
 * params for every histogram.
 *   count     number of histograms, >= 0 (0: nothing is launched)
 * Errors: as mctp_select_threshold; MCTP_EINVAL also for count < 0 or
 *         count > 2^31 / nbins.
 */
int mctp_select_threshold_batch(const uint64_t *hist, int32_t count, int32_t nbins, const mctp_thr_params *p,
                                uint8_t *keep_lut, int32_t *result, void *stream);

/*
 * Binary classification of every voxel (Sec. III-A; bins disposed of by the
 * histogram filter, Sec. III-D): out[i] = in[i] if in[i] < 2^bits and
 * keep_lut[bin(in[i])] != 0, else 0.
 *   in, out   device volumes described by *d; out may equal in (in place),
 *             other overlaps are not allowed
 *   keep_lut  device uint8[nbins]
 * Errors: MCTP_EINVAL, MCTP_EUNSUPPORTED.
 */
int mctp_filter_threshold(const void *in, const mctp_volume_desc *d, const uint8_t *keep_lut,
                          int32_t nbins, void *out, void *stream);

/*
 * Multi-resolution slicemap (Sec. III: slices converted into slicemaps;
 * Sec. II: a coarse dataset is shown before the full one).  Level 0 voxel i
 * along an axis of n source and m level voxels covers source voxels
 * [floor(i n/m), floor((i+1) n/m)); its value is the mean of the covered
 * voxels (after the keep table when keep_lut != NULL), rounded half up.
 * Level k >= 1 is the exact 2x2x2 mean of level k-1, rounded half up.
 *   vol       device source volume described by *d (read once)
 *   keep_lut  device uint8[nbins] or NULL (no filtering)
 *   sm        caller-filled: nlevels, dims, tiles, atlas (and optional
 *             maxgrid) pointers; sm->dtype, sm->bits and sm->src_dims must
 *             match *d.  Every atlas is written in full (unused tiles zeroed)
 *             and every non-NULL maxgrid is filled from its level.
 * Requirements: 1 <= m <= n per axis for level 0; level k dims = level k-1
 * dims / 2 exactly; tiles_x * tiles_y >= mz per level.
 * Errors: MCTP_EINVAL (bad chain or pointers), MCTP_ESIZE (tile grid too
 *         small), MCTP_EUNSUPPORTED.
 */
int mctp_build_slicemap(const void *vol, const mctp_volume_desc *d, const uint8_t *keep_lut,
                        int32_t nbins, const mctp_slicemap *sm, void *stream);

/*
 * mctp_build_slicemap for `count` volumes (many volumes previewed together):
 * vols[i], descs[i] and sms[i] (host arrays of count entries) as in
 * mctp_build_slicemap, keep table keep_luts[i nbins .. (i + 1) nbins) (device
 * uint8[count][nbins], or NULL for no filtering).  Every volume has the same
 * dtype.  The atlases are built volume by volume, on `stream` and two
 * streams forked from it (made once per host thread and device and kept;
 * they join `stream` again before the call returns, so the work stays
 * ordered on `stream` and records into a CUDA graph); the max grids of all
 * volumes' levels are filled in one launch afterwards.  Results equal those
 * of mctp_build_slicemap on each volume.
 * Errors: as mctp_build_slicemap for any volume (nothing is launched then);
 *         MCTP_EINVAL also for count < 0 or mixed dtypes.
 */
int mctp_build_slicemap_batch(const void *const *vols, const mctp_volume_desc *descs, const uint8_t *keep_luts,
                              int32_t nbins, const mctp_slicemap *sms, int32_t count, void *stream);

/*
 * Server-side rendering of slicemap views (Sec. III-C): orthographic
 * emission-absorption ray marching, front to back, per pixel:
 *   ray set-up in FP32 with one rounding per operation, in this order:
 *   sx = (i + 0.5)/W - 0.5, sy = 0.5 - (j + 0.5)/H (j from the top),
 *   o = ((c + (sx L) r) + (sy L) u) + L b, d = -b, with c the box centre,
 *   L = |box diagonal|, b = (cos el cos az, cos el sin az, sin el) and the
 *   basis vectors rounded once from FP64; slab test per axis with
 *   inv = 1/d_a, t = (0 - o_a) inv and (n_a - o_a) inv; Delta = step *
 *   min_a(n_a / m_a); n = floor((t_far - t_near) / Delta) samples at
 *   t_near + (k + 1/2) Delta,
 *   trilinear interpolation of the level (corner indices clamped to the
 *   level), v = min(raw / (2^bits - 1), 1), RGBA = linear interpolation of
 *   lut_rgba at v (nlut - 1), then w = (1 - A) alpha, C += w rgb, A += w,
 *   stopping once A >= alpha_stop.
 *   views     host array of nviews views (any mix of sizes and levels)
 *   lut_rgba  device float[nlut][4], straight (not premultiplied) colour,
 *             2 <= nlut <= 4096
 *   out_rgba  device float; view v is an [height][width][4] premultiplied
 *             RGBA image (row 0 = top) starting after the images of views
 *             0..v-1
 *   samples_taken device uint64[1] or NULL: overwritten with the number of
 *             samples marched over all rays (up to and including the
 *             early-exit sample)
 * Errors: MCTP_EINVAL (null pointers, bad view, bad level, nlut out of
 *         range, alpha_stop not in (0, 1]), MCTP_ESIZE (a view larger than
 *         2^28 pixels).
 */
int mctp_render_views(const mctp_slicemap *sm, const mctp_view *views, int32_t nviews,
                      const float *lut_rgba, int32_t nlut, float alpha_stop, float *out_rgba,
                      uint64_t *samples_taken, void *stream);

/*
 * Batched rendering: the views of many slicemaps in one persistent launch
 * (the paper renders one view per request, Sec. III-C; batching many volumes
 * and views is an extension of this library).  View i is rendered from
 * level views[i].level of sms[view_slicemap[i]] with transfer function
 * view_lut[i], exactly as mctp_render_views would render it alone: images
 * and sample counts are bit-identical.  Work is a queue of 32-ray warp tiles
 * over all views, taken by persistent warps with an atomic counter.
 *   sms           host array of nsm slicemaps, all of one dtype
 *   views, view_slicemap, view_lut  host arrays of nviews entries
 *   luts_rgba     device float[nluts][nlut][4] (layout of mctp_render_views'
 *                 lut_rgba, one table after another), 2 <= nlut <= 4096
 *   tuning        NULL or a mctp_batch_tuning (below); it changes speed only
 *   out_rgba      device float, 16-byte aligned; view i is an
 *                 [height][width][4] image after the images of views 0..i-1
 *   samples_taken device uint64[1] or NULL: overwritten with the samples
 *                 marched over all rays of the batch
 *   workspace     device memory of at least the size that
 *                 mctp_render_batch_workspace gives for the same arguments,
 *                 256-byte aligned, owned by the caller; its contents need no
 *                 initialisation and are rewritten by every call, so two
 *                 calls in flight at once must not share it.  When the call
 *                 has run with MCTP_BATCH_COUNT_EVALUATED, bytes 8..15 of the
 *                 workspace hold (uint64) the number of samples evaluated:
 *                 the samples taken minus those skipped as empty, i.e. the
 *                 samples whose corners were fetched and looked up.
 * When every (slicemap, level) of the batch has an atlas texture
 * (sm->texture[level] != 0), corner quads are gathered through the textures.
 * A set-up kernel rasterises, per view and 16 x 16 pixel tile, the depth
 * range of the level's marked cells (max grid), and each ray marches only
 * the samples in its tile's range (the others lie in unmarked cells): rays
 * that meet no marked cell take no step.  The workspace holds the raster.
 * Everything is enqueued on `stream` (kernel launches and memsets only; no
 * host synchronisation), so a call can be captured in a CUDA graph.
 * Errors: MCTP_EINVAL (null pointers, an index out of range, bad view,
 *         nlut or alpha_stop out of range, bad tuning, misaligned pointer),
 *         MCTP_EUNSUPPORTED (slicemaps of different dtypes), MCTP_ESIZE
 *         (workspace too small, a view larger than 2^28 pixels, more than
 *         2^31 warp tiles in the batch), MCTP_ECUDA.
 */
typedef struct {
    int32_t warp_w;      /* pixels per warp row: 4, 8, 16 or 32 (a warp covers
                            warp_w x 32/warp_w pixels); 0 = 8 */
    int32_t chunk;       /* warp tiles taken per queue access, 1..64; 0 = 2 */
    int32_t ctas_per_sm; /* cap on resident CTAs per SM; 0 = occupancy limit */
    int32_t flags;       /* 0 or MCTP_BATCH_COUNT_EVALUATED */
} mctp_batch_tuning;

/* count the evaluated samples into bytes 8..15 of the workspace (a register
 * more in the march, so a little slower); without it those bytes are 0 */
#define MCTP_BATCH_COUNT_EVALUATED 1

int mctp_render_batch_workspace(const mctp_slicemap *sms, int32_t nsm, const mctp_view *views,
                                const int32_t *view_slicemap, const int32_t *view_lut, int32_t nviews,
                                int32_t nluts, size_t *bytes);

int mctp_render_batch(const mctp_slicemap *sms, int32_t nsm, const mctp_view *views,
                      const int32_t *view_slicemap, const int32_t *view_lut, int32_t nviews,
                      const float *luts_rgba, int32_t nluts, int32_t nlut, float alpha_stop,
                      const mctp_batch_tuning *tuning, float *out_rgba, uint64_t *samples_taken,
                      void *workspace, size_t workspace_bytes, void *stream);

/*
 * mctp_render_batch without a workspace argument, for callers that cannot
 * give the library device memory (a C host program with no device allocator,
 * a serving loop that must not allocate once running).  The paper has no
 * counterpart; this is a calling convention of this library.  The scratch is
 * one fixed array of MCTP_BATCH_STATIC_SCRATCH bytes in the library's device
 * memory per device, so this call allocates nothing.
 *   Arguments, results and errors are those of mctp_render_batch; a batch
 *   whose workspace (mctp_render_batch_workspace) exceeds
 *   MCTP_BATCH_STATIC_SCRATCH bytes is rejected with MCTP_ESIZE before
 *   anything is enqueued.
 *   The first call with a device current looks up the scratch address on
 *   that device; make that first call before any stream capture.  The lookup
 *   allocates nothing itself, but CUDA loads a library's device code lazily:
 *   if no kernel of this library has run on the device yet, the lookup loads
 *   it, and loading places the code and the scratch array in device memory
 *   (as the first launch of any kernel would).  The address is kept for the
 *   life of the process; after cudaDeviceReset the library must be unloaded
 *   and loaded again before this call is used.
 *   Nothing in the scratch needs to start at zero: every call rewrites what
 *   it uses (the work counter is cleared by an in-stream memset).
 *   All calls on one device share the one scratch: two calls whose work can
 *   overlap on the device (different streams, or host threads without
 *   ordering) race and give wrong images.  Issue them on one stream, or order
 *   them with events.
 */
#define MCTP_BATCH_STATIC_SCRATCH (8u << 20)

int mctp_render_batch_static(const mctp_slicemap *sms, int32_t nsm, const mctp_view *views,
                             const int32_t *view_slicemap, const int32_t *view_lut, int32_t nviews,
                             const float *luts_rgba, int32_t nluts, int32_t nlut, float alpha_stop,
                             const mctp_batch_tuning *tuning, float *out_rgba, uint64_t *samples_taken,
                             void *stream);

/*
 * Serving (an extension of this library: the paper's server renders previews
 * on request and streams them to clients, Sec. III-C).  A server keeps the
 * given slicemaps, their atlas textures and the transfer functions (caller
 * memory and objects, kept alive until destroy) and renders requests as they
 * arrive:
 *   - requests are admitted in arrival order while their image fits in the
 *     free part of `arena` (caller device memory, 256-byte aligned; the
 *     server's per-stream counters and batch workspaces come first, the image
 *     heap after them): admission by memory;
 *   - MCTP_SERVE_BATCHED: a host thread packs admitted requests into batches
 *     of up to max_batch_views and launches each as one mctp_render_batch
 *     launch on a free stream (up to max_inflight streams); requests that
 *     arrive while batches are on the device join the next batch, which
 *     starts as soon as a stream is free (continuous batching); each
 *     stream's workspace has room for the depth bounds of views up to
 *     1024 x 1024 pixels, and a batch with larger views renders without them;
 *   - MCTP_SERVE_PER_VIEW: one mctp_render_views launch per request, in
 *     arrival order (the plain per-view baseline);
 *   - a request's image is bit-identical to rendering its view alone with
 *     mctp_render_views (same march).
 * Times are mctp_now() seconds (a monotonic host clock).  t_done is when the
 * server thread observed the completion of the request's launch.
 * Errors: create: MCTP_EINVAL (bad arguments), MCTP_EUNSUPPORTED (mixed
 * dtypes), MCTP_ESIZE (arena smaller than the server's fixed part),
 * MCTP_ECUDA; submit: MCTP_EINVAL (bad view or index), MCTP_ESIZE (image
 * larger than the whole image heap).  A launch failure is reported in the
 * request's result status.
 */
#define MCTP_SERVE_BATCHED 0
#define MCTP_SERVE_PER_VIEW 1

typedef struct mctp_server mctp_server; /* opaque */

typedef struct {
    int32_t mode;             /* MCTP_SERVE_BATCHED or MCTP_SERVE_PER_VIEW */
    int32_t max_batch_views;  /* BATCHED: views per launch, 1..4096 */
    int32_t max_inflight;     /* launches on the device at once (streams), 1..8 */
    int32_t reserved;         /* must be 0 */
    mctp_batch_tuning tuning; /* BATCHED: launch shape (zeros = defaults) */
} mctp_serve_params;

typedef struct {
    uint64_t ticket;
    int32_t status;           /* MCTP_OK, or the error of the request's launch */
    int32_t reserved;
    float *image;             /* device [height][width][4], valid until release */
    double t_submit, t_admit, t_launch, t_done;
} mctp_serve_result;

int mctp_server_create(const mctp_slicemap *sms, int32_t nsm, const float *luts_rgba, int32_t nluts,
                       int32_t nlut, float alpha_stop, void *arena, size_t arena_bytes,
                       const mctp_serve_params *params, mctp_server **server);
/* Queue one request; thread-safe. */
int mctp_server_submit(mctp_server *server, const mctp_view *view, int32_t slicemap, int32_t lut,
                       uint64_t *ticket);
/* Move up to max_results finished requests (in completion order) to results. */
int mctp_server_poll(mctp_server *server, mctp_serve_result *results, int32_t max_results, int32_t *count);
/* Return a finished request's image memory to the arena. */
int mctp_server_release(mctp_server *server, uint64_t ticket);
/* Cancel a request that has not been launched yet: it leaves the queue (and
 * returns its image memory when it was admitted) and is reported by poll with
 * status MCTP_ECANCELED, after which it is released like any other.  A request
 * already launched, finished or unknown is not cancelled (MCTP_EINVAL). */
int mctp_server_cancel(mctp_server *server, uint64_t ticket);
/* Host-side fault injection for tests: the next `n` launches of the server
 * fail as a failed kernel launch would (nothing is enqueued; their requests
 * finish with status MCTP_ECUDA), after which the server carries on.  No GPU
 * fault is made. */
int mctp_server_inject_launch_failures(mctp_server *server, int32_t n);
/* Samples marched, launches made and the image heap's high-water mark (bytes). */
int mctp_server_stats(mctp_server *server, uint64_t *samples, uint64_t *launches, uint64_t *arena_high_water);
/* Wait for launches in flight, drop requests not yet launched, free the server. */
int mctp_server_destroy(mctp_server *server);
/* Monotonic host clock, seconds. */
double mctp_now(void);

/*
 * Differentiable rendering of a reduced volume (the previews stand a reduced
 * volume in for the full one, Sec. I / Sec. III; fitting it so that its
 * renders match renders of the source is an extension of this library).
 *   vol       device float [mz][my][mx] intensities; the value at a sample is
 *             v = min(max(trilinear(vol), 0), 1), looked up in lut_rgba as in
 *             mctp_render_views (x = v (nlut - 1), linear between entries)
 *   src_dims  host int64[3]: the world box [0,nx]x[0,ny]x[0,nz] the volume
 *             spans (views and sample spacing as in mctp_render_views, with
 *             the volume as the only level: every view's level must be 0)
 *   out_rgba  device float, 16-byte aligned, images one after another
 *   samples_taken device uint64[1] or NULL: overwritten with the samples
 *             marched (up to and including each ray's early-exit sample)
 * No empty-space skipping (the transfer function is a variable here).
 * Errors: MCTP_EINVAL, MCTP_ESIZE (more than 2^31 voxels), MCTP_ECUDA.
 */
int mctp_render_dense(const float *vol, int32_t mx, int32_t my, int32_t mz, const int64_t *src_dims,
                      const mctp_view *views, int32_t nviews, const float *lut_rgba, int32_t nlut,
                      float alpha_stop, float *out_rgba, uint64_t *samples_taken, void *stream);

/*
 * Gradient of L with respect to vol and lut_rgba, given grad_rgba = dL/d(the
 * images of mctp_render_dense with the same arguments).  grad_vol (float,
 * like vol) and grad_lut (float [nlut][4]) are overwritten.  The stop index
 * of each ray's early exit is held fixed; where the intensity clamp is active
 * the volume gradient is 0.  The adjoint walks each ray back to front with
 * checkpoints every 64 samples (rays of up to 2048 samples: MCTP_ESIZE for
 * views whose sample spacing allows longer rays).  Results are accumulated
 * with float atomics, so the last bits vary between runs.
 */
int mctp_render_dense_backward(const float *vol, int32_t mx, int32_t my, int32_t mz, const int64_t *src_dims,
                               const mctp_view *views, int32_t nviews, const float *lut_rgba, int32_t nlut,
                               float alpha_stop, const float *grad_rgba, float *grad_vol, float *grad_lut,
                               void *stream);

/* loss (device float[1], overwritten) = scale * sum_i (x_i - target_i)^2;
 * grad (device, may be NULL) = 2 scale (x - target). */
int mctp_l2_loss(const float *x, const float *target, int64_t n, float scale, float *grad, float *loss,
                 void *stream);

/* One Adam step (Kingma & Ba) on n parameters with bias correction for step
 * number `step` (>= 1), then clamped to [lo, hi]; m and v are the moment
 * buffers (start them at zero). */
int mctp_adam_step(float *param, const float *grad, float *m, float *v, int64_t n, float lr, float beta1,
                   float beta2, float eps, int32_t step, float lo, float hi, void *stream);

/*
 * Information content of rendered views, for choosing the most informative
 * snapshot (Sec. III-C, Eq. 2): per view the Shannon entropy
 * H = -sum_i p_i log2 p_i of its 256-bin grey-level histogram, and the view
 * with the largest H.  Grey level of a pixel (the premultiplied render over
 * black): Rec. 709 luminance (0.2126 R + 0.7152 G) + 0.0722 B in FP32 with one
 * rounding per operation in this order, clamped to [0, 1] (NaN as 0),
 * quantised as floor(lum * 255 + 0.5).
 *   rgba     device float, 16-byte aligned, views one after another (the
 *            layout of mctp_render_views' output)
 *   views    host array (only width and height are used), nviews <= 65535
 *   hist     device uint64[nviews][256], overwritten
 *   entropy  device double[nviews], overwritten (bits)
 *   best     device int32[1] or NULL: index of the largest H (lowest index
 *            on ties; -1 for no views)
 */
int mctp_image_entropy(const float *rgba, const mctp_view *views, int32_t nviews, uint64_t *hist,
                       double *entropy, int32_t *best, void *stream);

/*
 * Container removal (Sec. III, Container Removal): find the sample
 * container's circle on slice z (the top slice), then zero every voxel
 * outside it in every slice.  The circle is found by a Hough circle transform
 * in the manner the paper cites (centre by votes along gradient lines, radius
 * by a histogram of edge distances), refined by least-squares circle fits:
 *   1. [1 4 6 4 1]^2 smoothing (borders clamped), integer Sobel gradient;
 *      edge pixels have |g|^2 >= (256 thr)^2 (thr in grey units);
 *   2. each edge pixel votes, against its gradient, at distances rmin..rmax
 *      into cells of cell x cell pixels (acc, ceil(ny/cell) x ceil(nx/cell));
 *      the fullest cell (first in row-major order on ties) is the centre;
 *   3. histogram (rhist, rmax + 1 bins) of the rounded distances of the edge
 *      pixels whose gradient points away from the centre; its mode (smallest
 *      on ties) is the radius;
 *   4. three least-squares circle fits over those pixels within 2 cell + 3,
 *      cell + 3 and 3 pixels of the current circle.
 * The inner wall of a bright container around darker air is found.
 *   acc, rhist  device uint32 outputs (vote counts)
 *   workspace   device, mctp_container_workspace(nx, ny) bytes, 256-byte aligned
 *   circle      device int32[3]: centre x, y (rounded) and radius (floor); radius
 *               -1 when no edge pixel votes for a circle in [rmin, rmax]
 *   fit         device double[3] or NULL: the unrounded circle
 * Errors: MCTP_EINVAL (bad arguments, nx or ny < 3), MCTP_ESIZE (workspace).
 */
size_t mctp_container_workspace(int64_t nx, int64_t ny);
int mctp_find_container(const void *vol, const mctp_volume_desc *d, int64_t z, int64_t thr, int32_t rmin,
                        int32_t rmax, int32_t cell, uint32_t *acc, uint32_t *rhist, void *workspace,
                        size_t workspace_bytes, int32_t *circle, double *fit, void *stream);

/* out = in with every voxel (x, y, z) where (x - cx)^2 + (y - cy)^2 >
 * max(r - margin, 0)^2 set to 0, (cx, cy, r) = circle (device int32[3], e.g.
 * from mctp_find_container); r < 0 keeps everything.  out may equal in. */
int mctp_mask_container(const void *in, const mctp_volume_desc *d, const int32_t *circle, int32_t margin,
                        void *out, void *stream);

/* Default atlas grid for mz slices: tiles_x = 2^ceil(log2 sqrt(mz)),
 * tiles_y = ceil(mz / tiles_x).  Returns MCTP_EINVAL for mz < 1. */
int mctp_default_tiles(int32_t mz, int32_t *tiles_x, int32_t *tiles_y);

/* Bytes of one atlas: tiles_x*mx * tiles_y*my * element size (0 on bad input). */
size_t mctp_atlas_bytes(int32_t mx, int32_t my, int32_t tiles_x, int32_t tiles_y, int32_t dtype);

/* Bytes of one level's maxgrid: ceil(mx/8)*ceil(my/8)*ceil(mz/8)*2 (0 on bad input). */
size_t mctp_maxgrid_bytes(int32_t mx, int32_t my, int32_t mz);

/* Static string for a status code. */
const char *mctp_status_string(int code);

/*
 * Checked build.  The build can make a second library, compiled with
 * MCTP_CHECKED, in which the histogram, filter, slicemap and render kernels
 * test their main indices (histogram bins, keep-table entries, atlas elements
 * written and read, transfer-function entries, slice offsets, bitmap words,
 * image pixels) against the extent of the buffer they address.  An index
 * outside sets a bit in a device status word and the access is skipped;
 * nothing traps.  The tests run the parity cases against it and expect no bit.
 *   mctp_checked_build    1 in the checked library, 0 in the normal one
 *   mctp_checked_status   waits for the device, ORs the status words into
 *                         *bits (1 histogram bin, 4 atlas write, 8 atlas read,
 *                         16 table read, 32 image pixel, 64 keep-table entry,
 *                         2^31 self-test) and clears them when reset != 0;
 *                         MCTP_EUNSUPPORTED in the normal library
 *   mctp_checked_selftest enqueues one check of an index outside its extent
 *                         (it sets the self-test bit and accesses nothing)
 * The paper has no counterpart; this is test infrastructure of the library.
 */
int mctp_checked_build(void);
int mctp_checked_status(uint32_t *bits, int32_t reset);
int mctp_checked_selftest(void *stream);

/* MCTP_ABI_VERSION of the loaded library. */
int mctp_version(void);

#ifdef __cplusplus
}
#endif

#endif
