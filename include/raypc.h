/*
 * raypc.h -- C ABI of the GB300 (sm_103a) library for brushed multivariate
 * direct volume rendering with linked parallel-coordinates histograms
 * (Fritsch et al., "RayPC: Interactive Ray Tracing Meets Parallel
 * Coordinates", arXiv 2207.12011).
 *
 * The method (Section 2, "Approach"; Section 2.2, "Rendering"): rays are
 * marched front to back through a multi-variable volume; at every sample all
 * variables restricted in the parallel-coordinates plot are queried, and the
 * sample is discarded when any of them lies outside its bounds (brushing
 * and linking). Kept samples are coloured by a 1D transfer function and
 * composited. The restrictions do not modify the data, so no acceleration
 * structure is rebuilt when they change: per-brick min/max are built once
 * and a brush edit only re-classifies bricks. The parallel-coordinates plot
 * (Section 2.1, Fig. 2) is fed by adjacent-axis density histograms of the
 * selected cells.
 *
 * Conventions used by every entry point:
 *   - A volume is a cubic grid of n^3 cells with nvars (1..8) variables,
 *     cell-centred over the world cube [-1,1]^3: value index i sits at
 *     p = -1 + (i + 1/2) * 2/n. The spherical shell r_in <= |p| <= r_out is
 *     the domain; everything outside it is empty.
 *   - Caller buffers are plain pointers. "_dev" buffers are device memory of
 *     the context's GPU; other pointers are host memory. The library copies
 *     what it keeps (volume data, brush, transfer function); it never keeps
 *     a pointer to a caller buffer after the call returns.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *     enqueued asynchronously on it; errors found by the device surface at
 *     the caller's next synchronisation. Host arguments are consumed before
 *     the call returns.
 *   - Every function returns RAYPC_OK (0) or an error code and never aborts
 *     the process. raypc_last_error() gives a message for the calling thread.
 *   - A context is bound to one device. Calls on one context are serialised
 *     by an internal lock; the library sets and restores the current device.
 */
#ifndef RAYPC_H
#define RAYPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int raypc_status;
#define RAYPC_OK 0
#define RAYPC_ERR_INVALID_ARG 1   /* bad pointer, size, id or value            */
#define RAYPC_ERR_OOM 2           /* device allocation failed or over budget   */
#define RAYPC_ERR_CUDA 3          /* a CUDA runtime call failed                */
#define RAYPC_ERR_TIMEOUT 4       /* a bounded wait gave up                    */
#define RAYPC_ERR_BUSY 5          /* resource in use                           */
#define RAYPC_ERR_NOT_FOUND 6     /* unknown volume / level / request          */
#define RAYPC_ERR_UNSUPPORTED 7   /* valid but not implemented (e.g. non-cubic) */

/* Element types of volume data. */
#define RAYPC_F32 0
#define RAYPC_F16 1               /* IEEE binary16; FP32 -> FP16 rounds to nearest even */

#define RAYPC_MAX_VARS 8
#define RAYPC_BRICK 8             /* brick edge in cells                       */
#define RAYPC_MAX_LOD 2           /* coarser levels beyond the full level 0    */
#define RAYPC_TF_ENTRIES 256

/* Indices into the optional device statistics array of raypc_render
 * (RAYPC_NSTATS unsigned 64-bit counters that the kernel ADDS to). */
#define RAYPC_STAT_MARCHED 0      /* lattice samples from entry to termination  */
#define RAYPC_STAT_EVALUATED 1    /* samples whose field values were fetched    */
#define RAYPC_STAT_KEPT 2         /* samples in shell and in brush (composited) */
#define RAYPC_STAT_SKIPPED 3      /* lattice samples jumped by brick skipping   */
#define RAYPC_STAT_RAYS 4         /* rays that hit the outer sphere             */
#define RAYPC_STAT_ERT 5          /* rays ended by early ray termination        */
#define RAYPC_NSTATS 8

/* Implicit position axes (Section 2.1 derives altitude from the position;
 * Section 3 cuts the volume by brushing Cartesian coordinates). Axis a of a
 * point p: RAYPC_POS_X/Y/Z the coordinate, RAYPC_POS_R the radius
 * sqrt_rn(fma(z, z, fma(y, y, x * x))) (altitude is r_out minus it), all in
 * FP32. A sample's point is its lattice position; a cell's is its centre,
 * coordinate RN((2i + 1 - n) / n). In PC axis lists (raypc_pc_histogram,
 * raypc_pc_subsample) RAYPC_AXIS_POS(a) names position axis a; ids
 * 0..nvars-1 name stored variables. */
#define RAYPC_POS_X 0
#define RAYPC_POS_Y 1
#define RAYPC_POS_Z 2
#define RAYPC_POS_R 3
#define RAYPC_NPOS 4
#define RAYPC_AXIS_POS(a) (8 + (a))

typedef struct raypc_ctx raypc_ctx;

/* Pinhole camera. The view direction is normalize(target - eye); right =
 * normalize(cross(view, up)); true up = cross(right, view). Pixel (x, y),
 * y = 0 at the top row, looks along view + sx*right + sy*trueup with
 * sx = ((2x+1)/w - 1) * tan_half_vfov * w/h and sy = (1 - (2y+1)/h) *
 * tan_half_vfov (pixel centres). tan_half_vfov = tan(vertical fov / 2). */
typedef struct raypc_camera {
    float eye[3];
    float target[3];
    float up[3];
    float tan_half_vfov;
} raypc_camera;

/* Launch choices of a render. Neither changes any pixel: they only change
 * speed. RAYPC_AUTO takes the choice raypc_autotune measured fastest for this
 * device, storage dtype and grid edge, or the default if none was measured. */
#define RAYPC_AUTO 0
#define RAYPC_SKIP_ON 1           /* brick-level empty-space skipping on (default) */
#define RAYPC_SKIP_OFF 2
#define RAYPC_VARIANT_8x4 1       /* warp tile 8x4 pixels, block tile 16x8 (default) */
#define RAYPC_VARIANT_16x2 2      /* warp tile 16x2, block tile 32x4 */
#define RAYPC_VARIANT_4x8 3       /* warp tile 4x8, block tile 8x16 */

/* Options of one render. Zero-initialised = defaults except `ert`, which the
 * caller sets explicitly. */
typedef struct raypc_render_opts {
    float step;          /* world distance between lattice samples; <= 0: half a
                            voxel of the rendered level, i.e. 1/n_level         */
    int ert;             /* nonzero: stop a ray once its opacity A >= 1 - 2^-12 */
    int skip;            /* RAYPC_AUTO, RAYPC_SKIP_ON or RAYPC_SKIP_OFF          */
    int variant;         /* RAYPC_AUTO or RAYPC_VARIANT_*                         */
    float bg[4];         /* premultiplied background RGBA composited under     */
    uint32_t *counts_dev;/* optional [h][w][2] uint32: per pixel, lattice
                            samples marched and samples kept (debug/testing)    */
    int tf_skip;         /* nonzero: TF-aware skipping (single frames and
                            batched views; served requests too). A sample whose two
                            transfer-function entries both have sigma = 0 adds
                            exactly nothing; a 4^3 sub-brick is skipped when its
                            colour values v in [min - d, max + d] (brush margin
                            d; never when max(|min|,|max|) > 2^126) reach only
                            entries J(v) .. J(v)+1 with sigma = 0 and entry 0
                            (where a NaN colour lands) has sigma = 0 too, with
                            J(v) = min(floor(clamp((v - v_lo) * (255 / (v_hi -
                            v_lo)), 0, 255)), 254) in FP32. The image is
                            unchanged bit for bit; samples in skipped
                            sub-bricks are not counted as kept.                 */
    float *depth_dev;    /* optional [h][w] float32: per pixel the ray parameter
                            t (world distance from the eye) of the first kept
                            sample, t0 + (k + j) * step in FP32 exactly as the
                            march computes it; +inf where no sample is kept.
                            The depth that raypc_warp_image reprojects.
                            raypc_render, raypc_render_progressive and
                            batched views (a batch with any depth output
                            runs 8x4 tiles); served requests reject it.         */
} raypc_render_opts;

/* ---------------------------------------------------------------------- */
/* Errors and contexts                                                    */
/* ---------------------------------------------------------------------- */

/* Message of the last failing call on this thread ("" if none). The string
 * is owned by the library and valid until the thread's next call. */
const char *raypc_last_error(void);

/* Create a context on CUDA device `device`. hbm_budget_bytes caps the device
 * memory the context may hold for volumes, levels and bricks (0 = no cap);
 * a load that would exceed it fails with RAYPC_ERR_OOM and changes nothing. */
raypc_status raypc_create(raypc_ctx **out, int device, size_t hbm_budget_bytes);

/* Free every volume and the context. NULL is accepted. */
raypc_status raypc_destroy(raypc_ctx *ctx);

/* Bytes of device memory the context currently holds. */
raypc_status raypc_memory_used(raypc_ctx *ctx, size_t *out_bytes);

/* ---------------------------------------------------------------------- */
/* Volumes (Section 2.1: data preprocessing)                              */
/* ---------------------------------------------------------------------- */

/* Copy a volume into the library. `src` holds nvars planes of nz*ny*nx values
 * of type src_dtype, x fastest: src[((v*nz + z)*ny + y)*nx + x]; it is device
 * memory if src_is_device, else host memory. The stored copy has element type
 * store_dtype (FP16 storage rounds to nearest even; FP16 -> FP32 is exact)
 * in the library's interleaved layout. Only cubic grids with
 * 2 <= nx == ny == nz <= 4096 are supported (RAYPC_ERR_UNSUPPORTED otherwise).
 * 0 <= r_in < r_out.
 * Writes the new volume id to *out_vol. Allocates; the stored copy lives
 * until raypc_free_volume or raypc_destroy. */
raypc_status raypc_load_volume(raypc_ctx *ctx, const void *src, int src_is_device,
                               int src_dtype, int store_dtype, int nx, int ny, int nz,
                               int nvars, float r_in, float r_out, void *stream,
                               int *out_vol);

raypc_status raypc_free_volume(raypc_ctx *ctx, int vol);

/* Re-ingest new values of the same shape into level 0 of an existing volume
 * (e.g. the next time step of the simulation, Section 2.1), with the source
 * layout and conversion of raypc_load_volume. A device source allocates
 * nothing and must stay valid until `stream` reaches the ingest. A host
 * source goes through two staging buffers of the source's size that the
 * volume keeps and uses in turn (allocated by the first host update, charged
 * to the HBM budget, freed with the volume; if the budget has no room, a
 * stream-ordered temporary is used instead). The host-to-device copy runs on
 * a copy stream of the volume's own that waits only until the ingest two
 * updates back has read its buffer, so the copies of consecutive time steps
 * run back to back and overlap the work still running on `stream` (from a
 * pinned source); `stream` waits for the copy before the ingest. A pageable host source is consumed before the call
 * returns; a pinned host source must stay unchanged until the work this call
 * enqueues on `stream` has completed. Coarser levels, bricks and the
 * classification become stale: raypc_build_bricks must run again before
 * raypc_render (RAYPC_ERR_INVALID_ARG until then). */
raypc_status raypc_update_volume(raypc_ctx *ctx, int vol, const void *src, int src_is_device,
                                 int src_dtype, void *stream);

/* Level of detail (Section 2.1: an octree-like pyramid with coarser levels of
 * 1/8 of the cells each) and brick min/max (Section 2.2: acceleration data
 * that a brush change does not rebuild). Builds n_lod (0..RAYPC_MAX_LOD)
 * coarser levels -- coarse cell = FP32 mean of its 2x2x2 fine cells, fine
 * indices clamped at the edge, summed as ((c000+c100)+(c010+c110)) +
 * ((c001+c101)+(c011+c111)) then times 1/8, stored in the volume's dtype --
 * and, for every level, per 8^3 brick and variable, the min and max of the
 * stored values at the brick's vertices 8b..min(8b+8, n-1) (NaN ignored),
 * and the same for the 4^3 sub-bricks (vertices 4s..min(4s+4, n-1)) whose
 * activity the render tests per sample. brick_dim must be RAYPC_BRICK.
 * Calling it again rebuilds. */
raypc_status raypc_build_bricks(raypc_ctx *ctx, int vol, int brick_dim, int n_lod,
                                void *stream);

/* Set the brush box (Section 2: "upper and lower bounds for each variable";
 * Section 2.2: a sample whose restricted values violate them is discarded).
 * lo, hi: host arrays of nvars floats; variable v is restricted iff bit v of
 * active_mask is set; a sample or cell passes iff lo[v] <= value <= hi[v]
 * for every restricted v (inclusive; NaN values fail; lo > hi is a legal
 * empty brush; infinite bounds are open sides; NaN bounds are rejected).
 * Re-classifies the bricks of every built level on `stream`: a brick is
 * active iff its sample box (widened by 2^-10) meets the shell and, for every
 * restricted v, max_v + d >= lo[v] and min_v - d <= hi[v] with
 * d = max(|min_v|, |max_v|) * 2^-20 + 2^-120 (covers FP32 interpolation
 * rounding), except that a variable with max(|min_v|, |max_v|) > 2^126 never
 * deactivates a brick (its interpolation can overflow to an infinite value);
 * skippable iff it and its 26 neighbours are inactive. The 4^3
 * sub-bricks are classified by the same rule, and the cell classes of level 0
 * (see raypc_get_cell_classes) are computed too; those of coarser levels are
 * computed by their first render. Requires raypc_build_bricks. */
raypc_status raypc_set_brush(raypc_ctx *ctx, int vol, const float *lo, const float *hi,
                             uint32_t active_mask, void *stream);

/* Set the position brush of a volume: position axis a (RAYPC_POS_*) is
 * restricted iff bit a of pos_mask is set, to lo[a] <= value <= hi[a]
 * (inclusive; NaN bounds rejected; lo > hi is a legal empty range; lo, hi:
 * host arrays of RAYPC_NPOS floats, read only for restricted axes, may be
 * NULL when pos_mask is 0). A sample (render) or cell (histograms with
 * use_brush, subsample flags) must pass it as well as the variable brush of
 * raypc_set_brush, which leaves the position brush unchanged (and this call
 * leaves the variable brush unchanged; before any raypc_set_brush no
 * variable is restricted). Bricks and sub-bricks are re-classified as by
 * raypc_set_brush, with one more condition: the widened sample box meets
 * every restricted coordinate range, and for the radius sqrt_rn(far^2) >= lo
 * and sqrt_rn(near^2) <= hi (far/near: the box's farthest and nearest
 * corner distances, squared like a sample's), so no passing sample lies in an
 * inactive brick. pos_mask bits >= RAYPC_NPOS are rejected. */
raypc_status raypc_set_position_brush(raypc_ctx *ctx, int vol, const float *lo, const float *hi,
                                      uint32_t pos_mask, void *stream);

/* Set the 1D transfer function (Section 3 and Fig. 4: colour by one chosen
 * variable). rgbs: host array of 256 x (r, g, b, sigma); sigma is the
 * extinction per world unit. The colour variable's value v maps to the
 * position s = clamp((v - v_lo) / (v_hi - v_lo) * 255, 0, 255) and the entry
 * is interpolated linearly between floor(s) and floor(s)+1. v_lo < v_hi. */
raypc_status raypc_set_tf(raypc_ctx *ctx, int vol, const float *rgbs, int color_var,
                          float v_lo, float v_hi, void *stream);

/* ---------------------------------------------------------------------- */
/* Rendering (Section 2.2)                                                 */
/* ---------------------------------------------------------------------- */

/* Render level `lod` of a volume into out_rgba_dev ([h][w][4] float32,
 * premultiplied RGBA, 16-byte aligned, caller-owned). Per pixel the ray enters
 * the sphere r_out at t0 (or starts at the eye when inside) and leaves at t1;
 * lattice samples sit at t_k = t0 + (k + 1/2) * step for t_k < t1. A sample is
 * kept iff r_in^2 <= |p|^2 <= r_out^2, p passes the position brush
 * (raypc_set_position_brush) and every restricted variable's FP32
 * trilinear value (clamped cell-centred interpolation, lerps along x, then y,
 * then z, each as fma(f, b - a, a)) lies in the brush. Kept samples take
 * (r, g, b, sigma) from the transfer function, alpha = 1 - exp(-sigma * step),
 * and composite front to back: C += (1 - A) alpha rgb, A += (1 - A) alpha.
 * The integer decisions use correctly rounded FP32 operations in one fixed
 * order, so they do not depend on skipping, tiling or launch shape. Samples
 * in inactive 4^3 sub-bricks are rejected before any interpolation; with
 * skipping on, a ray jumps over the rest of an inactive sub-brick (or of an
 * inactive 8^3 brick), and the jump never changes the image. Requires set_brush
 * and set_tf.
 * stats_dev: optional RAYPC_NSTATS uint64 device counters the kernel adds to.
 * opts may be NULL only if the defaults with ert = 1 are wanted. */
raypc_status raypc_render(raypc_ctx *ctx, int vol, int lod, const raypc_camera *cam,
                          int w, int h, const raypc_render_opts *opts,
                          float *out_rgba_dev, unsigned long long *stats_dev, void *stream);

/* One progressive pass (Section 2: while the view rests, further passes
 * refine the image). Pass `pass` of a sequence renders exactly like
 * raypc_render except for the lattice: t_k = t0 + (k + j) * step with one
 * offset j in [0, 1) per pixel and pass. Pass 0 takes j = 1/2 (the
 * raypc_render image, bit for bit); pass p >= 1 takes the top 24 bits of
 * SplitMix64's output function (Steele, Lea and Flood 2014) evaluated at the
 * state key + (pix + 1) * 0x9E3779B97F4A7C15 (mod 2^64), key = seed * 2^32 + p,
 * pix = y * w + x, times 2^-24. Over the passes each sample position is
 * uniform in its step, so the running mean converges to the image of the
 * continuous ray integral without the fixed lattice's aliasing.
 * out_rgba_dev receives this pass's image. accum_rgba_dev (optional, [h][w][4]
 * float32, 16-byte aligned, caller-owned, not aliasing out_rgba_dev) holds the
 * running mean M of passes 0..pass and is updated in place:
 * pass 0 writes M = image; pass p >= 1 writes M = fma(1/(p+1), image - M, M)
 * per channel (1/(p+1) rounded to FP32), so the caller renders passes
 * 0, 1, 2, ... in order on one stream. pass = 2^32 - 1 is rejected
 * (RAYPC_ERR_INVALID_ARG), as is any argument raypc_render rejects. */
raypc_status raypc_render_progressive(raypc_ctx *ctx, int vol, int lod, const raypc_camera *cam,
                                      int w, int h, const raypc_render_opts *opts,
                                      uint32_t seed, uint32_t pass, float *accum_rgba_dev,
                                      float *out_rgba_dev, unsigned long long *stats_dev,
                                      void *stream);

/* Image warping (Section 2.2: while a frame is being rendered, the last image
 * is warped to the current view to fill the missing frames). Forward
 * reprojection of a w x h image rendered with camera `from` (its premultiplied
 * RGBA src_rgba_dev [h][w][4] float32 and depth src_depth_dev [h][w] float32,
 * e.g. the render's depth_dev output) to camera `to`, same size. Source pixel
 * s = y*w + x with a finite depth D becomes P = eye + D * d (d its ray
 * direction as in raypc_render); with the new camera's basis F', R', U'
 * (raypc_camera meaning) and v = P - eye': z = v.F', X = v.R', Y = v.U' as
 * FP32 fma dot products; z <= 0 drops the point; qx = X / (z * tan' * w/h),
 * qy = Y / (z * tan'); it lands in column floor((qx + 1) * w/2) and row
 * floor((1 - qy) * h/2) if inside the image. Every target pixel takes the
 * colour of the landed source of smallest z (ties: smallest s); target pixels
 * that no source reaches take bg (host array of 4 floats, NULL = 0) -- or,
 * with fill_holes nonzero, the source chosen for the reached neighbour (of
 * their 8) whose source has the smallest z (ties: smallest s), in one pass
 * over the forward result (bg if no neighbour was reached).
 * out_src_dev (optional, [h][w] int32) receives the chosen s or -1. All
 * decisions use correctly rounded FP32 operations in one fixed order.
 * Buffers are caller-owned device memory; out_rgba_dev must not alias
 * src_rgba_dev; RGBA buffers 16-byte aligned. */
raypc_status raypc_warp_image(raypc_ctx *ctx, const raypc_camera *from, const raypc_camera *to, int w, int h,
                              const float *src_rgba_dev, const float *src_depth_dev, const float *bg,
                              int fill_holes, float *out_rgba_dev, int32_t *out_src_dev, void *stream);

/* ---------------------------------------------------------------------- */
/* Batched rendering (many views and brushes in one launch)                */
/* ---------------------------------------------------------------------- */

/* One view of a batch: a volume level, a camera and image, its own brush box
 * (same meaning as raypc_set_brush, applied to this view only; the volume's
 * own brush is not used or changed), render options and caller-owned outputs
 * (out_rgba_dev [h][w][4] float32, 16-byte aligned; stats_dev optional). The
 * transfer function is the volume's (raypc_set_tf). */
typedef struct raypc_view {
    int vol;
    int lod;
    raypc_camera cam;
    int w, h;
    float lo[RAYPC_MAX_VARS];
    float hi[RAYPC_MAX_VARS];
    uint32_t active_mask;
    raypc_render_opts opts;
    float *out_rgba_dev;
    unsigned long long *stats_dev;
    float pos_lo[RAYPC_NPOS];    /* this view's position brush (raypc_set_position_brush meaning) */
    float pos_hi[RAYPC_NPOS];
    uint32_t pos_mask;
} raypc_view;

typedef struct raypc_batch raypc_batch;

/* A reusable batch of up to max_views views (1..4096). It owns a device view
 * table, per-view classification bitmasks and sub-brick lists, per-view cell
 * classes, a tile counter and a CUDA graph of the batched launch (table
 * upload, per-view brick and sub-brick classification, per-view cell classes,
 * the empty-space distance of every view that renders with skipping, one
 * persistent render kernel), captured on first use and replayed afterwards.
 * Allocates device and pinned host memory; the per-view buffers are allocated
 * for a view slot on its first use and grown for larger levels: n^3 * 2 bytes
 * of cell classes plus about n^3 / 10 bytes of masks, lists and distances per
 * used slot (281 MB at 512^3), charged to the context's budget. */
raypc_status raypc_batch_create(raypc_ctx *ctx, int max_views, raypc_batch **out);
raypc_status raypc_batch_destroy(raypc_batch *batch);

/* Render nviews views in one launch on `stream` (Section 2.2 per view, same
 * results bit for bit as raypc_render of each view with its brush set). Every
 * view's volume must have bricks built (not stale after an update), a transfer
 * function, and the same storage dtype. The tile variant of the launch is view
 * 0's (after RAYPC_AUTO resolution); skipping is chosen per view, and a view
 * with skipping jumps by the empty-space distance of its own classification,
 * as a single-frame render does. Work is split into 16x8-pixel tiles
 * pulled dynamically by persistent thread blocks, so large and small images
 * balance across the GPU. The call returns after enqueueing; it may wait for
 * the batch submitted two calls earlier on this batch object to finish (the
 * view table is double-buffered). Concurrent calls on one batch object must be
 * serialised by the caller. */
raypc_status raypc_render_batch(raypc_batch *batch, const raypc_view *views, int nviews, void *stream);

/* ---------------------------------------------------------------------- */
/* Serving (continuous batching of render and histogram requests)          */
/* ---------------------------------------------------------------------- */

/* The paper's client renders asynchronously and progressively: the frame
 * loop does not wait for the ray tracer, and passes are refined while the
 * camera rests (Section 2, Section 2.2). The server here is the GPU-side
 * counterpart for many clients: a request is a brushed render of a resident
 * volume (optionally a coarse-level pass first, delivered early, then the
 * full pass) or a brushed PC-histogram request. A server thread admits
 * queued requests while slots and the output-memory budget allow, packs the
 * admitted work into one batched render launch per loop turn and free stream
 * (a request's coarse and full passes go into the same launch; coarse passes
 * and small images first), so requests that arrive while others run join the
 * next launch and their work overlaps on the device. The persistent kernel
 * publishes each finished view through a record in mapped host memory, so a
 * request completes when its own passes are done, not when its whole launch
 * is. Per-request timestamps are recorded. A request's results are identical to rendering /
 * histogramming it alone. Besides the output pool, each stream's batch holds
 * per-view buffers (see raypc_batch_create) for the view slots its launches
 * have used, at most num_streams * max_batch_views slots, and each stream a
 * histogram scratch for the largest histogram it has run (the sub-brick bits
 * of a request's brush and, from 128^3 on, 16 partial copies of its counts:
 * 21 MB for 5 x 256^2 bins), all charged to the context's budget. */

#define RAYPC_REQ_RENDER 0
#define RAYPC_REQ_HISTOGRAM 1

typedef struct raypc_server raypc_server;

typedef struct raypc_server_config {
    int max_inflight;            /* admitted requests at once (1..4096)           */
    size_t output_budget_bytes;  /* device memory for request outputs; 0 = 1 GiB */
    int max_batch_views;         /* render passes per launch (1..4096)            */
    int num_streams;             /* launch streams (1..8)                         */
    long long max_batch_pixels;  /* pixels per launch (a single pass may exceed
                                    it); 0 = no cap                               */
} raypc_server_config;

typedef struct raypc_request {
    int kind;                    /* RAYPC_REQ_RENDER or RAYPC_REQ_HISTOGRAM       */
    int vol;                     /* resident volume (bricks built, TF set)         */
    float lo[RAYPC_MAX_VARS];    /* the request's brush (raypc_set_brush meaning)  */
    float hi[RAYPC_MAX_VARS];
    uint32_t active_mask;
    /* render */
    raypc_camera cam;
    int w, h;
    int lod;                     /* level of the full pass                         */
    int coarse_lod;              /* level of a first, early pass; -1 = none        */
    raypc_render_opts opts;      /* counts_dev is ignored                          */
    /* histogram (level lod) */
    int axis_order[RAYPC_MAX_VARS];
    int naxes, bins;
    const float *edges;          /* host, naxes x (bins + 1); copied on submit     */
    int use_brush;
    float pos_lo[RAYPC_NPOS];    /* the request's position brush                   */
    float pos_hi[RAYPC_NPOS];
    uint32_t pos_mask;
} raypc_request;

typedef struct raypc_result {
    int status;                  /* RAYPC_OK, or the error that ended the request  */
    int coarse_ready;            /* coarse image available                         */
    int done;                    /* all outputs available                          */
    double t_submit, t_admit, t_coarse, t_done;   /* seconds, steady host clock    */
    const float *coarse_dev;     /* [h][w][4], server-owned (NULL if none)         */
    const float *image_dev;      /* [h][w][4], server-owned                        */
    const uint32_t *hist_dev;    /* [naxes-1][bins][bins], server-owned            */
    unsigned long long samples;  /* lattice samples marched by the full pass       */
} raypc_result;

/* Start a server on ctx (which must outlive it). Allocates its streams and
 * batch objects and starts one host thread. */
raypc_status raypc_server_create(raypc_ctx *ctx, const raypc_server_config *cfg, raypc_server **out);

/* Stop the thread after the in-flight launches finish; pending requests end
 * with RAYPC_ERR_BUSY; all outputs are freed. */
raypc_status raypc_server_destroy(raypc_server *srv);

/* Queue a request (validated now: volume, level, sizes, brush, edges). The
 * request struct and its edges may be reused as soon as the call returns. */
raypc_status raypc_serve_submit(raypc_server *srv, const raypc_request *req, uint64_t *out_id);

/* State of a request; waits up to timeout_us for it to finish (0 = do not
 * wait). Returns RAYPC_ERR_TIMEOUT if it is not done by then (the result
 * still holds the progress so far), RAYPC_ERR_NOT_FOUND for unknown ids. */
raypc_status raypc_serve_poll(raypc_server *srv, uint64_t id, int timeout_us, raypc_result *out);

/* Free a finished request's outputs (returns their memory to the budget). */
raypc_status raypc_serve_release(raypc_server *srv, uint64_t id);

/* ---------------------------------------------------------------------- */
/* Autotuning of the render launch                                         */
/* ---------------------------------------------------------------------- */

typedef struct raypc_tuning {
    int variant;         /* RAYPC_VARIANT_*            */
    int skip;            /* RAYPC_SKIP_ON / _OFF       */
    float ms;            /* measured time per round    */
} raypc_tuning;

/* Time every launch choice (3 tile variants x skipping on/off) on the given
 * views -- each view classified under its own brush, rendered one frame at a
 * time, `reps` rounds after one warm-up round -- and remember the fastest for
 * this device, the views' storage dtype and the grid edge of view 0's level.
 * Later renders and batches with RAYPC_AUTO use it. If the environment
 * variable RAYPC_TUNE_CACHE names a file, the table is read from it on first
 * use and rewritten after each tuning. The views' output buffers are
 * overwritten. Synchronises `stream`. all_out (optional) receives the 6
 * measurements in the order variant 1..3, each with skipping on then off. */
raypc_status raypc_autotune(raypc_ctx *ctx, const raypc_view *views, int nviews, int reps,
                            raypc_tuning *best_out, raypc_tuning *all_out, void *stream);

/* The tuned choice for (device of ctx, dtype, grid edge n); RAYPC_ERR_NOT_FOUND if none. */
raypc_status raypc_get_tuning(raypc_ctx *ctx, int dtype, int n, raypc_tuning *out);

/* ---------------------------------------------------------------------- */
/* Parallel-coordinates histograms (Section 2.1 PC data; Fig. 2)            */
/* ---------------------------------------------------------------------- */

/* Density histograms of adjacent parallel-coordinates axes. axis_order: host
 * array of naxes (2..8) axis ids (stored variables, or RAYPC_AXIS_POS(a) for
 * the position axes at the cell centre); edges: host array of naxes rows of
 * bins+1 floats (non-decreasing, no NaN); bins in 2..1024. A cell counts iff
 * its centre is in the shell -- S_in <= sum_a (2 i_a + 1 - n)^2 <= S_out with
 * S_in = ceil((r_in n)^2), S_out = floor((r_out n)^2) in double -- and, when
 * use_brush is nonzero, its stored values pass the brush and its centre the
 * position brush. Its bin on axis a is
 * the number of interior edges e_1..e_{bins-1} of row a that are <= its value.
 * out_counts_dev ([naxes-1][bins][bins] uint32, caller-owned) is zeroed and
 * filled: H[p][bin_p][bin_{p+1}] counts cells. Counts are exact integers. */
raypc_status raypc_pc_histogram(raypc_ctx *ctx, int vol, int lod, const int *axis_order,
                                int naxes, int bins, const float *edges, int use_brush,
                                uint32_t *out_counts_dev, void *stream);

/* PC line data (Section 2.1: the plot draws the polylines of a random
 * subsample of at most 100 000 cells). Among the in-shell cells of level lod
 * (the histograms' integer test), N of them, takes the m = min(k, N) cells
 * with the smallest keys K(c): the output of SplitMix64's output function
 * (Steele, Lea and Flood 2014) at the state
 * (seed * 2^32 + 2^32 - 1) + (c + 1) * 0x9E3779B97F4A7C15 mod 2^64,
 * c = (z * n + y) * n + x. Keys are distinct (the output function is a
 * bijection), so the subsample is exactly defined; across seeds it is a
 * uniform random m-subset. Writes, in increasing c, out_cells_dev[i] = c
 * (int64, 8-byte aligned), out_values_dev[i * naxes + a] = the value of PC
 * axis axis_order[a] at the cell (float32; stored value, or position axis at
 * the centre) and out_in_brush_dev[i] = 1 iff the cell passes the volume's
 * brush (stored values and the position brush at the centre; 1 when no brush
 * was set), 0 otherwise. All three are caller-owned device arrays of at least
 * m entries (m x naxes values). *out_count (host) receives m when the call
 * returns, before the stream has run. k in 0..2^31-1; naxes 0..8 (axis_order
 * may be NULL when naxes is 0). Reads no field data for the selection:
 * an exact radix select over the keys, then an ordered compaction. */
raypc_status raypc_pc_subsample(raypc_ctx *ctx, int vol, int lod, uint32_t seed, long long k,
                                const int *axis_order, int naxes, long long *out_cells_dev,
                                float *out_values_dev, uint8_t *out_in_brush_dev,
                                long long *out_count, void *stream);

/* Brush test of given points, e.g. pathline seeds (Section 3: only the
 * pathlines whose seed lies in the current selection are shown).
 * points_dev: [npts][3] float32 world coordinates (x, y, z), device,
 * 4-byte aligned; out_pass_dev[i] (uint8, device) receives 1 iff point i
 * passes exactly the per-sample test of raypc_render on level lod: FP32
 * |p|^2 in the shell, the position brush, and every restricted variable's
 * FP32 trilinear value in the volume's brush (NaN coordinates fail). Before
 * any raypc_set_brush only the shell restricts. Caller-owned buffers;
 * npts >= 0. */
raypc_status raypc_filter_points(raypc_ctx *ctx, int vol, int lod, const float *points_dev,
                                 long long npts, uint8_t *out_pass_dev, void *stream);

/* Same histograms as raypc_pc_histogram, for callers that cannot let the
 * library allocate device memory: hosts whose GPU memory is reserved up front
 * by their own pool (where a cudaMalloc would fail or fragment it), real-time
 * loops that must not wait on the allocator, applications that own every byte
 * of the device. The paper has no counterpart; this is a deployment variant.
 * It needs no context and no resident volume: cells_dev is the caller's field
 * in the planar layout of raypc_load_volume (nvars planes of n^3 values, x
 * fastest, 2 <= n <= 4096), aligned to its element size, and dtype is its
 * element type; out_counts_dev is 4-byte aligned. Axis ids name stored
 * variables 0..nvars-1 only: position axes (RAYPC_AXIS_POS) and the position
 * brush are not accepted here. lo/hi/active_mask/use_brush, the shell
 * r_in/r_out and the remaining arguments mean what they mean above. It runs
 * on the calling thread's current device and calls no cudaMalloc, cudaFree or
 * other allocating routine: the bin edges go into a fixed 32.8 KB device
 * array (RAYPC_MAX_VARS x 1025 floats) compiled into the library, which every
 * GPU that loads the library holds until exit. Larger edge tables (naxes > 8
 * or bins > 1024) are rejected with RAYPC_ERR_INVALID_ARG. The first call in
 * each context of a device (the first call on the device, and the first after
 * a device reset or a switch to another context) looks up that array's device
 * address with cudaGetSymbolAddress, so make it before any stream capture.
 * All calls share the array and it keeps the last call's edges; every call
 * rewrites the part it reads and zeroes out_counts_dev itself. Calls whose
 * work overlaps on the GPU (different streams, no ordering) race on the array
 * and must be serialised by the caller. */
raypc_status raypc_pc_histogram_noalloc(const void *cells_dev, int dtype, int n, int nvars,
                                        float r_in, float r_out, const float *lo, const float *hi,
                                        uint32_t active_mask, int use_brush, const int *axis_order,
                                        int naxes, int bins, const float *edges,
                                        uint32_t *out_counts_dev, void *stream);

/* ---------------------------------------------------------------------- */
/* Inspection (testing and tools)                                          */
/* ---------------------------------------------------------------------- */

/* Number of CUDA kernels this library has launched in this process (all
 * contexts, all devices); lets callers verify that work ran on the GPU. */
raypc_status raypc_kernel_launches(unsigned long long *out);

/* Geometry of a level: cube edge n, variables, storage dtype and bricks per axis. */
raypc_status raypc_volume_info(raypc_ctx *ctx, int vol, int lod, int *out_n, int *out_nvars,
                               int *out_dtype, int *out_bricks_per_axis);

/* Copy a level back in the planar layout of raypc_load_volume and in the
 * storage dtype: out_dev holds nvars * n^3 elements. */
raypc_status raypc_export_volume(raypc_ctx *ctx, int vol, int lod, void *out_dev, void *stream);

/* Copy a level's brick min/max: two [nb][nb][nb][nvars] float32 device arrays
 * (brick (bx,by,bz) at index (bz*nb + by)*nb + bx). */
raypc_status raypc_get_bricks(raypc_ctx *ctx, int vol, int lod, float *out_min_dev,
                              float *out_max_dev, void *stream);

/* Copy a level's classification under the current brush. active_bits_dev and
 * skippable_bits_dev receive ceil(nb^3 / 32) uint32 words (bit b%32 of word
 * b/32 for brick b); active_list_dev (optional, nb^3 uint32) receives the ids
 * of the active bricks in increasing order and n_active_dev (optional, one
 * uint32) their number. */
raypc_status raypc_get_skip_list(raypc_ctx *ctx, int vol, int lod, uint32_t *active_bits_dev,
                                 uint32_t *skippable_bits_dev, uint32_t *active_list_dev,
                                 uint32_t *n_active_dev, void *stream);

/* Copy a level's 4^3 sub-brick data (nsb = ceil(n/4) per axis, sub-brick
 * (sx,sy,sz) at index (sz*nsb + sy)*nsb + sx): min/max as two
 * [nsb^3][nvars] float32 device arrays over the vertices 4s..min(4s+4, n-1),
 * and the activity bits under the current brush, ceil(nsb^3/32) uint32 words,
 * with the activity rule of the 8^3 bricks (Section 2.2 brush test with the
 * rounding margin). Any output may be NULL. */
raypc_status raypc_get_sub_bricks(raypc_ctx *ctx, int vol, int lod, float *out_min_dev,
                                  float *out_max_dev, uint32_t *active_bits_dev, void *stream);

/* Copy a level's cell classes under the current brush (computed if needed):
 * out_dev receives n^3 uint16 words, [z][y][x] for the interpolation cell
 * with lower corner (x,y,z). Over the cell's 8 corner values, a restricted
 * variable v FAILS if a corner is NaN or, with m = max(|min|,|max|) <= 2^126
 * and d = m * 2^-20 + 2^-120, max + d < lo[v] or min - d > hi[v]; it is
 * INSIDE if m <= 2^126, min - d >= lo[v] and max + d <= hi[v]; else it must
 * be interpolated. Bit v of a word is set iff v must be interpolated; bit 15
 * iff some restricted variable fails. Only the words of cells inside active
 * 4^3 sub-bricks (see raypc_get_sub_bricks) are computed -- the only cells a
 * render consults; the other words are unspecified. raypc_render uses them to
 * decide samples without interpolating (Section 2.2 brush test, same
 * decisions). */
raypc_status raypc_get_cell_classes(raypc_ctx *ctx, int vol, int lod, uint16_t *out_dev, void *stream);

/* Copy a level's empty-space distance of the 4^3 sub-bricks under the current
 * brush (computed if needed): out_dev receives nsb^3 uint8 values indexed like
 * raypc_get_sub_bricks, the Chebyshev distance in sub-bricks from each
 * sub-brick to the nearest active one, capped at 8 (0: active). Renders with
 * skipping jump over the samples that stay inside the box of sub-bricks within
 * distance - 1 (Section 2.2: the brush drives the empty-space skipping; the
 * image is unchanged). */
raypc_status raypc_get_skip_distance(raypc_ctx *ctx, int vol, int lod, uint8_t *out_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* RAYPC_H */
