/*
 * flamerec.h -- C ABI of the GB300 flame volume reconstruction library
 * (render / compare / adjust loop of Shen et al., "Radiative Transport Based
 * Flame Volume Reconstruction from Videos", arXiv 1809.06417).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Status: every call returns fr_status.  FR_OK is 0.  On failure nothing
 *    has been launched unless the status is FR_ECUDA, and fr_last_error(ctx)
 *    returns a message that stays valid until the next call on that context.
 *    No call aborts, throws across the ABI or traps on the device.
 *  - Memory: pointers marked "device" are borrowed device pointers owned by
 *    the caller; they must stay valid until the work queued on the context's
 *    stream has finished.  Pointers marked "host" are read (or written) before
 *    the call returns unless stated otherwise.  The library allocates only
 *    its own scratch, which it owns and frees in fr_destroy.
 *  - Ordering: all device work is queued on the context's stream, in call
 *    order.  Calls do not synchronise the host except where stated.
 *    fr_reconstruct runs the adjustments of an iteration's views on a second
 *    stream the context owns, ordered after the call's earlier work on the
 *    context's stream and before its later work (events), so to the caller
 *    the call behaves as if all of it were queued on the context's stream.
 *  - Geometry: the volume is a node-centred grid.  Node (i, j, k) is a key
 *    point (a voxel vertex, Sec. 3.3 definitions) at world position
 *    origin + h (i, j, k); records are stored x fastest: index
 *    (k ny + j) nx + i.  Ray arithmetic is done in voxel units (world / h):
 *    the sampling step, segment lengths, extinction (per voxel length) and
 *    the key-point distance D of Eq. 10 are all in voxel edge lengths.
 *  - Images: float32, views concatenated, rows top to bottom, 3 channels
 *    interleaved: element ((v H + y) W + x) 3 + c.
 */
#ifndef FLAMEREC_H
#define FLAMEREC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FR_ABI_VERSION 3
#define FR_MAX_VIEWS 32          /* cameras per problem */

typedef enum fr_status {
    FR_OK = 0,
    FR_EINVAL = 1,       /* bad argument; nothing launched */
    FR_ENOMEM = 2,       /* device or host allocation failed, or a job can never fit */
    FR_ECUDA = 3,        /* a CUDA call failed; see fr_last_error */
    FR_ETIMEDOUT = 4,    /* a bounded wait ran out */
    FR_EBUSY = 5,        /* resource in use (e.g. a job table slot) */
    FR_ECANCELED = 6,    /* the job was cancelled */
    FR_ERANGE = 7        /* a bounded record overflowed (what fits is still returned) */
} fr_status;

typedef enum fr_dtype { FR_F32 = 0, FR_BF16 = 1, FR_F16 = 2 } fr_dtype;

/* Record kinds.  FR_KIND_RGB: {S_r, S_g, S_b, sigma_t} per node, the
 * emitted radiance per voxel length of the RTE (Eq. 5, first term) and the
 * extinction coefficient (Eq. 5, second term).  FR_KIND_TEMP: {T, sigma_t},
 * temperature in kelvin mapped to RGB through the colour-temperature table
 * (Sec. 3.3.3). */
typedef enum fr_kind { FR_KIND_RGB = 0, FR_KIND_TEMP = 1 } fr_kind;

/* A volume: descriptor plus a borrowed device pointer to nx*ny*nz records of
 * `dtype` with 4 (RGB) or 2 (TEMP) components each.  Every extent >= 2. */
typedef struct fr_volume {
    int32_t nx, ny, nz;
    int32_t kind;        /* fr_kind */
    int32_t dtype;       /* fr_dtype (storage; all arithmetic is float32) */
    int32_t pad_;
    float origin[3];     /* world position of node (0,0,0) */
    float h;             /* node spacing (world units) */
    void *data;          /* device */
} fr_volume;

/* Perspective pinhole camera (world units).  right, up, fwd orthonormal.
 * Pixel (x, y), row 0 on top, casts the ray through its centre:
 *   d = normalise(fwd + a right + b up),
 *   a = (2 (x + 0.5) / width - 1) tan_half_fov width / height,
 *   b = (1 - 2 (y + 0.5) / height) tan_half_fov. */
typedef struct fr_camera {
    float pos[3], right[3], up[3], fwd[3];
    float tan_half_fov;  /* tangent of half the vertical field of view */
    int32_t width, height;
    int32_t pad_;
} fr_camera;

typedef enum fr_rule {
    FR_RULE_PAPER = 0,    /* Eqs. 10-11: dV_j += G alpha_l dL T exp(-alpha_d D) */
    FR_RULE_GRADIENT = 1  /* V -= grad_step * d(0.5 sum m dL^2)/dV (exact adjoint) */
} fr_rule;

/* Method parameters.  fr_params_default() fills the paper's constants. */
typedef struct fr_params {
    float step;          /* sampling step, voxel edge lengths (Sec. 4.2: 1) */
    float alpha_l;       /* Eq. 10 residual scale (Sec. 5.1: 0.001) */
    float alpha_d;       /* Eq. 10 distance scale (Sec. 5.1: 1) */
    float tau;           /* > 0: constant sample opacity, Eqs. 7-8, 12 (Sec. 5.1: 0.05);
                            <= 0: extinction from the sigma_t field (Eq. 6) */
    float g_std;         /* spread of G(s), mean 1 (Eq. 11); 0 disables */
    float flame_thresh;  /* flame-pixel threshold, image units (Sec. 4.1: 30/255) */
    uint64_t seed;       /* key of the G(s) stream */
    int32_t clamp_nonneg;/* clamp adjusted values at 0 */
    int32_t rule;        /* fr_rule used by fr_reconstruct */
    float grad_step;     /* FR_RULE_GRADIENT step size */
    int32_t update_sigma;/* FR_RULE_GRADIENT: also step sigma_t */
    float lut_t_min, lut_t_max; /* colour-temperature table range, kelvin */
    const float *lut;    /* device, lut_size x 4 {r,g,b,0}, from fr_planck_lut (TEMP only) */
    int32_t lut_size;
    int32_t use_hull;    /* fr_reconstruct: hold records outside the visual hull at 0 (Sec. 4.3.1) */
    int32_t skip_empty;  /* forward march of RGB records without tau: skip bricks (fr_brick_cells()^3 cells) whose
                            records are all zero (exact: the result is bitwise the same); with
                            use_hull, the paper-rule adjustment also skips bricks with no key point
                            inside the hull (exact up to the order of its atomic sums) */
    const uint32_t *hull_tags; /* use_hull: device, one tag per node from fr_visual_hull for the same
                            cameras and targets; NULL: fr_reconstruct computes them each call */
    float hg_g;          /* in-scattering phase: Henyey-Greenstein asymmetry in (-1, 1) (Eq. 9);
                            0: isotropic, as in the paper.  g != 0: each view renders its own
                            source, the six directional radiances weighted towards the direction
                            from the volume's centre to its camera */
    int32_t sequential_views; /* fr_reconstruct: 1 = update the volume after each view in turn
                            (Kaczmarz order; the source is recomputed before each view) */
    int32_t tables;      /* fr_reconstruct and the server's jobs, paper rule with the visual hull, skip_empty, field mode
                            (tau <= 0), g_std = 0, all views at once: the extinction stays fixed and
                            G(s) = 1, so rendering (Eqs. 5-8) and the adjustment (Eq. 10) are linear
                            maps whose weights do not change between iterations.  0: build them once
                            per call (two marches over every ray) and stream them each iteration when
                            the call runs at least FR_TABLES_MIN_ITERS iterations; 1: never (march
                            every iteration); 2: whenever they apply.  Where they do not apply, or
                            their device memory would pass the scratch limit, the marches run.  The
                            build synchronises the context's stream once (the host reads the tables'
                            sizes and orders the tiles; fr_reconstruct_batch once per problem).  The
                            results are those of the marches up to float32 rounding (summation order) */
} fr_params;

/* Iterations from which fr_reconstruct builds the ray weight tables when
 * fr_params.tables is 0.  The build costs about as much as the tables save
 * over 7-8 iterations (128^3 grid, 8 views of 512^2: 2.3 ms to build, 0.31 ms
 * saved per iteration), so a caller timing calls of 4-7 iterations sets
 * tables = 1. */
#define FR_TABLES_MIN_ITERS 4

typedef struct fr_ctx fr_ctx;

/* Library ABI version (FR_ABI_VERSION). */
int32_t fr_abi_version(void);

/* Fills `p` with the paper's constants (Sec. 4.1, 4.2, 5.1). */
void fr_params_default(fr_params *p);

/* Create a context on `device`.  stream: the cudaStream_t to queue work on
 * (borrowed); NULL means CUDA's default stream, as in the runtime API. */
fr_status fr_create(fr_ctx **out, int device, void *stream);
fr_status fr_destroy(fr_ctx *ctx);
/* Bounds checks.  A library built with -DFR_CHECKED (build.py --checked)
 * checks the indices its kernels compute before every access (record
 * gathers, update reductions, pixels, flame-ray list entries, bricks, nodes
 * of the volume passes); an index out of range sets a bit in a device check
 * word (1 gather, 2 reduction, 4 pixel, 8 list entry, 16 brick, 32 volume
 * node) and is replaced by 0, never trapping.  fr_checks_enabled() tells the
 * build; fr_check_word synchronises the context's stream and returns the
 * word (0 in the normal build), clearing it when reset != 0. */
int32_t fr_checks_enabled(void);
/* Edge of the bricks the marches skip, in cells (the skipping granularity). */
int32_t fr_brick_cells(void);
fr_status fr_check_word(fr_ctx *ctx, uint32_t *word, int reset);

/* Device scratch the context allocates on first use and keeps (residuals,
 * accumulators, tables): at most `bytes` in all (0: no limit).  A call that
 * would need more fails with FR_ENOMEM, launches nothing and leaves the
 * context usable; raising the limit lets the next call proceed.  Scratch
 * already held is kept. */
fr_status fr_set_scratch_limit(fr_ctx *ctx, size_t bytes);
/* Device scratch the context holds now, in bytes (host output). */
fr_status fr_scratch_bytes(const fr_ctx *ctx, size_t *held);

/* Replace the context's stream (borrowed; NULL = CUDA's default stream). */
fr_status fr_set_stream(fr_ctx *ctx, void *stream);
/* Message of the last failure on this context ("" if none). */
const char *fr_last_error(const fr_ctx *ctx);
/* Blocks until the context's queued work is done. */
fr_status fr_synchronize(fr_ctx *ctx);

/* Sec. 4.1 pre-processing of target frames, in place.  Pixels whose largest
 * channel exceeds `thresh` are flame pixels; all others are set to black.
 * bbox (device, ncam x 4 int32: x0, y0, x1, y1 inclusive) receives the tight
 * box of each view's flame pixels, with x0 > x1 for a view without any.
 * targets: device, ncam x height x width x 3. */
fr_status fr_prepare_targets(fr_ctx *ctx, int ncam, int height, int width,
                             float *targets, float thresh, int32_t *bbox);

/* Sec. 3.3.1 / Eqs. 5-8 (Algorithm 2, rendering half): ray-march every pixel
 * of every camera through `vol` front to back.  Field mode: a segment of
 * length l sampled (trilinearly, at its midpoint) at source S and extinction s
 * adds T S (1 - exp(-s l)) / s and multiplies T by exp(-s l); tau > 0 uses the
 * constant-opacity blend of Eqs. 7-8.  Background black.  All cameras must
 * share one image size.  out_rgb: device, ncam x H x W x 3. */
fr_status fr_render(fr_ctx *ctx, const fr_volume *vol, const fr_camera *cams,
                    int ncam, const fr_params *p, float *out_rgb);

/* Rendering fused with the colour constraint of Sec. 3.3.2 and the error
 * measure of Sec. 5.1.  targets (device) must have been through
 * fr_prepare_targets.  For every pixel dL = target - rendered;
 *   residual (device, like the image) = dL on flame pixels, 0 elsewhere;
 *   rendered (device, nullable) = the rendered image;
 *   sq_err (device, 4 floats, overwritten) = sum over the per-view boxes of
 *   dL^2 per channel, and the number of boxed pixels.
 * RMSE on the paper's [0, 255] scale is 255 sqrt(sq_err[c] / sq_err[3]). */
fr_status fr_render_residual(fr_ctx *ctx, const fr_volume *vol, const fr_camera *cams,
                             int ncam, const fr_params *p, const float *targets,
                             const int32_t *bbox, float *rendered, float *residual,
                             float *sq_err);

/* Eq. 10 (Algorithm 2, adjustment half): for every pixel with a non-zero
 * residual, every sample s on its ray and each of the sample's eight key
 * points j, accumulate
 *   dV[j] += G(s) alpha_l dL T(s, s_e) exp(-alpha_d D(j, s))
 * with T the transmittance in front of the sample (Eq. 12 when tau > 0) and
 * G(s) the Gaussian factor of Eq. 11 drawn from the counter-based stream
 * keyed by (seed, iteration, view, pixel, sample).  Accumulation order is
 * unspecified (float atomics).  vol supplies sigma_t only (RGB kind).
 * dV: device, nodes x 4 float32 {r, g, b, unused}, accumulated into. */
fr_status fr_adjust(fr_ctx *ctx, const fr_volume *vol, const fr_camera *cams, int ncam,
                    const fr_params *p, const float *residual, int iteration, float *dV);

/* Eq. 11: V <- V + scale dV on the colour components (and on sigma_t when
 * with_sigma, from dV's fourth component), optional clamp at 0, rounded to
 * the volume's storage type; dV is zeroed afterwards when zero_dV. */
fr_status fr_apply_update(fr_ctx *ctx, fr_volume *vol, float *dV, float scale,
                          int with_sigma, int clamp_nonneg, int zero_dV);

/* Exact gradient of the rendered images (the differentiable variant of the
 * adjustment): given grad_img = d(loss)/d(pixel) and the radiance L_total the
 * forward pass rendered, accumulate d(loss)/d(record) into grad (device,
 * nodes x 4 float32 for RGB {S_r,S_g,S_b,sigma}; nodes x 2 {T, sigma} for
 * TEMP).  Transmittance is recomputed along each ray, never stored. */
fr_status fr_render_backward(fr_ctx *ctx, const fr_volume *vol, const fr_camera *cams,
                             int ncam, const fr_params *p, const float *L_total,
                             const float *grad_img, float *grad);

/* In-scattering source (Eq. 5, third term, isotropic phase function Eq. 9
 * with g = 0).  J at each node is the mean over the six axis directions of the
 * emitted radiance arriving along grid lines (single scattering); the output
 * records are S = q + albedo sigma_t J with sigma_t copied.  emission: RGB
 * volume {q, sigma}; albedo: device, nodes float32; out: RGB volume of the
 * same grid (any storage type); J (device, nodes x 4 float32) is scratch
 * supplied by the caller. */
fr_status fr_scatter_source(fr_ctx *ctx, const fr_volume *emission, const float *albedo,
                            float *J, fr_volume *out);

/* Colour-temperature table (Sec. 3.3.3): Planck's law integrated against
 * three Gaussian channel responses (centres 600, 540, 460 nm, width 40 nm,
 * 380-780 nm, trapezoid rule in 1 nm steps), scaled so green(2000 K) = 1.
 * lut: device, m x 4 float32 {r, g, b, 0} at t_min + i (t_max - t_min)/(m-1). */
fr_status fr_planck_lut(fr_ctx *ctx, float t_min, float t_max, int m, float *lut);

/* Visual hull (Sec. 4.3.1, Algorithm 1).  Bit v of tags[node] is set when the
 * centre of a flame pixel of view v (prepared target above p->flame_thresh)
 * lies in the image rectangle bounding the projection of the box of the eight
 * cells that share the node ([i-1, i+1] x [j-1, j+1] x [k-1, k+1], clipped to
 * the volume): every ray that samples one of those cells passes through that
 * rectangle, so the tags are conservative.  The projection is evaluated in
 * float32 with one rounding per operation (an integer decision):
 *   o = (pos - origin) * (1/h);  x_c = ((X - o_x) r_x + (Y - o_y) r_y) + (Z - o_z) r_z,
 *   likewise y_c (up) and z_c (fwd);  u = ((x_c / z_c) / t_x + 1) (W/2) - 1/2,
 *   t_x = tan_half W / H;  v = (1 - (y_c / z_c) / tan_half) (H/2) - 1/2;
 *   pixels [ceil(u_min), floor(u_max)] x [ceil(v_min), floor(v_max)] clipped to
 *   the image, the whole image if a corner has z_c <= 0.
 * A node is inside the hull when all ncam bits are set.  vol: the grid (its
 * data is not read).  targets: device, prepared.  tags: device, nodes uint32. */
fr_status fr_visual_hull(fr_ctx *ctx, const fr_volume *vol, const fr_camera *cams, int ncam,
                         const float *targets, const fr_params *p, uint32_t *tags);

/* The reconstruction loop (Sec. 3, Algorithm 2 repeated): for `iters`
 * iterations: [in-scattering source when albedo != NULL] -> render and
 * residual -> adjust (p->rule) -> apply.  vol is updated in place.
 * targets_are_host != 0: targets is pinned host memory and is copied to the
 * device before the loop (the context keeps a device copy).  targets must be
 * prepared (fr_prepare_targets) and bbox (device) must be its box.
 * rmse (nullable): iters x 3 float32 on the paper's [0, 255] scale, of the
 * image rendered at the start of each iteration; rmse_is_host != 0 means a
 * host array filled before the call returns (the call then synchronises). */
fr_status fr_reconstruct(fr_ctx *ctx, fr_volume *vol, const float *albedo,
                         const fr_camera *cams, int ncam, const float *targets,
                         int targets_are_host, const int32_t *bbox, int iters,
                         int first_iteration, const fr_params *p, float *rmse,
                         int rmse_is_host);

/* The reconstruction loop with the stop criterion of Sec. 3: iterations as in
 * fr_reconstruct until the image error (the rmse rows below) changes by less
 * than stop_delta (>= 0, on the [0, 255] scale) in every channel between two
 * consecutive iterations, or max_iters (>= 1) iterations have run; the paper
 * stops at 0.01.  The iterations run as one CUDA graph whose conditional while
 * node the device ends, so the host does not wait on each iteration.  rmse
 * (nullable; host when rmse_is_host, else device): room for max_iters x 3,
 * the first *iters_done rows written.  *iters_done (host, required): the
 * iterations run; the call synchronises the context's stream.  Phase tracing
 * does not see inside the graph. */
fr_status fr_reconstruct_until(fr_ctx *ctx, fr_volume *vol, const float *albedo,
                               const fr_camera *cams, int ncam, const float *targets,
                               int targets_are_host, const int32_t *bbox, int max_iters,
                               float stop_delta, int first_iteration, const fr_params *p,
                               float *rmse, int rmse_is_host, int32_t *iters_done);

/* One reconstruction problem of a batch (e.g. one video frame, Sec. 5.2, whose
 * frames the paper reconstructs independently). */
typedef struct fr_problem {
    fr_volume vol;             /* RGB records, updated in place */
    const fr_camera *cams;     /* host, ncam cameras sharing one image size */
    int32_t ncam;
    int32_t pad_;
    const float *targets;      /* device, prepared by fr_prepare_targets */
    const int32_t *bbox;       /* device, ncam x 4 */
    float *rmse;               /* device, iters x 3, or NULL */
    const uint32_t *hull_tags; /* device, one tag per node, or NULL; with p->use_hull these tags
                                  (e.g. from fr_visual_hull, kept across calls) are used instead
                                  of computing the problem's hull from its targets */
} fr_problem;

/* fr_reconstruct with the paper rule over nprob independent problems at
 * once: each iteration runs one forward launch, one error reduction, one
 * adjustment launch over the flame rays of all problems and one update
 * launch, whatever nprob is.  Volumes share one storage type; grids, cameras
 * and image sizes may differ.  Parameters are shared.  p->use_hull: each
 * problem's visual hull is its hull_tags, or else computed from its own
 * targets (p->hull_tags is not read), and its records outside it are held at
 * 0; p->skip_empty: empty bricks are skipped as in fr_reconstruct.  use_graph != 0 captures the iterations in
 * a CUDA graph and launches it once; the call then returns after the work is
 * done.  Scratch is sized from all problems at once. */
fr_status fr_reconstruct_batch(fr_ctx *ctx, const fr_problem *probs, int nprob, int iters,
                               int first_iteration, const fr_params *p, int use_graph);

/* ---------------------------------------------------------------------------
 * Serving: a continuous-batching reconstruction server (no counterpart in the
 * paper, which reconstructs one frame at a time).  Jobs are admitted in
 * arrival order while their device footprint fits the server's memory budget;
 * every step advances all resident jobs by one iteration of the paper rule in
 * shared launches (their rays batched together); jobs join and leave at step
 * boundaries.  Volumes are held in the server's storage type with float32
 * arithmetic.  With use_hull, skip_empty, field mode and g_std = 0 (and
 * p->tables as for fr_reconstruct), a job builds its ray weight tables at
 * admission (its footprint then grows by their size, inside the budget; a job
 * with no room for them marches) and its iterations stream them in shared
 * launches.  Calls on one server must not run concurrently.
 * ------------------------------------------------------------------------- */
typedef struct fr_server fr_server;
typedef struct fr_job fr_job;

typedef enum fr_job_state {
    FR_JOB_QUEUED = 0, FR_JOB_RUNNING = 1, FR_JOB_DONE = 2, FR_JOB_CANCELED = 3
} fr_job_state;

/* A job.  Host buffers must stay valid until the job is done or cancelled. */
typedef struct fr_job_desc {
    int32_t nx, ny, nz;
    float alpha_l;              /* Eq. 10 residual scale of this job; 0 = the server's */
    float origin[3];
    float h;
    const fr_camera *cams;      /* host, ncam cameras sharing one image size (copied) */
    int32_t ncam;
    int32_t iters;              /* iterations to run */
    const void *init_records;   /* host, nodes x 4 records in the server's storage type:
                                   initial {S_r, S_g, S_b, sigma} */
    const float *targets;       /* host, ncam x H x W x 3 raw frames (prepared on admission) */
    void *result_records;       /* host, nodes x 4 records: written when the job completes */
    float *rmse;                /* host, iters x 3 per-iteration error, or NULL */
    const uint32_t *hull_tags;  /* host, one tag per node, or NULL; with the server's use_hull
                                   these tags are copied at admission instead of computing the
                                   job's hull from its frames */
} fr_job_desc;

typedef struct fr_job_info {
    int32_t state;              /* fr_job_state */
    int32_t iters_done;
    double t_submit, t_admit, t_done;  /* seconds on the server's clock (steady) */
    size_t footprint;           /* device bytes while resident */
} fr_job_info;

/* budget_bytes: device memory the server may hold for resident jobs; 0 means
 * 80% of the device's free memory at creation.  dtype: storage type of every
 * job's volume.  p: shared method parameters (paper rule); with p->use_hull
 * each job's visual hull is computed from its frames at admission, and
 * p->skip_empty skips empty bricks, as in fr_reconstruct_batch. */
fr_status fr_server_create(fr_ctx *ctx, const fr_params *p, int dtype, size_t budget_bytes,
                           fr_server **out);
fr_status fr_server_destroy(fr_server *srv);
/* Queue a job.  FR_ENOMEM if its footprint exceeds the whole budget. */
fr_status fr_server_submit(fr_server *srv, const fr_job_desc *desc, fr_job **out);
/* One step: retire finished jobs, admit queued jobs that fit, advance every
 * resident job by one iteration.  Blocks until the step's device work is done.
 * running (nullable): resident jobs after the step; queued: jobs waiting. */
fr_status fr_server_step(fr_server *srv, int *running, int *queued);
fr_status fr_job_get_info(const fr_job *job, fr_job_info *info);
/* Step the server until the job is done or timeout_ms passes (FR_ETIMEDOUT). */
fr_status fr_job_wait(fr_server *srv, fr_job *job, int timeout_ms);
/* Cancel a queued or running job (its memory is released at the next step). */
fr_status fr_job_cancel(fr_server *srv, fr_job *job);
/* Free a finished or cancelled job's handle (FR_EBUSY while it is queued or running). */
fr_status fr_job_release(fr_server *srv, fr_job *job);
/* Device bytes currently held for resident jobs. */
fr_status fr_server_memory(const fr_server *srv, size_t *used, size_t *budget);

/* Temperature from the green channel (Sec. 3.3.3): the paper reconstructs the
 * green channel and reads the temperature off the colour-temperature mapping.
 * Per node, T = the inverse of the table's piecewise-linear green column
 * (p->lut, lut_size x {r, g, b, 0} float32 from fr_planck_lut over
 * [p->lut_t_min, p->lut_t_max]; its green column must increase strictly, which
 * it does over 800-2000 K) at the record's green value, clamped to the range;
 * the record's extinction is copied.  rgb: RGB records; temp: temperature
 * records on the same grid (any storage types).  Asynchronous. */
fr_status fr_temperature_from_green(fr_ctx *ctx, const fr_volume *rgb, const fr_params *p, fr_volume *temp);

/* Volume data error (Sec. 5.1): per colour channel, the root mean square of
 * the difference between the emission of two RGB volumes on the same grid
 * (any storage types), over the key points whose tag equals full_mask (the
 * visual hull's key points when tags come from fr_visual_hull and full_mask =
 * 2^ncam - 1), or over all key points when tags is NULL; in the volumes' own
 * units.  tags: device, one per node, nullable.  rmse3 (host, 3 floats) and
 * *count (host, nullable: the key points compared) are written before the call
 * returns (it synchronises the stream); rmse3 is 0 when none is compared. */
fr_status fr_volume_rmse(fr_ctx *ctx, const fr_volume *a, const fr_volume *b, const uint32_t *tags,
                         uint32_t full_mask, float *rmse3, int64_t *count);

/* ---- Cameras and grids (host arithmetic, no context, no device) ---- */

/* A pinhole camera from a 3x4 projection P (row-major, double), pixel
 * coordinates [u, v, w] = P [X, Y, Z, 1] with pixel centres at integers, u to
 * the right and v down: P = K [R | -R C], K = [[f, s, c_u], [0, f_v, c_v],
 * [0, 0, 1]], found by an RQ decomposition of P's left 3x3 block.  The model of
 * fr_camera has square pixels, no skew and the principal point at the image
 * centre: FR_EINVAL unless |s| and |f - f_v| are below 1e-6 f and the principal
 * point is within 1e-3 pixel of ((width - 1) / 2, (height - 1) / 2).  Output:
 * pos = C, right = R row 0, up = -R row 1, fwd = R row 2,
 * tan_half_fov = height / (2 f_v). */
fr_status fr_camera_from_projection(const double P[12], int width, int height, fr_camera *out);

/* Volume dimensions (Sec. 4.2): for the world box [box_min, box_max] and the
 * cameras, each of the box's 12 edges is projected into every image; the
 * largest number of pixels an edge along axis d spans in u or v over all
 * images is n_d, and the voxel edge that rule asks for along d is
 * alpha l_d / n_d (l_d the box length, alpha = 1.5 in the paper).  The grid
 * here has cubic voxels, so h = the smallest of the three edges and
 * dims[d] = ceil(l_d / h) + 1 nodes, from origin box_min.  FR_EINVAL when a
 * box corner is not in front of a camera (z_c <= 0) or the box is empty.
 * n (nullable): the three n_d. */
fr_status fr_volume_dims(const fr_camera *cams, int ncam, const float box_min[3], const float box_max[3],
                         float alpha, int32_t dims[3], float *h, float n[3]);

/* ---- Volumes held by the library ---- */

/* A volume whose records the library allocates on the context's device:
 * nx x ny x nz key points (Sec. 3.3: the voxel vertices) of `kind` stored as
 * `dtype`, kept in GPU memory across calls as the paper keeps its volume
 * (Sec. 4.3.2).  *out receives the descriptor every other entry point takes;
 * its data (device, 256-byte aligned) is owned by the library, zeroed, and
 * freed by fr_volume_free or fr_destroy.  FR_ENOMEM when the device cannot
 * hold it. */
fr_status fr_volume_create(fr_ctx *ctx, int nx, int ny, int nz, const float origin[3], float h, int kind,
                           int dtype, fr_volume *out);
/* Frees a volume from fr_volume_create on this context (after the context's
 * queued work is done) and sets vol->data to NULL; FR_EINVAL for any other
 * volume. */
fr_status fr_volume_free(fr_ctx *ctx, fr_volume *vol);
/* Writes a volume's records from float32 values in record layout (nodes x 4
 * {S_r, S_g, S_b, sigma} for RGB, nodes x 2 {T, sigma} for TEMP), rounded to
 * the storage type to nearest even.  src: host memory when src_is_host (copied
 * in stream order: pinned memory must stay unchanged until the context's
 * stream has passed the copy), else device memory, 16-byte aligned.  16-bit
 * volumes need 8-byte-aligned data.  Asynchronous. */
fr_status fr_volume_upload(fr_ctx *ctx, fr_volume *vol, const float *src, int src_is_host);
/* Reads a volume's records as float32 values in record layout into dst (host
 * when dst_is_host: filled when the call returns, which synchronises the
 * context's stream; else device, 16-byte aligned, asynchronous). */
fr_status fr_volume_download(fr_ctx *ctx, const fr_volume *vol, float *dst, int dst_is_host);

/* ---- Camera sets (host memory owned by the library, no device) ---- */

typedef struct fr_cams fr_cams;

/* k calibrated cameras from 3x4 projections (P: k x 12 doubles, row-major,
 * each as fr_camera_from_projection takes it; wh: k x {width, height}), the
 * calibration output of Sec. 4.1.  FR_EINVAL when a projection is not a
 * pinhole of fr_camera's model or the images differ in size. */
fr_status fr_cams_create(int k, const double *P, const int32_t *wh, fr_cams **out);
/* k cameras on a ring around `center` (world units), as the paper's simulated
 * cameras surround the fire looking at it (Sec. 5.1): camera i at azimuth
 * phase + 2 pi i / k (radians, measured from +x towards +z) and elevation
 * elevation_deg[i] (degrees, NULL: 0), at `radius` from the centre, looking at
 * it with +y up, vertical field of view fov_deg, images width x height. */
fr_status fr_cams_ring(int k, int width, int height, const float center[3], float radius, float fov_deg,
                       const float *elevation_deg, float phase, fr_cams **out);
/* The number of cameras, and the array the other entry points take (valid
 * until fr_cams_destroy). */
int32_t fr_cams_count(const fr_cams *cams);
const fr_camera *fr_cams_data(const fr_cams *cams);
fr_status fr_cams_destroy(fr_cams *cams);

/* ---- Tracing: device time per phase of fr_reconstruct ---- */

typedef enum {
    FR_PHASE_SETUP = 0,   /* flame-ray list; visual hull tags, clear and bricks;
                             the ray weight tables' build */
    FR_PHASE_SCATTER = 1, /* in-scattering source (Sec. 3.2) */
    FR_PHASE_PACK = 2,    /* x-pair records and brick occupancy */
    FR_PHASE_FORWARD = 3, /* forward march with the residual (Eqs. 5-8); on the
                             tables, the staging of the records and the forward
                             table */
    FR_PHASE_REDUCE = 4,  /* squared-error reduction (0 on the tables, whose
                             adjustment launch runs it) */
    FR_PHASE_ADJUST = 5,  /* adjustment (Eqs. 10-12) or the exact gradient; on
                             the tables also the update and the error sums */
    FR_PHASE_APPLY = 6,   /* update of the volume, hull clear */
    FR_PHASE_FINISH = 7,  /* error measure of the call */
    FR_PHASE_COUNT = 8
} fr_phase;

/* on != 0: the following fr_reconstruct calls record a CUDA event on the
 * context's stream after each phase (a few microseconds of device time per
 * event); on == 0 stops.  Either way, what was recorded before is dropped. */
fr_status fr_trace_phases(fr_ctx *ctx, int on);
/* Waits for the recorded events and writes ms[p] (host, n >= FR_PHASE_COUNT
 * entries) = milliseconds spent in phase p summed over every call recorded
 * since tracing was turned on or last read, and *calls (host, nullable) = the
 * number of those calls; then drops the record.  FR_ERANGE when more than
 * 65536 events went unread (the later ones were not recorded). */
fr_status fr_phase_times(fr_ctx *ctx, float *ms, int n, int32_t *calls);

/* Sizes of the ray weight tables the context's last fr_reconstruct or
 * fr_reconstruct_until call built (fr_params.tables; all 0 when that call
 * marched): stats[0] forward entries (one per ray and key point of the hull
 * it samples, padded to whole rows of 32 rays; 8 bytes each), stats[1]
 * adjustment entries (one per flame ray and key point; 8 bytes each),
 * stats[2] flame rays, stats[3] key points inside the hull.  Host only; no
 * device work. */
fr_status fr_table_stats(const fr_ctx *ctx, uint64_t stats[4]);

/* Number of samples (segments) the rays of `cams` take through the volume's
 * box: all rays when residual is NULL (one render; when p->skip_empty applies,
 * the samples in bricks whose records are all zero are skipped by the render
 * and not counted), else only the rays whose residual (device, image layout)
 * is non-zero (one adjustment; with p->skip_empty, p->use_hull and
 * p->hull_tags, the samples fr_reconstruct's adjustment evaluates).  Counted by a
 * device kernel; *samples (host) is written before the call returns (the
 * call synchronises the stream). */
fr_status fr_count_samples(fr_ctx *ctx, const fr_volume *vol, const fr_camera *cams,
                           int ncam, const fr_params *p, const float *residual,
                           int64_t *samples);

/* fr_render_residual without any allocation.  (The paper has no counterpart:
 * this is a service for callers that cannot allocate device memory while they
 * render -- e.g. a process that gives all device memory to its own pool at
 * start-up, or a latency-critical loop that forbids cudaMalloc/cudaFree after
 * start-up because they can synchronise the whole device.)
 * The same results as fr_render_residual within float32 rounding (the records
 * are gathered one by one rather than in x-pairs and the error sums are added
 * in another order); the caller passes every input and output.  The per-tile
 * squared-error partials live in one fixed device array compiled into the
 * library (FR_NOALLOC_MAX_TILES tiles of 16 x 8 pixels, 1 MiB), which every GPU
 * that loads the library holds until the process exits.  Images of more
 * tiles, ncam * ceil(W/16) * ceil(H/8), are rejected with FR_EINVAL.  The first
 * call on a device, with the device made current (the calling thread's current
 * device is restored afterwards), looks up that array's device address and
 * loads the array and every kernel this entry point launches -- the module
 * loading that CUDA would otherwise do lazily at a first launch, which takes
 * device memory.  Make that first call before the caller's pool takes the
 * device's memory and before any stream capture; after a cudaDeviceReset in
 * the same process the looked-up address is stale, so the entry point must not
 * be called again on that device.  All calls share the array: calls whose work
 * overlaps on the GPU (e.g. on two streams at once) race; calls queued one
 * after another are safe, since every tile overwrites its own partials and
 * nothing needs clearing.
 * stream: cudaStream_t to queue on (NULL = default stream).  err (nullable):
 * receives the failure message (empty on success), at most err_len bytes. */
#define FR_NOALLOC_MAX_TILES 65536
fr_status fr_render_residual_noalloc(int device, void *stream, const fr_volume *vol,
                                     const fr_camera *cams, int ncam, const fr_params *p,
                                     const float *targets, const int32_t *bbox, float *rendered,
                                     float *residual, float *sq_err, char *err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* FLAMEREC_H */
