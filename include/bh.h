/*
 * bh.h -- C-ABI of the GB300 Schwarzschild light-ray renderer.
 *
 * The renderer computes, for every pixel of one or more pinhole cameras, the
 * light ray that reaches the pixel in the Schwarzschild geometry of a
 * non-spinning black hole of mass M (units G = c = 1):
 *   - one ray per pixel (Naddell & Ponce, PEARC '25, Sec. 1, last paragraph);
 *   - the ray is reduced to its orbital plane through the hole and the
 *     photon-orbit equation in u = 1/r against the azimuth phi is integrated
 *     (Sec. 1, Eq. 1; printed as u'' - u = 3Mu^2, used with the sign fixed by
 *     the first integral (u')^2 + u^2 - 2Mu^3 = 1/b^2, i.e. u'' = 3Mu^2 - u);
 *   - initial conditions come from the camera ray (Sec. 2.2);
 *   - the paper's fixed-step GSL stepper and piecewise-linear intersection
 *     (Sec. 2.1-2.2) are replaced by adaptive Dormand-Prince 5(4) with event
 *     location on the quintic Hermite interpolant of each step;
 *   - events: escape, capture by the hole, a thin equatorial disk, up to 8
 *     opaque spheres; the result is mapped back to 3-D and shaded against a
 *     procedural checkerboard sky.
 *
 * Conventions shared by every entry point:
 *   - Pointers named out_* / dev_* are DEVICE pointers unless stated; the
 *     caller owns them.  Host arrays (w, h, cams) are read during the call.
 *   - Rendering is asynchronous on opts->stream (a cudaStream_t; NULL is the
 *     legacy default stream) unless the entry point says it synchronises.
 *   - Every function returns BH_OK (0) or a negative BH_E_* code and never
 *     throws; bh_last_error() gives a text for the calling thread's last
 *     failure.
 *   - Output layout: rays are ordered camera-major, then row-major within a
 *     camera (row 0 at the top of the image), total N = sum_i w[i] * h[i].
 *     out_dirs is structure-of-arrays: theta[0..N) then phi[N..2N), float32
 *     in the FP32 / MIXED / SURROGATE modes and float64 in the FP64 mode.
 *     theta = acos(z) in [0, pi], phi = atan2(y, x) in [0, 2 pi) of the
 *     asymptotic exit direction (escape) or of the hit position (disk,
 *     sphere); NaN when captured or when the step cap was reached.
 *     out_flags is uint16 per ray: low byte = BH_FLAG_* bits, high byte =
 *     sphere index for BH_FLAG_SPHERE.  out_rgba8 is uint32 per ray with bytes
 *     R, G, B, A in memory order (A = 255).
 *   - A scene object may be used by one render at a time: its device
 *     workspace (queue counters, statistics, overflow lists) is shared by
 *     every call on it.
 */
#ifndef BH_H_
#define BH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BH_ABI_VERSION 2
#define BH_MAX_SPHERES 8

/* ---- return codes ---------------------------------------------------- */
#define BH_OK 0
#define BH_E_INVALID (-1)      /* bad argument: null pointer, size, range */
#define BH_E_NOMEM (-2)        /* device or host allocation failed        */
#define BH_E_CUDA (-3)         /* a CUDA runtime call failed              */
#define BH_E_DEVICE (-4)       /* device status word: watchdog / abort    */
#define BH_E_NO_SURROGATE (-5) /* surrogate mode without trained weights  */
#define BH_E_IO (-6)           /* file read/write failed or corrupt       */
#define BH_E_UNSUPPORTED (-7)  /* option or mode this entry point lacks   */

/* ---- precision modes ------------------------------------------------- */
#define BH_MODE_FP64 0      /* FP64 everywhere                              */
#define BH_MODE_FP32 1      /* FP32 everywhere                              */
#define BH_MODE_MIXED 2     /* FP32 stepping; FP64 for the periastron reset
                               of rays with |b - 3 sqrt(3) M| < 2M and the
                               integration of rays with |b - 3 sqrt(3) M| <
                               band                                         */
#define BH_MODE_SURROGATE 3 /* MLP surrogate with integrator fallback       */
#define BH_MODE_PAPER_EPS 4 /* the paper's own stepping (Sec. 2.1-2.2): fixed
                               steps paper_eps in phi with the classical
                               fourth-order Runge-Kutta method, straight
                               segments between the points, objects found by
                               segment intersection; FP64 (the paper's
                               precision), directions stored as double     */
#define BH_MODE_PAPER_EPS_FP32 5 /* the same in FP32, directions as float  */

/* most strips a bh_render_host frame is cut into (bh_render_opts)          */
#define BH_MAX_HOST_STRIPS 16

/* ---- initial-condition conventions (Sec. 2.2 reading) ---------------- */
#define BH_IC_STATIC 0    /* camera is a static observer (default)        */
#define BH_IC_EUCLIDEAN 1 /* successor point along the straight direction */

/* ---- per-ray flags (low byte of out_flags) ---------------------------- */
#define BH_FLAG_ESC 1u         /* escaped to infinity                       */
#define BH_FLAG_CAPT 2u        /* captured by the hole                      */
#define BH_FLAG_DISK 4u        /* hit the thin disk                         */
#define BH_FLAG_SPHERE 8u      /* hit a sphere (index in the high byte)     */
#define BH_FLAG_BAND 16u       /* |b - b_c| < band (MIXED / SURROGATE)      */
#define BH_FLAG_FP64 32u       /* integrated in FP64                        */
#define BH_FLAG_SURR 64u       /* result taken from the surrogate           */
#define BH_FLAG_STEP_LIMIT 128u/* step or angle cap reached                 */

/* ---- device status bits (bh_stats.status) ----------------------------- */
#define BH_STATUS_ABORTED 1u   /* abort_after item count reached            */
#define BH_STATUS_WATCHDOG 2u  /* persistent loop iteration limit reached, or
                                  a tensor-core layer of the surrogate pass
                                  not completed within its wait limit      */

typedef struct bh_scene bh_scene; /* opaque; owns device state */

typedef struct bh_sphere {
  double center[3]; /* world position, units of length (M = mass)         */
  double radius;    /* > 0                                                 */
  double albedo[3]; /* linear RGB in [0, 1]                                */
} bh_sphere;

/* Scene description (copied by bh_scene_create). */
typedef struct bh_scene_desc {
  double mass;        /* M >= 0                                            */
  int disk_enabled;   /* thin equatorial (z = 0) disk annulus              */
  double disk_r_in;   /* 2M < r_in < r_out                                  */
  double disk_r_out;
  int n_spheres;      /* 0..BH_MAX_SPHERES; |c| - R > 2M, no overlap check */
  bh_sphere spheres[BH_MAX_SPHERES];
  uint64_t sky_seed;  /* checkerboard sky tint seed                        */
  int ic;             /* BH_IC_STATIC or BH_IC_EUCLIDEAN                   */
} bh_scene_desc;

/* Pinhole camera.  bh_camera_set fills every field from the four angles;
 * the derived basis is what the kernels read.  The renderers accept only
 * cameras that look at the hole (fwd = -pos / r_obs, right and up an
 * orthonormal basis perpendicular to it, to 1e-9), as bh_camera_set makes
 * them: the kernels reduce each ray to its orbital plane from its image-plane
 * coordinates (Sec. 2.2: the camera's line of sight through the hole). */
typedef struct bh_camera {
  double r_obs, incl_deg, azim_deg, fov_deg;
  double pos[3];   /* r_obs (sin i cos a, sin i sin a, cos i)              */
  double fwd[3];   /* -pos / r_obs: looks at the hole                      */
  double right[3]; /* fwd x up_world, normalised (up_world = +z, or +x)    */
  double up[3];    /* right x fwd                                          */
  double tan_half; /* tan(fov / 2), fov across the full image width        */
} bh_camera;

typedef struct bh_render_opts {
  int mode;           /* BH_MODE_*                                          */
  double rtol, atol;  /* Dormand-Prince tolerances (0: 1e-10 / 1e-10 in FP64,
                         1e-5 / 1e-7 in FP32 and MIXED)                     */
  double band;        /* FP64 / fallback band half-width in b (0: 0.05 M)    */
  double band_rtol;   /* rtol = atol of the MIXED FP64 band pass (0: 1e-8)   */
  double phi_max;     /* azimuth cap in rad (0: 64)                          */
  int max_steps;      /* attempted-step cap per ray (0: 100000)              */
  double h_max;       /* largest step in rad (0: none in FP64, 0.3 otherwise;
                         the quintic event interpolant needs short steps)   */
  void *stream;       /* cudaStream_t                                       */
  /* launch shape; 0 selects the tuned value for this device and mode      */
  int block_size;     /* threads per block: 64, 128, 256 or 512             */
  int blocks_per_sm;  /* resident blocks per SM in the persistent grid      */
  int tile_w, tile_h; /* pixel tile of the work queue: tile_w * tile_h a
                         power of two in [32, 256], tile_w a power of two;
                         its pixels are queued row-major, and a warp takes
                         them 32 at a time                                 */
  int budget;         /* steps a ray may take in the coherent pass before it
                         moves to the long-ray queue                        */
  int periastron_reset; /* MIXED: reset the state at the turning point from
                           the FP64 periastron: 1 (or 0) = for rays with
                           |b - 3 sqrt(3) M| < 2M (default), 2 = for every
                           ray with a turning point, -1 = off               */
  uint32_t abort_after; /* fault injection: stop after this many work items
                           and report BH_E_DEVICE (0 = off)                 */
  double h_max_far;   /* largest step in rad for rays with |b - 3 sqrt(3) M|
                         >= 2M in the FP32 passes, whose outputs are far less
                         sensitive to stepping errors (0: 0.5; FP64: h_max) */
  double paper_eps;   /* fixed step in rad of the BH_MODE_PAPER_EPS modes
                         (0: 0.01)                                          */
  int spp;            /* samples per pixel, a square n*n (0 or 1: one ray
                         through the pixel centre).  With n > 1 the n x n
                         stratified sub-pixel samples (centres of an n x n
                         grid over the pixel) are averaged in linear colour
                         into RGBA8 (box filter) and one more ray through
                         the pixel centre gives its direction and flags.
                         BH_MODE_FP32 and BH_MODE_FP64 only (else
                         BH_E_UNSUPPORTED); n <= 16                          */
  int doppler;        /* 1: shade the disk as gas on prograde Keplerian orbits
                         about +z, seen by the static camera: frequency ratio
                         g = sqrt(1 - 3M/r) / (sqrt(1 - 2M/r_obs)(1 + Omega b
                         n_z)), Omega = sqrt(M/r^3), b n_z the traced ray's
                         angular momentum about z; the colour ramp is taken
                         at g t and scaled by g^3 (g = 0 inside 3M).  The
                         integrator modes only (else BH_E_UNSUPPORTED)      */
  double rtol_far;    /* rtol of rays with |b - 3 sqrt(3) M| >= 2M in the FP32
                         passes (their atol scales with it); their exit
                         directions amplify local errors far less (0: 10 x
                         rtol; FP64: rtol)                                  */
  int host_strips;    /* bh_render_host: the frame is rendered in this many
                         strips of whole tile rows, each copied to the host
                         while the next renders (0: about 2^21 rays a strip;
                         at most BH_MAX_HOST_STRIPS; the surrogate renders
                         whole)                                             */
  double rtol_near;   /* BH_MODE_FP32: rtol of rays with |b - 3 sqrt(3) M| <
                         band (their atol scales with it); their capture
                         decision and exit direction depend on the first
                         integral to a few parts in 1e6 (0: rtol / 100; the
                         other modes integrate those rays in FP64)          */
  int queue_chunk;    /* queue slots (rays) a warp takes per grab of the
                         global work counter, a multiple of 32 in [32, 1024];
                         0: the tuned value                                 */
} bh_render_opts;

typedef struct bh_stats {
  uint64_t rays;          /* rays traced (including padding-free pixels only)*/
  uint64_t steps;         /* attempted Dormand-Prince steps                  */
  uint64_t rejected;      /* rejected steps                                  */
  uint64_t n_esc, n_capt, n_disk, n_sphere, n_step_limit;
  uint64_t n_band;        /* rays integrated in FP64 because of the band     */
  uint64_t n_long;        /* rays moved to the long-ray queue               */
  uint64_t n_surrogate;   /* rays answered by the surrogate                  */
  uint64_t n_fallback;    /* surrogate rays sent back to the integrator      */
  uint64_t queue_grabs;   /* work-queue atomic grabs                         */
  uint64_t periastron;    /* periastron resets (MIXED)                       */
  uint64_t events;        /* event-handling passes (nodes, windows, roots)   */
  uint64_t steps_fp64;    /* attempted steps taken in FP64 (part of steps)   */
  uint32_t status;        /* BH_STATUS_* bits of the last render             */
  float kernel_ms[4];     /* device time of the last render: [0] the tile pass
                             and the long-ray pass, which starts as its
                             programmatic dependent (MIXED: with the band
                             list and the FP64 band pass, which runs beside
                             them; SURROGATE: the band list and the
                             surrogate pass), [1] the surrogate mode's
                             integrator pass over the rays the network does
                             not answer (0 otherwise), [2] FP64 band pass
                             of the surrogate mode (on a side stream beside
                             [0] and [1]; 0 otherwise), [3] whole render   */
  uint64_t mlp_rays;      /* rays the surrogate network was evaluated for:
                             32 per warp that had a ray to serve            */
} bh_stats;

/* Library version (BH_ABI_VERSION). */
int bh_version(void);

/* Text of the calling thread's last error ("" if none).  The pointer stays
 * valid until the thread's next failing call. */
const char *bh_last_error(void);

/* Create a scene: validates desc (mass >= 0, 2M < r_in < r_out, at most 8
 * spheres each with radius > 0 lying outside r = 2M, ic in {0, 1}), copies
 * it and allocates the device workspace on the current device.
 * Errors: BH_E_INVALID, BH_E_NOMEM, BH_E_CUDA. */
int bh_scene_create(const bh_scene_desc *desc, bh_scene **out);

/* Release a scene and its device memory (NULL is ignored).  Waits for the
 * device to finish using it. */
void bh_scene_destroy(bh_scene *scene);

/* Fill a camera looking at the hole from radius r_obs > 2M at inclination
 * incl_deg from the +z axis and azimuth azim_deg, with 0 < fov_deg < 180
 * across the image width (Sec. 1: one ray through each pixel centre).
 * Errors: BH_E_INVALID. */
int bh_camera_set(bh_camera *cam, double r_obs, double incl_deg, double azim_deg,
                  double fov_deg);

/* Use an image as the sky (the paper renders photographs as backgrounds,
 * Sec. 3.1) in place of the procedural checker: texels is a host array of
 * w x h RGBA8 values (red in the low byte), row-major, equirectangular --
 * row j holds theta = (j + 1/2) pi / h measured from the +z pole, column i
 * holds phi = (i + 1/2) 2 pi / w.  The colour in a direction is bilinear in
 * linear colour between the four nearest texel centres, wrapping in phi and
 * clamped at the first and last rows.  The library copies the image to the
 * device (the caller keeps ownership of texels); texels = NULL restores the
 * checker.  Synchronises the device.  w <= 65536, h <= 32768.
 * Errors: BH_E_INVALID, BH_E_CUDA. */
int bh_scene_sky_texture(bh_scene *scene, const uint32_t *texels, int w, int h);

/* Render n_cams cameras in one persistent launch sequence.
 *   cams[n_cams], w[n_cams], h[n_cams]: host arrays; w, h >= 1; the total
 *     ray count must stay below 2^31 - 1.
 *   out_dirs: device, 2N elements (float32 or float64, see above).
 *   out_flags: device, N uint16.   out_rgba8: device, N uint32.
 * Any output pointer may be NULL to skip that output.  Asynchronous on
 * opts->stream; the camera table is uploaded on that stream.
 * Errors: BH_E_INVALID, BH_E_NOMEM, BH_E_CUDA, BH_E_NO_SURROGATE. Device-side
 * aborts surface through bh_render_stats / bh_scene_sync. */
int bh_render(const bh_scene *scene, const bh_camera *cams, int n_cams, const int *w,
              const int *h, void *out_dirs, uint16_t *out_flags, uint32_t *out_rgba8,
              const bh_render_opts *opts);

/* Same render into HOST buffers (pageable or pinned; pinned copies are
 * faster): renders into scene-owned device staging and copies back, then
 * synchronises before returning.  Layouts as for bh_render, results
 * identical to it.  The integrator modes render the frame in strips of
 * whole tile rows (opts->host_strips) on opts->stream, each strip's outputs
 * copied on a scene-owned copy stream while the next strip renders; the
 * MIXED FP64 band pass runs once for the frame on the scene's side stream.
 * The surrogate mode renders whole, then copies.  Kernel times are not
 * recorded for bh_render_stats (its counts cover the whole frame).
 * Errors: as bh_render; BH_E_INVALID for host_strips outside
 * [0, BH_MAX_HOST_STRIPS]. */
int bh_render_host(const bh_scene *scene, const bh_camera *cams, int n_cams, const int *w,
                   const int *h, void *host_dirs, uint16_t *host_flags,
                   uint32_t *host_rgba8, const bh_render_opts *opts);

/* Wait for the scene's last render and report its device status:
 * BH_E_DEVICE if an abort or watchdog bit is set, else BH_OK. */
int bh_scene_sync(const bh_scene *scene);

/* Statistics of the scene's last render (synchronises its stream). */
int bh_render_stats(const bh_scene *scene, bh_stats *out);

/* ---- MLP surrogate -------------------------------------------------------
 * An MLP maps (b/M, r_obs/M, psi0) -- impact parameter, observer radius and
 * the azimuth of the first disk node in the orbital plane -- to the
 * deflection delta = phi_inf - alpha (alpha: the flat-space exit angle) and
 * u b at the disk nodes psi0 and psi0 + pi: 3 inputs, 3 hidden layers of 64
 * with SiLU, 3 outputs; tensor-core operands with FP32 accumulation: BF16
 * in training (FP32 master weights and Adam), the trained BF16 weight values
 * held exactly in FP16 for inference, whose activations enter as FP16
 * high + low pairs.  It is
 * trained on labels the FP64 integrator computes, and calibrated on held-
 * out samples: per bin of (ln(b - 3 sqrt 3 M), r_obs) the 99.9th-percentile
 * error decides whether BH_MODE_SURROGATE may answer rays there.  Rays in
 * the photon-sphere band, outside the training domain, in a failing bin, or
 * whose orbital plane cuts a sphere are finished by the integrator.  There
 * is no surrogate in the paper; the integrator is the reference for its error. */
typedef struct bh_train_opts {
  int epochs;            /* passes over the training samples (0: 20)       */
  int batch;             /* samples per Adam step, multiple of 32 (0: 16384) */
  double lr;             /* peak Adam learning rate, cosine decay (0: 2e-3) */
  uint64_t seed;         /* weight initialisation and shuffling            */
  double val_fraction;   /* held out for calibration (0: 0.05)             */
  double err_threshold;  /* served bins: p99.9 |delta error| (0: 1e-3 rad) */
  double r_err_threshold;/* and p99.9 relative crossing-radius error |dr|/r
                            (0: 2e-3)                                       */
  void *stream;          /* cudaStream_t                                   */
} bh_train_opts;

typedef struct bh_train_report {
  int n_samples, n_valid, n_train, n_val, steps;
  float final_loss;      /* mean training loss of the last epoch           */
  float val_rmse[3];     /* held-out RMSE of the three normalised outputs  */
  float served_fraction; /* held-out samples falling in served bins        */
  float label_ms, train_ms, calib_ms;
} bh_train_report;

/* FP64 labels of bare orbits (device arrays of n): from r_obs with impact
 * parameter b (units of M = mass), ingoing, static-observer initial state;
 * phi_inf = escape azimuth, u_a / u_b = u at psi0 / psi0 + pi (continued
 * past escape, where u < 0).  status: 0 ok, 1 no such ray from r_obs
 * (b too large), 2 captured, 3 cap reached (labels NaN unless 0).
 * Asynchronous on stream.  Errors: BH_E_INVALID, BH_E_CUDA. */
int bh_surrogate_labels(double mass, int n, const double *b, const double *r_obs,
                        const double *psi0, double *phi_inf, double *u_a, double *u_b,
                        int *status, void *stream);

/* Train the scene's surrogate on n host samples (b, r_obs, psi0) in units
 * of M (labels from bh_surrogate_labels; invalid samples are dropped),
 * calibrate it and keep it on the scene.  The loss is the mean squared
 * error of the normalised outputs with the deflection term weighted by
 * min(25, (10/b)^2), as its error in radians scales like 1/b.
 * Synchronous.  report may be NULL.
 * Errors: BH_E_INVALID, BH_E_NOMEM, BH_E_CUDA. */
int bh_surrogate_train(bh_scene *scene, int n, const double *b, const double *r_obs,
                       const double *psi0, const bh_train_opts *opts, bh_train_report *report);

/* Recalibrate the scene's trained surrogate on n host samples (b, r_obs,
 * psi0), units of M, that it was not trained on.  Each sample is labelled
 * with the FP64 integrator (bh_surrogate_labels) and predicted by the
 * network; samples are binned by the network's first feature
 * (ln(b - 3 sqrt 3) normalised to [-1, 1], nb_lb bins) and by r_obs over
 * [15, 100] M (nb_r bins).  Per bin the 99.9th percentile of the
 * deflection error (rad) and of the relative disk-crossing radius error
 * |dr| / r (true crossings within 2.5 M < r < 60 M) are taken; a bin is served when it
 * holds >= 50 samples and both are within the thresholds.  The new table
 * replaces the scene's (and is what bh_surrogate_save writes).
 * Outputs (host, nb_lb * nb_r entries, bin = i_lb * nb_r + i_r, NULL to
 * skip): p999_delta (rad), p999_r (relative), counts; served_fraction = share of valid
 * samples in served bins.  Synchronous.
 * Errors: BH_E_INVALID, BH_E_NO_SURROGATE, BH_E_NOMEM, BH_E_CUDA. */
typedef struct bh_calib_opts {
  int nb_lb;              /* bins over ln(b - 3 sqrt 3) (0: 32, <= 1024)   */
  int nb_r;               /* bins over r_obs in [15, 100] M (0: 8, <= 1024) */
  double err_threshold;   /* p99.9 |delta error| bound (0: 1e-3 rad)       */
  double r_err_threshold; /* p99.9 relative crossing-radius bound (0: 2e-3) */
  void *stream;           /* cudaStream_t                                  */
} bh_calib_opts;
int bh_surrogate_calibrate(bh_scene *scene, int n, const double *b, const double *r_obs,
                           const double *psi0, const bh_calib_opts *opts, float *p999_delta,
                           float *p999_r, int *counts, float *served_fraction);

/* Copy the trained surrogate out (any pointer may be NULL): FP32 parameters
 * (BH_MLP_NPARAM), calibration table (nb_lb * nb_r bytes).
 * Errors: BH_E_INVALID, BH_E_NO_SURROGATE. */
#define BH_MLP_NPARAM 10448
int bh_surrogate_get(const bh_scene *scene, float *params, unsigned char *table, int *nb_lb,
                     int *nb_r);

/* Save / load the trained surrogate (parameters and calibration table; a
 * file with magic, version, shapes and an FNV-1a checksum).
 * Errors: BH_E_INVALID, BH_E_NO_SURROGATE, BH_E_IO, BH_E_CUDA. */
int bh_surrogate_save(const bh_scene *scene, const char *path);
int bh_surrogate_load(bh_scene *scene, const char *path);

/* Diagnostics of the training kernels, on HOST arrays: one forward and
 * backward pass of the MLP with FP32 parameters params (BH_MLP_NPARAM,
 * row-major W[in][out] per layer, weights BF16-rounded on the device) over
 * n samples (multiple of 32) of feature rows x[n][16] (12 used) and
 * targets t[n][3]: outputs y[n][3], the gradient of the mean squared error
 * over the 3 outputs with respect to every parameter, and the loss.
 * Synchronous. */
int bh_mlp_grad(const float *params, int n, const float *x, const float *t, float *y,
                float *grad, float *loss, void *stream);
/* The render's inference path (tcgen05 tensor-core MLP, 128 rows a CTA, the
 * parameters' BF16 weight values held in FP16) on host feature rows
 * x[n][16] -> y[n][3].  Synchronous.  BH_E_DEVICE if a layer's MMAs did
 * not complete within the kernel's wait limit. */
int bh_mlp_infer(const float *params, int n, const float *x, float *y, void *stream);

/* Self-test of the bounded waits of the tensor-core kernels: one CTA
 * allocates tensor memory as those kernels do, waits on an mbarrier that
 * nothing arrives on with their wait (up to `tries` waits of `wait_ns`
 * nanoseconds each, both clamped to [1, 10000] and [1, 1000000]), gives up,
 * frees the tensor memory and reports.  *timed_out = 1 when the wait gave up
 * (the expected outcome), *waited_ms = the wait's device time.  Nothing
 * faults or hangs; the device stays usable.  Synchronous.  BH_E_INVALID for
 * null outputs. */
int bh_selftest_wait_timeout(int tries, int wait_ns, int *timed_out, double *waited_ms);

/* ---- batched launch in a CUDA graph, autotuning ------------------------
 * One render of n_cams cameras (Sec. 3.2's scaling runs render many images;
 * here many cameras of uneven resolution share one persistent launch
 * sequence) captured once and replayed.  The graph owns a copy of the
 * camera table; it renders into the output buffers given at creation and
 * uses the scene's workspace, so graph launches and other renders on the
 * same scene must not overlap.  Modes: FP64, FP32, MIXED.
 * Errors: BH_E_INVALID, BH_E_NOMEM, BH_E_CUDA, BH_E_UNSUPPORTED. */
typedef struct bh_graph bh_graph;
int bh_graph_create(bh_scene *scene, const bh_camera *cams, int n_cams, const int *w,
                    const int *h, void *out_dirs, uint16_t *out_flags, uint32_t *out_rgba8,
                    const bh_render_opts *opts, bh_graph **out);
/* Replay on a stream (a cudaStream_t); asynchronous. */
int bh_graph_launch(bh_graph *graph, void *stream);
void bh_graph_destroy(bh_graph *graph);

typedef struct bh_tune_result {
  int block_size, blocks_per_sm, tile_w, tile_h, budget; /* the fastest shape */
  float ms_best;     /* its render time                                   */
  float ms_default;  /* render time with the built-in default shape        */
  int trials;        /* shapes timed                                       */
  int queue_chunk;   /* queue slots per warp grab of the fastest shape     */
} bh_tune_result;

/* Time candidate launch shapes (block size, tile shape, step budget and, in
 * MIXED, the resident blocks left to the band pass) on this workload -- each
 * a full render into the given device buffers, synchronising the stream --
 * and keep the fastest for the scene's device and this mode: later renders
 * and graphs whose opts leave those fields 0 use it.  Modes: FP64, FP32,
 * MIXED.  Errors as bh_render, plus BH_E_UNSUPPORTED. */
int bh_autotune(bh_scene *scene, const bh_camera *cams, int n_cams, const int *w, const int *h,
                void *out_dirs, uint16_t *out_flags, uint32_t *out_rgba8,
                const bh_render_opts *opts, bh_tune_result *out);
/* Forget every tuned shape (back to the built-in defaults). */
int bh_autotune_reset(void);

/* ---- render without allocating ----------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot call cudaMalloc: hosts that give all device memory to their own
 * pool or a fixed budget and forbid other allocations, and real-time loops
 * in which an allocation may synchronise the device or fail in mid-frame.
 *
 * It renders like bh_render in BH_MODE_FP32 or BH_MODE_FP64 (other modes:
 * BH_E_UNSUPPORTED) but allocates nothing and needs no bh_scene: the scene
 * is read from desc on every call, and the only scratch -- the work-queue
 * counter, status and statistics words and the camera table -- lives in one
 * fixed library-owned device array of about 48 KB, present on every device
 * that loads the library until the process exits.  Every ray is finished by
 * the coherent pass (no long-ray list) with the kernels bh_render uses, so
 * the outputs equal bh_render's for the same options.
 *   - desc, cams, w, h: host, as for bh_scene_create / bh_render;
 *     n_cams <= BH_NOALLOC_MAX_CAMERAS, else BH_E_INVALID.
 *   - out_dirs, out_flags, out_rgba8: caller-owned device buffers laid out
 *     as for bh_render.
 *   - Asynchronous on opts->stream.  The camera table reaches the scratch
 *     array in the launch parameters of a copy kernel on that stream, so no
 *     device work of the call reads the caller's host memory after it
 *     returns.
 *   - opts->abort_after must be 0 (BH_E_UNSUPPORTED otherwise): this entry
 *     point reads no device status back.
 *   - The first call on a device looks up the scratch array's device
 *     address (with that device current); make that first call before any
 *     stream capture.
 *   - All calls share the one array and it keeps the last call's contents
 *     (counters are cleared at the start of each call): calls that overlap
 *     on the GPU, on any streams, race and must be serialised by the caller.
 * Errors: BH_E_INVALID, BH_E_UNSUPPORTED, BH_E_CUDA. */
#define BH_NOALLOC_MAX_CAMERAS 64
int bh_render_noalloc(const bh_scene_desc *desc, const bh_camera *cams, int n_cams,
                      const int *w, const int *h, void *out_dirs, uint16_t *out_flags,
                      uint32_t *out_rgba8, const bh_render_opts *opts);

#ifdef __cplusplus
}
#endif

#endif /* BH_H_ */
