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

#define BH_ABI_VERSION 1
#define BH_MAX_SPHERES 8

/* ---- return codes ---------------------------------------------------- */
#define BH_OK 0
#define BH_E_INVALID (-1)      /* bad argument: null pointer, size, range */
#define BH_E_NOMEM (-2)        /* device or host allocation failed        */
#define BH_E_CUDA (-3)         /* a CUDA runtime call failed              */
#define BH_E_DEVICE (-4)       /* device status word: watchdog / abort    */
#define BH_E_NO_SURROGATE (-5) /* surrogate mode without trained weights  */
#define BH_E_IO (-6)           /* file read/write failed or corrupt       */
#define BH_E_UNSUPPORTED (-7)  /* option not available in this build      */

/* ---- precision modes ------------------------------------------------- */
#define BH_MODE_FP64 0      /* FP64 everywhere                              */
#define BH_MODE_FP32 1      /* FP32 everywhere                              */
#define BH_MODE_MIXED 2     /* FP32 stepping; FP64 for the periastron reset
                               and for rays with |b - 3 sqrt(3) M| < band   */
#define BH_MODE_SURROGATE 3 /* MLP surrogate with integrator fallback       */

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
#define BH_STATUS_WATCHDOG 2u  /* persistent loop iteration limit reached   */

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
 * the derived basis is what the kernels read. */
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
  double band_rtol;   /* rtol = atol of the MIXED FP64 band pass (0: 1e-9)   */
  double phi_max;     /* azimuth cap in rad (0: 64)                          */
  int max_steps;      /* attempted-step cap per ray (0: 100000)              */
  double h_max;       /* largest step in rad (0: none in FP64, 0.3 otherwise;
                         the quintic event interpolant needs short steps)   */
  void *stream;       /* cudaStream_t                                       */
  /* launch shape; 0 selects the tuned value for this device and mode      */
  int block_size;     /* threads per block: 64, 128 or 256                  */
  int blocks_per_sm;  /* resident blocks per SM in the persistent grid      */
  int tile_w, tile_h; /* pixel tile that one warp takes (tile_w*tile_h = 32)*/
  int budget;         /* steps a ray may take in the coherent pass before it
                         moves to the long-ray queue                        */
  int periastron_reset; /* MIXED: 1 = reset state at the turning point (default),
                           -1 = off                                         */
  uint32_t abort_after; /* fault injection: stop after this many work items
                           and report BH_E_DEVICE (0 = off)                 */
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
  float kernel_ms[4];     /* device time of the last render: [0] coherent pass
                             (with the MIXED band pre-pass), [1] long-ray pass,
                             [2] FP64 band pass (MIXED; it overlaps [0] and [1]
                             on a side stream), [3] whole render            */
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

/* Same render into HOST buffers (pageable or pinned): renders into scene-
 * owned device staging, copies back and synchronises the stream before
 * returning.  Layouts as for bh_render. */
int bh_render_host(const bh_scene *scene, const bh_camera *cams, int n_cams, const int *w,
                   const int *h, void *host_dirs, uint16_t *host_flags,
                   uint32_t *host_rgba8, const bh_render_opts *opts);

/* Wait for the scene's last render and report its device status:
 * BH_E_DEVICE if an abort or watchdog bit is set, else BH_OK. */
int bh_scene_sync(const bh_scene *scene);

/* Statistics of the scene's last render (synchronises its stream). */
int bh_render_stats(const bh_scene *scene, bh_stats *out);

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
 * fixed library-owned device array of about 10 KB, present on every device
 * that loads the library until the process exits.  Every ray is finished by
 * the coherent pass (no long-ray list), so results equal bh_render's.
 *   - desc, cams, w, h: host, as for bh_scene_create / bh_render;
 *     n_cams <= BH_NOALLOC_MAX_CAMERAS, else BH_E_INVALID.
 *   - out_dirs, out_flags, out_rgba8: caller-owned device buffers laid out
 *     as for bh_render.
 *   - Asynchronous on opts->stream; the camera table is copied on it.
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
