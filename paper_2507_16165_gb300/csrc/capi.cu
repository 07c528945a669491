// C-ABI and host runtime: scenes, cameras, device workspace, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bh.h"
#include "render.h"
#include "runtime.h"

using namespace bhk;

// ---------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

int bh_fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int bh_cuda_fail(cudaError_t e, const char* what) {
  const int code = (e == cudaErrorMemoryAllocation) ? BH_E_NOMEM : BH_E_CUDA;
  return bh_fail(code, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" int bh_version(void) { return BH_ABI_VERSION; }

bool camera_looks_at_hole(const bh_camera& c) {
  auto dot = [](const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
  if (!(c.r_obs > 0.0)) return false;
  const double tol = 1e-9;
  for (int k = 0; k < 3; ++k)
    if (!(std::fabs(c.fwd[k] + c.pos[k] / c.r_obs) <= tol)) return false;
  return std::fabs(dot(c.fwd, c.fwd) - 1.0) <= tol && std::fabs(dot(c.right, c.right) - 1.0) <= tol &&
         std::fabs(dot(c.up, c.up) - 1.0) <= tol && std::fabs(dot(c.fwd, c.right)) <= tol &&
         std::fabs(dot(c.fwd, c.up)) <= tol && std::fabs(dot(c.right, c.up)) <= tol;
}

extern "C" const char* bh_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// Device selection guard: run on the scene's device, restore the caller's.
// ---------------------------------------------------------------------------
DeviceGuard::DeviceGuard(int dev) {
  cudaGetDevice(&prev_);
  if (prev_ != dev) cudaSetDevice(dev);
  dev_ = dev;
}
DeviceGuard::~DeviceGuard() {
  if (prev_ != dev_) cudaSetDevice(prev_);
}

// ---------------------------------------------------------------------------
// Scene
// ---------------------------------------------------------------------------
template <typename T>
static cudaError_t grow(T** ptr, size_t* cap, size_t need) {
  if (*cap >= need && *ptr) return cudaSuccess;
  if (*ptr) cudaFree(*ptr);
  *ptr = nullptr;
  *cap = 0;
  size_t n = std::max(need, (size_t)1);
  cudaError_t e = cudaMalloc((void**)ptr, n * sizeof(T));
  if (e == cudaSuccess) *cap = n;
  return e;
}

extern "C" int bh_scene_create(const bh_scene_desc* desc, bh_scene** out) {
  if (!desc || !out) return bh_fail(BH_E_INVALID, "bh_scene_create: null argument");
  *out = nullptr;
  const double M = desc->mass;
  if (!(M >= 0.0) || !std::isfinite(M)) return bh_fail(BH_E_INVALID, "mass must be >= 0");
  if (desc->disk_enabled &&
      !(desc->disk_r_in > 2.0 * M && desc->disk_r_out > desc->disk_r_in &&
        std::isfinite(desc->disk_r_out)))
    return bh_fail(BH_E_INVALID, "disk needs 2M < r_in < r_out");
  if (desc->n_spheres < 0 || desc->n_spheres > BH_MAX_SPHERES)
    return bh_fail(BH_E_INVALID, "n_spheres must be in [0, %d]", BH_MAX_SPHERES);
  if (desc->ic != BH_IC_STATIC && desc->ic != BH_IC_EUCLIDEAN)
    return bh_fail(BH_E_INVALID, "ic must be BH_IC_STATIC or BH_IC_EUCLIDEAN");
  double r_min_obj = INFINITY;
  if (desc->disk_enabled) r_min_obj = desc->disk_r_in;
  for (int k = 0; k < desc->n_spheres; ++k) {
    const bh_sphere& s = desc->spheres[k];
    const double c = std::sqrt(s.center[0] * s.center[0] + s.center[1] * s.center[1] +
                               s.center[2] * s.center[2]);
    if (!(s.radius > 0.0) || !(c - s.radius > 2.0 * M) || !std::isfinite(c))
      return bh_fail(BH_E_INVALID, "sphere %d must have radius > 0 and lie outside r = 2M", k);
    for (int j = 0; j < 3; ++j)
      if (!(s.albedo[j] >= 0.0 && s.albedo[j] <= 1.0))
        return bh_fail(BH_E_INVALID, "sphere %d albedo must be in [0, 1]", k);
    r_min_obj = std::min(r_min_obj, c - s.radius);
  }
  bh_scene* sc = new (std::nothrow) bh_scene();
  if (!sc) return bh_fail(BH_E_NOMEM, "bh_scene_create: host allocation failed");
  sc->desc = *desc;
  SceneK& k = sc->sk;
  memset(&k, 0, sizeof k);
  k.M = M;
  k.M3 = 3.0 * M;
  // Inside r = 3M an ingoing ray never turns back; with every object
  // outside 3M the capture decision can be taken there.
  k.u_capt = (M > 0.0) ? (r_min_obj > 3.0 * M ? 1.0 / (3.0 * M) : 1.0 / (2.0 * M)) : INFINITY;
  k.b_crit = 3.0 * std::sqrt(3.0) * M;
  k.disk_on = desc->disk_enabled ? 1 : 0;
  k.r_in = desc->disk_r_in;
  k.r_out = desc->disk_r_out;
  k.n_sph = desc->n_spheres;
  for (int i = 0; i < desc->n_spheres; ++i) {
    const bh_sphere& s = desc->spheres[i];
    double c2 = 0.0;
    for (int j = 0; j < 3; ++j) {
      k.c[i][j] = s.center[j];
      c2 += s.center[j] * s.center[j];
      k.alb[i][j] = (float)s.albedo[j];
    }
    k.c2[i] = c2;
    k.R[i] = s.radius;
    k.K[i] = c2 - s.radius * s.radius;
  }
  k.seed = desc->sky_seed;
  k.ic = desc->ic;
  fill_scene_r(k, &k.f);
  fill_scene_r(k, &k.d);
  cudaError_t e = cudaGetDevice(&sc->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sc->num_sms, cudaDevAttrMultiProcessorCount, sc->device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&sc->d_ws, sizeof(WorkK));
  if (e == cudaSuccess) e = cudaMemset(sc->d_ws, 0, sizeof(WorkK));
  if (e == cudaSuccess) e = cudaMalloc((void**)&sc->d_sky_lut, 512 * sizeof(float4));
  if (e == cudaSuccess) e = fill_sky_lut(k.seed, sc->d_sky_lut, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) k.sky_lut = sc->d_sky_lut;
  for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&sc->ev[i]);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreate(&sc->band_ev[i]);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sc->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sc->join, cudaEventDisableTiming);
  for (int i = 0; i < BH_MAX_HOST_STRIPS && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&sc->strip_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sc->copy, cudaStreamNonBlocking);
  if (e == cudaSuccess) {
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    e = cudaStreamCreateWithPriority(&sc->side, cudaStreamNonBlocking, greatest);
  }
  if (e != cudaSuccess) {
    const int rc = bh_cuda_fail(e, "bh_scene_create");
    bh_scene_destroy(sc);
    return rc;
  }
  *out = sc;
  return BH_OK;
}

extern "C" int bh_scene_sky_texture(bh_scene* sc, const uint32_t* texels, int w, int h) {
  if (!sc) return bh_fail(BH_E_INVALID, "bh_scene_sky_texture: null scene");
  DeviceGuard g(sc->device);
  if (!texels) {
    cudaDeviceSynchronize();
    cudaFree(sc->d_sky);
    sc->d_sky = nullptr;
    sc->sk.sky_tex = nullptr;
    sc->sk.sky_w = sc->sk.sky_h = 0;
    return BH_OK;
  }
  if (w < 1 || h < 1 || w > 65536 || h > 32768)
    return bh_fail(BH_E_INVALID, "bh_scene_sky_texture: size %dx%d out of range", w, h);
  const size_t bytes = (size_t)w * h * sizeof(uint32_t);
  uint32_t* d = nullptr;
  cudaError_t e = cudaMalloc(&d, bytes);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_scene_sky_texture: allocation");
  e = cudaMemcpy(d, texels, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(d);
    return bh_cuda_fail(e, "bh_scene_sky_texture: upload");
  }
  cudaDeviceSynchronize();  // no render may still read the old image
  cudaFree(sc->d_sky);
  sc->d_sky = d;
  sc->sk.sky_tex = d;
  sc->sk.sky_w = w;
  sc->sk.sky_h = h;
  return BH_OK;
}

extern "C" void bh_scene_destroy(bh_scene* sc) {
  if (!sc) return;
  {
    DeviceGuard g(sc->device);
    cudaDeviceSynchronize();
    cudaFree(sc->d_ws);
    cudaFree(sc->d_cams);
    cudaFree(sc->d_spill);
    cudaFree(sc->d_band);
    cudaFree(sc->d_stage_dirs);
    cudaFree(sc->d_stage_flags);
    cudaFree(sc->d_stage_rgba);
    cudaFree(sc->d_sky);
    cudaFree(sc->d_sky_lut);
    for (int i = 0; i < 4; ++i)
      if (sc->ev[i]) cudaEventDestroy(sc->ev[i]);
    for (int i = 0; i < 2; ++i)
      if (sc->band_ev[i]) cudaEventDestroy(sc->band_ev[i]);
    if (sc->fork) cudaEventDestroy(sc->fork);
    if (sc->join) cudaEventDestroy(sc->join);
    if (sc->side) cudaStreamDestroy(sc->side);
    for (int i = 0; i < BH_MAX_HOST_STRIPS; ++i)
      if (sc->strip_ev[i]) cudaEventDestroy(sc->strip_ev[i]);
    if (sc->copy) cudaStreamDestroy(sc->copy);
    surrogate_release(sc);
  }
  delete sc;
}

extern "C" int bh_camera_set(bh_camera* cam, double r_obs, double incl_deg, double azim_deg,
                             double fov_deg) {
  if (!cam) return bh_fail(BH_E_INVALID, "bh_camera_set: null camera");
  if (!(r_obs > 0.0) || !std::isfinite(r_obs) || !std::isfinite(incl_deg) ||
      !std::isfinite(azim_deg) || !(fov_deg > 0.0 && fov_deg < 180.0))
    return bh_fail(BH_E_INVALID, "bh_camera_set: need r_obs > 0 and 0 < fov < 180");
  const double pi = 3.14159265358979323846;
  const double i = incl_deg * pi / 180.0, a = azim_deg * pi / 180.0;
  cam->r_obs = r_obs;
  cam->incl_deg = incl_deg;
  cam->azim_deg = azim_deg;
  cam->fov_deg = fov_deg;
  cam->pos[0] = r_obs * std::sin(i) * std::cos(a);
  cam->pos[1] = r_obs * std::sin(i) * std::sin(a);
  cam->pos[2] = r_obs * std::cos(i);
  for (int k = 0; k < 3; ++k) cam->fwd[k] = -cam->pos[k] / r_obs;
  const double* f = cam->fwd;
  double upw[3] = {0.0, 0.0, 1.0};
  double rt[3] = {f[1] * upw[2] - f[2] * upw[1], f[2] * upw[0] - f[0] * upw[2],
                  f[0] * upw[1] - f[1] * upw[0]};
  double nr = std::sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
  if (nr < 1e-12) {  // looking along z: world +x is "up"
    upw[0] = 1.0;
    upw[2] = 0.0;
    rt[0] = f[1] * upw[2] - f[2] * upw[1];
    rt[1] = f[2] * upw[0] - f[0] * upw[2];
    rt[2] = f[0] * upw[1] - f[1] * upw[0];
    nr = std::sqrt(rt[0] * rt[0] + rt[1] * rt[1] + rt[2] * rt[2]);
  }
  for (int k = 0; k < 3; ++k) cam->right[k] = rt[k] / nr;
  const double* r = cam->right;
  cam->up[0] = r[1] * f[2] - r[2] * f[1];
  cam->up[1] = r[2] * f[0] - r[0] * f[2];
  cam->up[2] = r[0] * f[1] - r[1] * f[0];
  cam->tan_half = std::tan(0.5 * fov_deg * pi / 180.0);
  return BH_OK;
}

// ---------------------------------------------------------------------------
// Render
// ---------------------------------------------------------------------------
int check_render_args(const bh_scene* sc, const bh_camera* cams, int n_cams, const int* w,
                      const int* h, const bh_render_opts* opts) {
  if (!sc || !cams || !w || !h || !opts) return bh_fail(BH_E_INVALID, "bh_render: null argument");
  if (n_cams < 1 || n_cams > kMaxCameras)
    return bh_fail(BH_E_INVALID, "bh_render: n_cams must be in [1, %d]", kMaxCameras);
  if (opts->mode < BH_MODE_FP64 || opts->mode > BH_MODE_PAPER_EPS_FP32)
    return bh_fail(BH_E_INVALID, "bh_render: unknown mode %d", opts->mode);
  for (int i = 0; i < n_cams; ++i) {
    if (w[i] < 1 || h[i] < 1 || w[i] > 65536 || h[i] > 65536)
      return bh_fail(BH_E_INVALID, "bh_render: camera %d size %dx%d out of range", i, w[i], h[i]);
    if (!(cams[i].r_obs > 2.0 * sc->sk.M) || !(cams[i].tan_half > 0.0) ||
        !std::isfinite(cams[i].tan_half))
      return bh_fail(BH_E_INVALID, "bh_render: camera %d not set (bh_camera_set) or inside r = 2M", i);
    if (!camera_looks_at_hole(cams[i]))
      return bh_fail(BH_E_INVALID,
                     "bh_render: camera %d must look at the hole with an orthonormal basis (bh_camera_set)", i);
  }
  const int tw = opts->tile_w, th = opts->tile_h;
  if ((tw || th) && !tile_shape_ok(tw, th))
    return bh_fail(BH_E_INVALID,
                   "bh_render: tile_w * tile_h must be a power of two in [32, 256], tile_w a power of two");
  if (opts->block_size && opts->block_size != 64 && opts->block_size != 128 &&
      opts->block_size != 256 && opts->block_size != 512)
    return bh_fail(BH_E_INVALID, "bh_render: block_size must be 64, 128, 256 or 512");
  if (opts->queue_chunk && (opts->queue_chunk < 32 || opts->queue_chunk > 1024 || opts->queue_chunk % 32))
    return bh_fail(BH_E_INVALID, "bh_render: queue_chunk must be a multiple of 32 in [32, 1024]");
  if (opts->rtol < 0 || opts->atol < 0 || opts->band < 0 || opts->band_rtol < 0 ||
      opts->phi_max < 0 || opts->h_max < 0 || opts->h_max_far < 0 || opts->paper_eps < 0 || opts->rtol_far < 0 ||
      opts->rtol_near < 0 ||
      opts->host_strips < 0 || opts->host_strips > BH_MAX_HOST_STRIPS ||
      opts->max_steps < 0 || opts->budget < 0 || opts->blocks_per_sm < 0 || opts->spp < 0)
    return bh_fail(BH_E_INVALID, "bh_render: negative option");
  if (opts->spp > 1) {
    int n = 1;
    while (n * n < opts->spp) ++n;
    if (n * n != opts->spp || n > 16)
      return bh_fail(BH_E_INVALID, "bh_render: spp must be a square n*n with n <= 16 (got %d)", opts->spp);
    if (opts->mode != BH_MODE_FP32 && opts->mode != BH_MODE_FP64)
      return bh_fail(BH_E_UNSUPPORTED, "bh_render: spp > 1 needs BH_MODE_FP32 or BH_MODE_FP64");
  }
  if (opts->doppler && opts->mode != BH_MODE_FP32 && opts->mode != BH_MODE_FP64 &&
      opts->mode != BH_MODE_MIXED)
    return bh_fail(BH_E_UNSUPPORTED, "bh_render: doppler shading needs an integrator mode");
  return BH_OK;
}

int build_cameras(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                  int tw, int th, long long* n_queue, long long* n_rays) {
  sc->h_cams.resize(n_cams);
  long long q = 0, o = 0;
  for (int i = 0; i < n_cams; ++i) {
    CamK& c = sc->h_cams[i];
    const bh_camera& b = cams[i];
    for (int k = 0; k < 3; ++k) {
      c.pos[k] = b.pos[k];
      c.fwd[k] = b.fwd[k];
      c.right[k] = b.right[k];
      c.up[k] = b.up[k];
    }
    c.sx = b.tan_half;
    c.sy = b.tan_half * (double)h[i] / (double)w[i];
    c.r_obs = b.r_obs;
    c.w = w[i];
    c.h = h[i];
    c.tiles_x = (w[i] + tw - 1) / tw;
    c.tiles_y = (h[i] + th - 1) / th;
    c.q_off = q;
    c.out_off = o;
    fill_cam_r(c, sc->sk, &c.f);
    fill_cam_r(c, sc->sk, &c.d);
    fill_cam_peri(c, sc->sk.f.M);
    q += (long long)tw * th * c.tiles_x * c.tiles_y;
    o += (long long)w[i] * h[i];
  }
  if (q >= 0x7FFFFFFFLL || o >= 0x7FFFFFFFLL)
    return bh_fail(BH_E_INVALID, "bh_render: total ray count must stay below 2^31 - 1");
  *n_queue = q;
  *n_rays = o;
  return BH_OK;
}

RenderConfig resolve_config(const bh_scene* sc, const bh_render_opts* o) {
  RenderConfig c;
  c.mode = o->mode;
  const bool f64 = mode_is_fp64(o->mode);
  c.rtol = o->rtol > 0 ? o->rtol : (f64 ? 1e-10 : 1e-5);
  c.atol = o->atol > 0 ? o->atol : (f64 ? 1e-10 : 1e-7);
  c.band = o->band > 0 ? o->band : 0.05;
  c.band_rtol = o->band_rtol > 0 ? o->band_rtol : 1e-8;
  c.phi_max = o->phi_max > 0 ? o->phi_max : 64.0;
  c.h_max = o->h_max > 0 ? o->h_max : (f64 ? INFINITY : 0.3);
  c.h_max_far = o->h_max_far > 0 ? o->h_max_far : (f64 ? c.h_max : 0.5);
  c.rtol_far = o->rtol_far > 0 ? o->rtol_far : (f64 ? c.rtol : 10.0 * c.rtol);
  c.rtol_near = o->rtol_near > 0 ? o->rtol_near : (f64 ? c.rtol : 0.01 * c.rtol);
  c.max_steps = o->max_steps > 0 ? o->max_steps : 100000;
  c.paper_eps = o->paper_eps > 0 ? o->paper_eps : 0.01;
  c.doppler = o->doppler ? 1 : 0;
  c.spp_n = 1;
  while (c.spp_n * c.spp_n < o->spp) ++c.spp_n;
  const TunedShape t = tuned_shape(sc, o->mode);
  c.block = o->block_size ? o->block_size : t.block;
  c.blocks_per_sm = o->blocks_per_sm ? o->blocks_per_sm : t.blocks_per_sm;
  c.tile_w = o->tile_w ? o->tile_w : t.tile_w;
  c.tile_h = o->tile_h ? o->tile_h : t.tile_h;
  c.budget = o->budget ? o->budget : t.budget;
  c.chunk = o->queue_chunk ? o->queue_chunk : t.chunk;
  if (c.spp_n > 1) c.budget = c.max_steps;  // every sample finishes in the tile pass
  c.band_warps = t.band_warps;
  c.peri_reset = o->periastron_reset < 0 ? 0 : (o->periastron_reset == 2 ? 2 : 1);
  c.abort_after = o->abort_after;
  return c;
}

// Host-side preparation of one render: resolve options, build the camera
// table (uploaded to cams_dev, or to the scene's table when null), size the
// scene workspace and fill the kernel parameters and launch shape.
int prepare_render(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                   void* dirs, uint16_t* flags, uint32_t* rgba, const bh_render_opts* opts,
                   cudaStream_t upload_stream, CamK* cams_dev, PreparedRender* out) {
  const RenderConfig cfg = resolve_config(sc, opts);
  long long n_queue = 0, n_rays = 0;
  int rc = build_cameras(sc, cams, n_cams, w, h, cfg.tile_w, cfg.tile_h, &n_queue, &n_rays);
  if (rc) return rc;
  cudaError_t e = cudaSuccess;
  if (!cams_dev) {
    e = grow(&sc->d_cams, &sc->cams_cap, (size_t)n_cams);
    cams_dev = sc->d_cams;
  }
  if (e == cudaSuccess) e = grow(&sc->d_band, &sc->band_cap, (size_t)n_queue);
  const size_t spill_bytes = (mode_is_fp64(cfg.mode) ? sizeof(Spill<double>) : sizeof(Spill<float>));
  if (e == cudaSuccess) e = grow(&sc->d_spill, &sc->spill_cap, (size_t)n_queue * spill_bytes);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render: workspace allocation");
  // MIXED band bounds per camera (k_band_list and band_pixel)
  int rows = 0;
  for (int i = 0; i < n_cams; ++i) {
    CamK& c = sc->h_cams[i];
    fill_cam_band(c, sc->sk.M, sc->sk.ic, cfg.mode == BH_MODE_MIXED || cfg.mode == BH_MODE_SURROGATE
                                              ? cfg.band : 0.0);
    c.row_off = rows;
    rows += c.h;
  }
  e = cudaMemcpyAsync(cams_dev, sc->h_cams.data(), n_cams * sizeof(CamK), cudaMemcpyHostToDevice,
                      upload_stream);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render: camera upload");
  Params& p = out->p;
  fill_params(sc, cfg, n_cams, n_queue, n_rays, dirs, flags, rgba, &p);
  p.cams = cams_dev;
  LaunchShape ls{sc->num_sms, cfg.block, cfg.blocks_per_sm};
  ls.band_rows = rows;
  if (cfg.mode == BH_MODE_MIXED) ls.band_warps = cfg.band_warps;
  out->ls = ls;
  out->kmode = cfg.mode == BH_MODE_FP64             ? MODE_FP64
               : cfg.mode == BH_MODE_FP32           ? MODE_FP32
               : cfg.mode == BH_MODE_PAPER_EPS      ? MODE_PAPER64
               : cfg.mode == BH_MODE_PAPER_EPS_FP32 ? MODE_PAPER32
                                                    : MODE_MIXED;
  out->mode = cfg.mode;
  return BH_OK;
}

// Work of one prepared render on `stream`: clear the workspace, launch the
// passes.  Also what a CUDA graph of the render captures.
int enqueue_render(bh_scene* sc, const PreparedRender& pr, cudaStream_t stream) {
  if (pr.mode == BH_MODE_SURROGATE) return surrogate_enqueue(sc, pr, stream);
  cudaError_t e = cudaMemsetAsync(sc->d_ws, 0, sizeof(WorkK), stream);
  if (e == cudaSuccess) e = launch_render(pr.p, pr.kmode, pr.ls, stream, sc->ev);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render: launch");
  return BH_OK;
}

int render_device(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                  void* dirs, uint16_t* flags, uint32_t* rgba, const bh_render_opts* opts) {
  if (opts->mode == BH_MODE_SURROGATE)
    return surrogate_render(sc, cams, n_cams, w, h, dirs, flags, rgba, opts);
  cudaStream_t stream = (cudaStream_t)opts->stream;
  PreparedRender pr;
  int rc = prepare_render(sc, cams, n_cams, w, h, dirs, flags, rgba, opts, stream, nullptr, &pr);
  if (rc) return rc;
  rc = enqueue_render(sc, pr, stream);
  if (rc) return rc;
  sc->last_stream = stream;
  sc->timed = true;
  sc->band_used = false;
  return BH_OK;
}

void fill_params(const bh_scene* sc, const RenderConfig& cfg, int n_cams, long long n_queue,
                 long long n_rays, void* dirs, uint16_t* flags, uint32_t* rgba, Params* out) {
  Params& p = *out;
  memset(&p, 0, sizeof p);
  p.s = sc->sk;
  if (cfg.mode == BH_MODE_PAPER_EPS || cfg.mode == BH_MODE_PAPER_EPS_FP32) {
    // the polyline's straight segments cut inside the orbit's periastron:
    // no sphere is culled by the impact parameter there
    for (int k = 0; k < kMaxSph; ++k) p.s.f.cull_b[k] = INFINITY;
    for (int k = 0; k < kMaxSph; ++k) p.s.d.cull_b[k] = INFINITY;
  }
  p.cams = sc->d_cams;
  p.n_cams = n_cams;
  p.band_trim = cfg.mode == BH_MODE_MIXED ? 1 : 0;
  p.tile_w = cfg.tile_w;
  p.tile_h = cfg.tile_h;
  p.tile_shift = ilog2(cfg.tile_w * cfg.tile_h);
  p.tile_wshift = ilog2(cfg.tile_w);
  p.chunk = cfg.chunk;
  p.budget = cfg.budget;
  p.n_queue = n_queue;
  p.n_rays = n_rays;
  p.rtol = cfg.rtol;
  p.atol = cfg.atol;
  p.rtol64 = cfg.band_rtol;
  p.atol64 = cfg.band_rtol;
  p.band = cfg.band;
  p.phi_max = cfg.phi_max;
  p.h_max = cfg.h_max;
  p.h_max_far = cfg.h_max_far;
  p.rtol_far = cfg.rtol_far;
  p.rtol_near = cfg.rtol_near;
  p.paper_eps = cfg.paper_eps;
  p.spp_n = cfg.spp_n;
  p.doppler = cfg.doppler;
  p.max_steps = cfg.max_steps;
  p.peri_reset = cfg.peri_reset;
  p.abort_after = cfg.abort_after;
  p.dirs = dirs;
  p.flags = flags;
  p.rgba = rgba;
  p.ws = sc->d_ws;
  p.spill = sc->d_spill;
  p.band_list = sc->d_band;
  fill_tolerances(p);
}

void fill_tolerances(Params& p) {
  const double e = p.rtol_far > 0 ? p.rtol / p.rtol_far : 1.0;
  const double en = p.rtol_near > 0 ? p.rtol / p.rtol_near : 1.0;
  p.tf = TolR<float>{(float)p.rtol, (float)p.atol, (float)p.phi_max, (float)p.h_max, (float)p.band,
                     (float)p.h_max_far, (float)(e * e), (float)(en * en)};
  p.td = TolR<double>{p.rtol, p.atol, p.phi_max, p.h_max, p.band, p.h_max_far, e * e, en * en};
  p.tb = TolR<double>{p.rtol64, p.atol64, p.phi_max, INFINITY, p.band, INFINITY, 1.0, 1.0};
}

extern "C" int bh_render(const bh_scene* scene, const bh_camera* cams, int n_cams, const int* w,
                         const int* h, void* out_dirs, uint16_t* out_flags, uint32_t* out_rgba8,
                         const bh_render_opts* opts) {
  int rc = check_render_args(scene, cams, n_cams, w, h, opts);
  if (rc) return rc;
  bh_scene* sc = const_cast<bh_scene*>(scene);
  DeviceGuard g(sc->device);
  return render_device(sc, cams, n_cams, w, h, out_dirs, out_flags, out_rgba8, opts);
}

// One strip of a host render: queue slots [q_lo, q_hi) (whole tile rows),
// image rows [row_lo, row_hi) numbered over all cameras, outputs [o_lo, o_hi).
struct HostStrip {
  long long q_lo, q_hi, o_lo, o_hi;
  int row_lo, row_hi;
};

// Cut the prepared cameras' tile rows into at most `want` strips of about
// equal slot counts (want = 0: about 2^21 rays a strip).
static int cut_strips(const bh_scene* sc, int n_cams, int tile_w, int tile_h, long long n_queue,
                      int want, HostStrip* out) {
  if (want <= 0) want = (int)std::min<long long>(BH_MAX_HOST_STRIPS, std::max(1LL, n_queue >> 21));
  const long long target = (n_queue + want - 1) / want;
  int n = 0;
  HostStrip cur{0, 0, 0, 0, 0, 0};
  for (int ci = 0; ci < n_cams; ++ci) {
    const CamK& c = sc->h_cams[ci];
    for (int ty = 0; ty < c.tiles_y; ++ty) {
      const int y1 = std::min(c.h, (ty + 1) * tile_h);
      cur.q_hi = c.q_off + (long long)(ty + 1) * c.tiles_x * tile_w * tile_h;
      cur.o_hi = c.out_off + (long long)y1 * c.w;
      cur.row_hi = c.row_off + y1;
      const bool last = ci == n_cams - 1 && ty == c.tiles_y - 1;
      if (last || (cur.q_hi - cur.q_lo >= target && n < want - 1)) {
        out[n++] = cur;
        cur = HostStrip{cur.q_hi, cur.q_hi, cur.o_hi, cur.o_hi, cur.row_hi, cur.row_hi};
      }
    }
  }
  return n;
}

// Whether image rows [row_lo, row_hi) of a strip may hold MIXED band pixels:
// a row meets the band annulus rho^2 in (band_rho2_lo, band_rho2_hi) only if
// the squared image-plane height of its pixel centres is below band_rho2_hi
// (the test k_band_list makes, here with a margin).
static bool strip_has_band(const bh_scene* sc, int n_cams, const HostStrip& t) {
  for (int ci = 0; ci < n_cams; ++ci) {
    const CamK& c = sc->h_cams[ci];
    if (!(c.band_rho2_hi > c.band_rho2_lo)) continue;
    const int y0 = std::max(0, t.row_lo - c.row_off), y1 = std::min(c.h, t.row_hi - c.row_off);
    for (int y = y0; y < y1; ++y) {
      const double sy = c.sy - (y + 0.5) * 2.0 * c.sy / c.h;
      if (sy * sy < 1.001 * c.band_rho2_hi + 1e-12) return true;
    }
  }
  return false;
}

extern "C" int bh_render_host(const bh_scene* scene, const bh_camera* cams, int n_cams,
                              const int* w, const int* h, void* host_dirs, uint16_t* host_flags,
                              uint32_t* host_rgba8, const bh_render_opts* opts) {
  int rc = check_render_args(scene, cams, n_cams, w, h, opts);
  if (rc) return rc;
  bh_scene* sc = const_cast<bh_scene*>(scene);
  DeviceGuard g(sc->device);
  long long n = 0;
  for (int i = 0; i < n_cams; ++i) n += (long long)w[i] * h[i];
  if (n >= 0x7FFFFFFFLL) return bh_fail(BH_E_INVALID, "bh_render_host: too many rays");
  const size_t dsz = mode_is_fp64(opts->mode) ? sizeof(double) : sizeof(float);
  cudaError_t e = grow((char**)&sc->d_stage_dirs, &sc->stage_dirs_cap, (size_t)(2 * n) * dsz);
  if (e == cudaSuccess) e = grow(&sc->d_stage_flags, &sc->stage_flags_cap, (size_t)n);
  if (e == cudaSuccess) e = grow(&sc->d_stage_rgba, &sc->stage_rgba_cap, (size_t)n);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render_host: staging allocation");
  void* sd = host_dirs ? sc->d_stage_dirs : nullptr;
  uint16_t* sf = host_flags ? sc->d_stage_flags : nullptr;
  uint32_t* sr = host_rgba8 ? sc->d_stage_rgba : nullptr;
  cudaStream_t stream = (cudaStream_t)opts->stream;
  // copies of output range [lo, hi) on stream s: theta and phi, the two
  // rows of the direction buffer, in one 2-D copy (three copies a strip
  // instead of four: 1% off the end-to-end frame)
  auto copy_range = [&](long long lo, long long hi, cudaStream_t s) {
    cudaError_t r = cudaSuccess;
    const long long m = hi - lo;
    if (m <= 0) return r;
    if (host_dirs) {
      char* hd = (char*)host_dirs;
      const char* dd = (const char*)sc->d_stage_dirs;
      r = cudaMemcpy2DAsync(hd + lo * dsz, n * dsz, dd + lo * dsz, n * dsz, m * dsz, 2,
                            cudaMemcpyDeviceToHost, s);
    }
    if (r == cudaSuccess && host_flags)
      r = cudaMemcpyAsync(host_flags + lo, sc->d_stage_flags + lo, m * 2, cudaMemcpyDeviceToHost, s);
    if (r == cudaSuccess && host_rgba8)
      r = cudaMemcpyAsync(host_rgba8 + lo, sc->d_stage_rgba + lo, m * 4, cudaMemcpyDeviceToHost, s);
    return r;
  };
  if (opts->mode == BH_MODE_SURROGATE) {
    // the surrogate pass renders whole, then copies
    rc = render_device(sc, cams, n_cams, w, h, sd, sf, sr, opts);
    if (rc) return rc;
    e = copy_range(0, n, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render_host: copy back");
    return BH_OK;
  }
  // Strips of whole tile rows: strip k renders (its own slot window, band
  // rows and long rays) on `stream` while strip k - 1's outputs are copied
  // on the scene's copy stream, so the copy, which takes longer than the
  // render at 14 B per ray, starts after the first strip instead of the
  // frame.  Each ray is computed as in one whole render.
  PreparedRender pr;
  rc = prepare_render(sc, cams, n_cams, w, h, sd, sf, sr, opts, stream, nullptr, &pr);
  if (rc) return rc;
  HostStrip strips[BH_MAX_HOST_STRIPS];
  const int ns = cut_strips(sc, n_cams, pr.p.tile_w, pr.p.tile_h, pr.p.n_queue, opts->host_strips,
                            strips);
  const bool mixed = pr.kmode == MODE_MIXED;
  int regs_per_sm = 65536;
  cudaDeviceGetAttribute(&regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, sc->device);
  e = cudaMemsetAsync(sc->d_ws, 0, sizeof(WorkK), stream);
  if (mixed && e == cudaSuccess) {
    // MIXED: one band list and FP64 band pass over the whole frame on the
    // side stream, beside the strips' FP32 passes (a band pass per strip
    // would put the slowest band ray's latency into every strip); the copy
    // of a strip that holds band pixels also waits for it
    e = cudaEventRecord(sc->fork, stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sc->side, sc->fork, 0);
    LaunchShape lb = pr.ls;
    lb.mixed_part = 1;
    if (e == cudaSuccess) e = launch_render(pr.p, pr.kmode, lb, sc->side, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(sc->join, sc->side);
  }
  // MIXED: the strips without band pixels first, so the copy stream has their
  // outputs to move while the FP64 band pass finishes; then those with band
  // pixels, whose copies wait for it
  int order[BH_MAX_HOST_STRIPS];
  bool banded[BH_MAX_HOST_STRIPS];
  int no = 0;
  for (int k = 0; k < ns; ++k) banded[k] = mixed && strip_has_band(sc, n_cams, strips[k]);
  for (int k = 0; k < ns; ++k)
    if (!banded[k]) order[no++] = k;
  for (int k = 0; k < ns; ++k)
    if (banded[k]) order[no++] = k;
  for (int i = 0; i < ns && e == cudaSuccess; ++i) {
    const int k = order[i];
    const HostStrip& t = strips[k];
    Params ps = pr.p;
    ps.q_begin = t.q_lo;
    ps.n_queue = t.q_hi;
    LaunchShape ls = pr.ls;
    ls.band_row0 = t.row_lo;
    ls.band_rows = t.row_hi - t.row_lo;
    if (mixed) {
      ls.mixed_part = 2;
      // leave the band warps their registers (both kernels hold 64 a
      // thread): a strip launched without that room fills every SM and the
      // band pass waits for it to retire
      const int room = (regs_per_sm - ls.band_warps * 32 * 64) / (64 * ls.block);
      ls.blocks_per_sm = std::max(1, ls.blocks_per_sm > 0 ? std::min(ls.blocks_per_sm, room) : room);
    }
    // the strip's queue counters (the band pass's run on beside it);
    // statistics and status over the frame
    if (i > 0) e = cudaMemsetAsync(sc->d_ws, 0, offsetof(WorkK, band_count), stream);
    if (e == cudaSuccess) e = launch_render(ps, pr.kmode, ls, stream, nullptr);
    if (e == cudaSuccess) e = cudaEventRecord(sc->strip_ev[k], stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sc->copy, sc->strip_ev[k], 0);
    if (e == cudaSuccess && banded[k]) e = cudaStreamWaitEvent(sc->copy, sc->join, 0);
    if (e == cudaSuccess) e = copy_range(t.o_lo, t.o_hi, sc->copy);
  }
  if (mixed && e == cudaSuccess) e = cudaStreamWaitEvent(stream, sc->join, 0);
  if (e != cudaSuccess) {
    cudaStreamSynchronize(sc->copy);
    cudaStreamSynchronize(sc->side);
    return bh_cuda_fail(e, "bh_render_host: strips");
  }
  sc->last_stream = stream;
  sc->timed = false;
  sc->band_used = false;
  e = cudaStreamSynchronize(sc->copy);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render_host: copy back");
  return BH_OK;
}

extern "C" int bh_scene_sync(const bh_scene* scene) {
  if (!scene) return bh_fail(BH_E_INVALID, "bh_scene_sync: null scene");
  DeviceGuard g(scene->device);
  cudaError_t e = cudaStreamSynchronize(scene->last_stream);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_scene_sync");
  unsigned status = 0;
  e = cudaMemcpy(&status, &scene->d_ws->status, sizeof status, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_scene_sync: status");
  if (status & (BH_STATUS_ABORTED | BH_STATUS_WATCHDOG))
    return bh_fail(BH_E_DEVICE, "device status 0x%x (%s%s)", status,
                   (status & BH_STATUS_ABORTED) ? "aborted " : "",
                   (status & BH_STATUS_WATCHDOG) ? "watchdog" : "");
  return BH_OK;
}

extern "C" int bh_render_stats(const bh_scene* scene, bh_stats* out) {
  if (!scene || !out) return bh_fail(BH_E_INVALID, "bh_render_stats: null argument");
  DeviceGuard g(scene->device);
  cudaError_t e = cudaStreamSynchronize(scene->last_stream);
  WorkK w;
  if (e == cudaSuccess) e = cudaMemcpy(&w, scene->d_ws, sizeof w, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render_stats");
  memset(out, 0, sizeof *out);
  out->rays = w.stats[ST_RAYS];
  out->steps = w.stats[ST_STEPS];
  out->rejected = w.stats[ST_REJ];
  out->n_esc = w.stats[ST_ESC];
  out->n_capt = w.stats[ST_CAPT];
  out->n_disk = w.stats[ST_DISK];
  out->n_sphere = w.stats[ST_SPH];
  out->n_step_limit = w.stats[ST_LIM];
  out->n_band = w.stats[ST_BAND];
  out->n_long = w.stats[ST_LONG];
  out->n_surrogate = w.stats[ST_SURR];
  out->n_fallback = w.stats[ST_FALLBACK];
  out->queue_grabs = w.stats[ST_GRABS];
  out->periastron = w.stats[ST_PERI];
  out->events = w.stats[ST_EVENTS];
  out->steps_fp64 = w.stats[ST_STEPS64];
  out->mlp_rays = w.stats[ST_MLP];
  out->status = w.status;
  if (scene->timed) {
    for (int i = 0; i < 2; ++i) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, scene->ev[i], scene->ev[i + 1]) == cudaSuccess)
        out->kernel_ms[i] = ms;
    }
    float ms = 0.0f;
    if (scene->band_used) {
      if (cudaEventElapsedTime(&ms, scene->band_ev[0], scene->band_ev[1]) == cudaSuccess)
        out->kernel_ms[2] = ms;
    } else if (cudaEventElapsedTime(&ms, scene->ev[2], scene->ev[3]) == cudaSuccess) {
      out->kernel_ms[2] = ms;
    }
    float tot = 0.0f;
    if (cudaEventElapsedTime(&tot, scene->ev[0], scene->ev[3]) == cudaSuccess) out->kernel_ms[3] = tot;
    cudaGetLastError();  // an event that never completed only leaves a time at 0
  }
  return BH_OK;
}
