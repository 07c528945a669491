// bh_render_noalloc: a render entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: hosts that hand all device memory to
// their own pool or fixed budget and forbid other allocations, and real-time
// loops where an allocation may synchronise the device or fail mid-frame.
// This entry point keeps the only scratch the coherent render pass needs --
// the work-queue counter, status and statistics words, and the camera table
// -- in one file-scope __device__ array of fixed size, and runs the coherent
// pass alone with a step budget equal to the step cap, so no long-ray or
// band list is needed.  The caller passes the scene description, cameras and
// output buffers.  The camera table reaches the scratch array through the
// launch parameters of a small copy kernel, so no device work of the call
// reads host memory after the call has returned.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "bh.h"
#include "render.h"
#include "runtime.h"

using namespace bhk;

namespace {

constexpr int kNoAllocMaxCams = BH_NOALLOC_MAX_CAMERAS;
constexpr size_t kWorkBytes = (sizeof(WorkK) + 255) & ~size_t(255);
constexpr size_t kScratchBytes = kWorkBytes + kNoAllocMaxCams * sizeof(CamK);
constexpr int kMaxDevices = 64;

// The scratch: one copy per device that loads the library, kept until exit.
// Its name in host code is only a stand-in; kernels get the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Cameras per launch of the copy kernel: 16 camera records (about 6.5 KB)
// travel in its parameter block.
constexpr int kCamsPerCopy = 16;
struct CamChunk {
  CamK c[kCamsPerCopy];
  int n;
};

static_assert(sizeof(CamChunk) <= 32000, "camera chunk must fit a kernel's parameter block");

__global__ void k_noalloc_cams(const __grid_constant__ CamChunk src, CamK* dst) {
  for (int i = threadIdx.x; i < src.n; i += blockDim.x) dst[i] = src.c[i];
}

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Once per device, with that device current: look up the scratch address
// and the SM count.
int noalloc_setup(int dev, unsigned char** scratch, int* num_sms) {
  if (dev < 0 || dev >= kMaxDevices)
    return bh_fail(BH_E_UNSUPPORTED, "bh_render_noalloc: device index %d >= %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render_noalloc: cudaGetSymbolAddress");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render_noalloc: device attribute");
    g_num_sms[dev] = sms;
    g_scratch_addr[dev] = ptr;
  }
  *scratch = static_cast<unsigned char*>(g_scratch_addr[dev]);
  *num_sms = g_num_sms[dev];
  return BH_OK;
}

// Scene constants from a description, with the same checks as bh_scene_create.
int noalloc_scene(const bh_scene_desc* d, SceneK* k) {
  const double M = d->mass;
  if (!(M >= 0.0) || !std::isfinite(M)) return bh_fail(BH_E_INVALID, "mass must be >= 0");
  if (d->disk_enabled &&
      !(d->disk_r_in > 2.0 * M && d->disk_r_out > d->disk_r_in && std::isfinite(d->disk_r_out)))
    return bh_fail(BH_E_INVALID, "disk needs 2M < r_in < r_out");
  if (d->n_spheres < 0 || d->n_spheres > BH_MAX_SPHERES)
    return bh_fail(BH_E_INVALID, "n_spheres must be in [0, %d]", BH_MAX_SPHERES);
  if (d->ic != BH_IC_STATIC && d->ic != BH_IC_EUCLIDEAN)
    return bh_fail(BH_E_INVALID, "ic must be BH_IC_STATIC or BH_IC_EUCLIDEAN");
  memset(k, 0, sizeof *k);
  double r_min_obj = d->disk_enabled ? d->disk_r_in : INFINITY;
  for (int i = 0; i < d->n_spheres; ++i) {
    const bh_sphere& s = d->spheres[i];
    double c2 = 0.0;
    for (int j = 0; j < 3; ++j) {
      k->c[i][j] = s.center[j];
      c2 += s.center[j] * s.center[j];
      if (!(s.albedo[j] >= 0.0 && s.albedo[j] <= 1.0))
        return bh_fail(BH_E_INVALID, "sphere %d albedo must be in [0, 1]", i);
      k->alb[i][j] = (float)s.albedo[j];
    }
    const double c = std::sqrt(c2);
    if (!(s.radius > 0.0) || !(c - s.radius > 2.0 * M) || !std::isfinite(c))
      return bh_fail(BH_E_INVALID, "sphere %d must have radius > 0 and lie outside r = 2M", i);
    k->c2[i] = c2;
    k->R[i] = s.radius;
    k->K[i] = c2 - s.radius * s.radius;
    r_min_obj = std::fmin(r_min_obj, c - s.radius);
  }
  k->M = M;
  k->M3 = 3.0 * M;
  k->u_capt = (M > 0.0) ? (r_min_obj > 3.0 * M ? 1.0 / (3.0 * M) : 1.0 / (2.0 * M)) : INFINITY;
  k->b_crit = 3.0 * std::sqrt(3.0) * M;
  k->disk_on = d->disk_enabled ? 1 : 0;
  k->r_in = d->disk_r_in;
  k->r_out = d->disk_r_out;
  k->n_sph = d->n_spheres;
  k->seed = d->sky_seed;
  k->ic = d->ic;
  fill_scene_r(*k, &k->f);
  fill_scene_r(*k, &k->d);
  return BH_OK;
}

}  // namespace

extern "C" int bh_render_noalloc(const bh_scene_desc* desc, const bh_camera* cams, int n_cams,
                                 const int* w, const int* h, void* out_dirs, uint16_t* out_flags,
                                 uint32_t* out_rgba8, const bh_render_opts* opts) {
  if (!desc || !cams || !w || !h || !opts)
    return bh_fail(BH_E_INVALID, "bh_render_noalloc: null argument");
  if (n_cams < 1 || n_cams > kNoAllocMaxCams)
    return bh_fail(BH_E_INVALID, "bh_render_noalloc: n_cams must be in [1, %d] (scratch holds %d cameras)",
                   kNoAllocMaxCams, kNoAllocMaxCams);
  if (opts->mode != BH_MODE_FP32 && opts->mode != BH_MODE_FP64)
    return bh_fail(BH_E_UNSUPPORTED, "bh_render_noalloc: only BH_MODE_FP32 and BH_MODE_FP64");
  if (opts->spp > 1 || opts->doppler)
    return bh_fail(BH_E_UNSUPPORTED, "bh_render_noalloc: one sample per pixel, plain disk shading only");
  if (opts->abort_after)
    return bh_fail(BH_E_UNSUPPORTED,
                   "bh_render_noalloc: abort_after is not available (no status is read back)");
  if ((opts->tile_w || opts->tile_h) && !tile_shape_ok(opts->tile_w, opts->tile_h))
    return bh_fail(BH_E_INVALID,
                   "bh_render_noalloc: tile_w * tile_h must be a power of two in [32, 256], tile_w a power of two");
  if (opts->block_size && opts->block_size != 64 && opts->block_size != 128 &&
      opts->block_size != 256 && opts->block_size != 512)
    return bh_fail(BH_E_INVALID, "bh_render_noalloc: block_size must be 64, 128, 256 or 512");
  if (opts->queue_chunk && (opts->queue_chunk < 32 || opts->queue_chunk > 1024 || opts->queue_chunk % 32))
    return bh_fail(BH_E_INVALID, "bh_render_noalloc: queue_chunk must be a multiple of 32 in [32, 1024]");
  if (opts->rtol < 0 || opts->atol < 0 || opts->phi_max < 0 || opts->h_max < 0 || opts->h_max_far < 0 || opts->rtol_far < 0 ||
      opts->rtol_near < 0 || opts->band < 0 || opts->max_steps < 0 || opts->blocks_per_sm < 0)
    return bh_fail(BH_E_INVALID, "bh_render_noalloc: negative option");
  SceneK sk;
  int rc = noalloc_scene(desc, &sk);
  if (rc) return rc;
  const bool f64 = opts->mode == BH_MODE_FP64;
  const int tw = opts->tile_w ? opts->tile_w : 8, th = opts->tile_h ? opts->tile_h : 4;
  CamK hc[kNoAllocMaxCams];
  long long q = 0, o = 0;
  for (int i = 0; i < n_cams; ++i) {
    if (w[i] < 1 || h[i] < 1 || w[i] > 65536 || h[i] > 65536)
      return bh_fail(BH_E_INVALID, "bh_render_noalloc: camera %d size %dx%d out of range", i, w[i], h[i]);
    const bh_camera& b = cams[i];
    if (!(b.r_obs > 2.0 * sk.M) || !(b.tan_half > 0.0) || !std::isfinite(b.tan_half))
      return bh_fail(BH_E_INVALID, "bh_render_noalloc: camera %d not set or inside r = 2M", i);
    if (!camera_looks_at_hole(b))
      return bh_fail(BH_E_INVALID,
                     "bh_render_noalloc: camera %d must look at the hole with an orthonormal basis", i);
    CamK& c = hc[i];
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
    fill_cam_r(c, sk, &c.f);
    fill_cam_r(c, sk, &c.d);
    fill_cam_peri(c, sk.f.M);
    fill_cam_band(c, sk.M, sk.ic, 0.0);  // no band pass here
    c.row_off = 0;
    q += (long long)tw * th * c.tiles_x * c.tiles_y;
    o += (long long)w[i] * h[i];
  }
  if (q >= 0x7FFFFFFFLL || o >= 0x7FFFFFFFLL)
    return bh_fail(BH_E_INVALID, "bh_render_noalloc: total ray count must stay below 2^31 - 1");

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render_noalloc: cudaGetDevice");
  unsigned char* scratch = nullptr;
  int num_sms = 0;
  rc = noalloc_setup(dev, &scratch, &num_sms);
  if (rc) return rc;
  WorkK* ws = reinterpret_cast<WorkK*>(scratch);
  CamK* dcams = reinterpret_cast<CamK*>(scratch + kWorkBytes);
  cudaStream_t stream = (cudaStream_t)opts->stream;
  // the scratch keeps the previous call's contents: clear the counters
  e = cudaMemsetAsync(ws, 0, sizeof(WorkK), stream);
  for (int i0 = 0; i0 < n_cams && e == cudaSuccess; i0 += kCamsPerCopy) {
    CamChunk chunk;
    memset(&chunk, 0, sizeof chunk);
    chunk.n = std::min(kCamsPerCopy, n_cams - i0);
    for (int i = 0; i < chunk.n; ++i) chunk.c[i] = hc[i0 + i];
    k_noalloc_cams<<<1, 32, 0, stream>>>(chunk, dcams + i0);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render_noalloc: upload");

  Params p;
  memset(&p, 0, sizeof p);
  p.s = sk;
  p.cams = dcams;
  p.n_cams = n_cams;
  p.tile_w = tw;
  p.tile_h = th;
  p.tile_shift = ilog2(tw * th);
  p.tile_wshift = ilog2(tw);
  p.chunk = opts->queue_chunk ? opts->queue_chunk : 32;
  p.n_queue = q;
  p.n_rays = o;
  p.rtol = opts->rtol > 0 ? opts->rtol : (f64 ? 1e-10 : 1e-5);
  p.atol = opts->atol > 0 ? opts->atol : (f64 ? 1e-10 : 1e-7);
  p.rtol64 = 1e-10;
  p.atol64 = 1e-10;
  p.band = opts->band > 0 ? opts->band : 0.05;  // FP32: the rtol_near rays
  p.phi_max = opts->phi_max > 0 ? opts->phi_max : 64.0;
  p.h_max = opts->h_max > 0 ? opts->h_max : (f64 ? INFINITY : 0.3);
  p.h_max_far = opts->h_max_far > 0 ? opts->h_max_far : (f64 ? p.h_max : 0.5);
  p.rtol_far = opts->rtol_far > 0 ? opts->rtol_far : (f64 ? p.rtol : 10.0 * p.rtol);
  p.rtol_near = opts->rtol_near > 0 ? opts->rtol_near : (f64 ? p.rtol : 0.01 * p.rtol);
  p.max_steps = opts->max_steps > 0 ? opts->max_steps : 100000;
  p.budget = p.max_steps;  // every ray finishes in the coherent pass
  p.peri_reset = 0;
  p.abort_after = 0;
  p.dirs = out_dirs;
  p.flags = out_flags;
  p.rgba = out_rgba8;
  p.ws = ws;
  p.spill = nullptr;
  p.band_list = nullptr;
  fill_tolerances(p);
  LaunchShape ls{num_sms, opts->block_size ? opts->block_size : 256, opts->blocks_per_sm};
  e = launch_coherent_only(p, f64 ? MODE_FP64 : MODE_FP32, ls, stream);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_render_noalloc: launch");
  return BH_OK;
}
