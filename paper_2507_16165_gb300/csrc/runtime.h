// Host runtime internals shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "bh.h"
#include "bh_types.cuh"
#include "render.h"

constexpr int kMaxCameras = 4096;

struct SurrogateState;  // trained MLP weights and calibration (surrogate.cu)

// Opaque scene of the C-ABI.
struct bh_scene {
  bh_scene_desc desc;
  bhk::SceneK sk;
  int device = 0;
  int num_sms = 1;
  bhk::WorkK* d_ws = nullptr;
  bhk::CamK* d_cams = nullptr;
  size_t cams_cap = 0;
  std::vector<bhk::CamK> h_cams;
  char* d_spill = nullptr;  // bytes
  size_t spill_cap = 0;
  int* d_band = nullptr;
  size_t band_cap = 0;
  void* d_stage_dirs = nullptr;  // bh_render_host staging
  size_t stage_dirs_cap = 0;
  uint16_t* d_stage_flags = nullptr;
  size_t stage_flags_cap = 0;
  uint32_t* d_stage_rgba = nullptr;
  size_t stage_rgba_cap = 0;
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t band_ev[2] = {nullptr, nullptr};
  cudaStream_t side = nullptr;               // FP64 band pass (MIXED)
  cudaEvent_t fork = nullptr, join = nullptr;
  bool timed = false;
  bool band_used = false;  // last render ran the side-stream band pass
  SurrogateState* surr = nullptr;
  uint32_t* d_sky = nullptr;  // sky image texels (bh_scene_sky_texture)
  float4* d_sky_lut = nullptr;  // checker cell colours (SceneK::sky_lut)
  cudaStream_t copy = nullptr;  // bh_render_host: copies of finished strips
  cudaEvent_t strip_ev[BH_MAX_HOST_STRIPS] = {};
};

// Resolved options of one render.
struct RenderConfig {
  int mode;
  double rtol, atol, band, band_rtol, phi_max, h_max, h_max_far, rtol_far, rtol_near, paper_eps;
  int spp_n;  // samples per pixel side
  int doppler;
  int max_steps;
  int block, blocks_per_sm, tile_w, tile_h, budget, chunk;
  int band_warps;
  int peri_reset;
  unsigned long long abort_after;
};

// Launch shape picked by the autotuner (or the built-in default).
struct TunedShape {
  int block, blocks_per_sm, tile_w, tile_h, budget;
  int chunk;  // queue slots per warp grab
  int band_warps;  // FP64 band pass: warps per SM launched (see k_longrays)
};

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev);
  ~DeviceGuard();

 private:
  int prev_ = 0, dev_ = 0;
};

int bh_fail(int code, const char* fmt, ...);
// A camera the kernels can render: it looks at the hole (fwd = -pos / r_obs)
// with right and up an orthonormal image basis perpendicular to fwd, as
// bh_camera_set makes it.
bool camera_looks_at_hole(const bh_camera& c);
int bh_cuda_fail(cudaError_t e, const char* what);
int check_render_args(const bh_scene* sc, const bh_camera* cams, int n_cams, const int* w,
                      const int* h, const bh_render_opts* opts);
int build_cameras(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                  int tw, int th, long long* n_queue, long long* n_rays);
RenderConfig resolve_config(const bh_scene* sc, const bh_render_opts* o);
// Modes whose directions are stored as double.
inline bool mode_is_fp64(int mode) { return mode == BH_MODE_FP64 || mode == BH_MODE_PAPER_EPS; }
void fill_params(const bh_scene* sc, const RenderConfig& cfg, int n_cams, long long n_queue,
                 long long n_rays, void* dirs, uint16_t* flags, uint32_t* rgba, bhk::Params* out);
void fill_tolerances(bhk::Params& p);

// A render prepared on the host: kernel parameters and launch shape.
struct PreparedRender {
  bhk::Params p;
  bhk::LaunchShape ls;
  int kmode;  // bhk::Mode of the main pass
  int mode;   // BH_MODE_*
};
int prepare_render(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                   void* dirs, uint16_t* flags, uint32_t* rgba, const bh_render_opts* opts,
                   cudaStream_t upload_stream, bhk::CamK* cams_dev, PreparedRender* out);
int enqueue_render(bh_scene* sc, const PreparedRender& pr, cudaStream_t stream);
int render_device(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                  void* dirs, uint16_t* flags, uint32_t* rgba, const bh_render_opts* opts);

// autotune.cu
TunedShape tuned_shape(const bh_scene* sc, int mode);

// surrogate.cu
int surrogate_prepare(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                      void* dirs, uint16_t* flags, uint32_t* rgba, const bh_render_opts* opts,
                      cudaStream_t upload_stream, bhk::CamK* cams_dev, PreparedRender* pr);
int surrogate_enqueue(bh_scene* sc, const PreparedRender& pr, cudaStream_t stream);
int surrogate_render(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                     void* dirs, uint16_t* flags, uint32_t* rgba, const bh_render_opts* opts);
void surrogate_release(bh_scene* sc);
