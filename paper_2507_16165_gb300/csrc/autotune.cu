// Launch-shape autotuner: times candidate shapes on the caller's workload
// and keeps the fastest per (device, mode) for later renders that leave the
// shape fields of bh_render_opts at 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "runtime.h"

namespace {

std::mutex g_tune_mu;
std::map<std::pair<int, int>, TunedShape> g_tuned;  // (device, mode) -> shape

TunedShape default_shape(int mode) {
  TunedShape t;
  t.block = 256;
  t.blocks_per_sm = 0;
  t.tile_w = 8;
  t.tile_h = 4;
  t.budget = (mode == BH_MODE_FP64) ? 256 : 48;
  // MIXED: 128-thread blocks, eight per SM (the full register file at 64
  // registers); seven fit beside the FP64 band pass's four warps per SM and
  // the eighth starts as they leave
  if (mode == BH_MODE_MIXED) {
    t.block = 128;
    t.blocks_per_sm = 8;
  }
  t.band_lanes = 32;
  t.band_warps = 4;
  return t;
}

}  // namespace

TunedShape tuned_shape(const bh_scene* sc, int mode) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find({sc->device, mode});
  return it != g_tuned.end() ? it->second : default_shape(mode);
}

extern "C" int bh_autotune(bh_scene* scene, const bh_camera* cams, int n_cams, const int* w,
                           const int* h, void* out_dirs, uint16_t* out_flags, uint32_t* out_rgba8,
                           const bh_render_opts* opts, bh_tune_result* result) {
  int rc = check_render_args(scene, cams, n_cams, w, h, opts);
  if (rc) return rc;
  if (!result) return bh_fail(BH_E_INVALID, "bh_autotune: null result");
  if (opts->mode == BH_MODE_SURROGATE)
    return bh_fail(BH_E_UNSUPPORTED, "bh_autotune: tune the integrator modes");
  DeviceGuard g(scene->device);
  const int mode = opts->mode;
  cudaStream_t stream = (cudaStream_t)opts->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) return bh_cuda_fail(ce, "bh_autotune: events");

  std::vector<TunedShape> cands;
  const int tiles[3][2] = {{8, 4}, {4, 8}, {16, 2}};
  const int budgets32[2] = {32, 64}, budgets64[2] = {128, 256};
  // (block size, resident blocks per SM; 0 = as many as fit)
  const int res_mixed[3][2] = {{128, 8}, {128, 7}, {256, 4}};
  const int res_other[2][2] = {{128, 0}, {256, 0}};
  const bool mixed = mode == BH_MODE_MIXED;
  const int n_res = mixed ? 3 : 2;
  for (int ri = 0; ri < n_res; ++ri)
    for (auto& t : tiles)
      for (int bi = 0; bi < 2; ++bi) {
        TunedShape s = default_shape(mode);
        s.block = mixed ? res_mixed[ri][0] : res_other[ri][0];
        s.blocks_per_sm = mixed ? res_mixed[ri][1] : res_other[ri][1];
        s.tile_w = t[0];
        s.tile_h = t[1];
        s.budget = mode == BH_MODE_FP64 ? budgets64[bi] : budgets32[bi];
        cands.push_back(s);
      }
  auto time_shape = [&](const TunedShape& s, float* best) -> int {
    bh_render_opts o = *opts;
    o.block_size = s.block;
    o.blocks_per_sm = s.blocks_per_sm;
    o.tile_w = s.tile_w;
    o.tile_h = s.tile_h;
    o.budget = s.budget;
    *best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, stream);
      int r = render_device(scene, cams, n_cams, w, h, out_dirs, out_flags, out_rgba8, &o);
      if (r) return r;
      cudaEventRecord(e1, stream);
      cudaError_t err = cudaEventSynchronize(e1);
      if (err != cudaSuccess) return bh_cuda_fail(err, "bh_autotune: render");
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) *best = std::min(*best, ms);  // the first run warms up
    }
    return BH_OK;
  };
  float ms_default = 0.0f;
  rc = time_shape(default_shape(mode), &ms_default);
  TunedShape best_s = default_shape(mode);
  float best_ms = ms_default;
  for (const TunedShape& s : cands) {
    if (rc) break;
    float ms = 0.0f;
    rc = time_shape(s, &ms);
    if (!rc && ms < best_ms) {
      best_ms = ms;
      best_s = s;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[{scene->device, mode}] = best_s;
  }
  memset(result, 0, sizeof *result);
  result->block_size = best_s.block;
  result->blocks_per_sm = best_s.blocks_per_sm;
  result->tile_w = best_s.tile_w;
  result->tile_h = best_s.tile_h;
  result->budget = best_s.budget;
  result->ms_best = best_ms;
  result->ms_default = ms_default;
  result->trials = (int)cands.size() + 1;
  return BH_OK;
}

extern "C" int bh_autotune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned.clear();
  return BH_OK;
}
