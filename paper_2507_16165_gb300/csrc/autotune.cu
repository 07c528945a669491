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
  // chunks of 64 (FP32) and 128 (MIXED) slots measured 2-3% faster than
  // 32 at 4096^2; the FP32 budget leaves the rays of the near-critical
  // tolerance tier (up to about 100 steps) in the tile pass
  t.chunk = mode == BH_MODE_FP32 ? 64 : (mode == BH_MODE_MIXED ? 128 : 32);
  t.budget = mode == BH_MODE_FP64 ? 256 : (mode == BH_MODE_FP32 ? 128 : 48);
  // MIXED: 128-thread blocks, eight per SM (the full register file at 64
  // registers); seven fit beside the FP64 band pass's four warps per SM and
  // the eighth starts as they leave
  if (mode == BH_MODE_MIXED) {
    t.block = 128;
    t.blocks_per_sm = 8;
  }
  t.band_warps = 4;
  return t;
}

}  // namespace

TunedShape tuned_shape(const bh_scene* sc, int mode) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tuned.find({sc->device, mode});
  return it != g_tuned.end() ? it->second : default_shape(mode);
}

// Staged sweep, each stage keeping the best shape so far:
//   1. block size (with the resident blocks per SM) x tile shape
//      {8x4, 4x8, 8x8, 16x16}, at the default queue chunk and step budget;
//   2. queue chunk in {32, 64, ..., 1024} slots per warp grab;
//   3. step budget of the coherent pass.
// The surrogate pass has a fixed block (its shared-memory staging is sized
// for four warps), so only its tile, chunk and budget are swept.
extern "C" int bh_autotune(bh_scene* scene, const bh_camera* cams, int n_cams, const int* w,
                           const int* h, void* out_dirs, uint16_t* out_flags, uint32_t* out_rgba8,
                           const bh_render_opts* opts, bh_tune_result* result) {
  int rc = check_render_args(scene, cams, n_cams, w, h, opts);
  if (rc) return rc;
  if (!result) return bh_fail(BH_E_INVALID, "bh_autotune: null result");
  const int mode = opts->mode;
  if (mode != BH_MODE_FP64 && mode != BH_MODE_FP32 && mode != BH_MODE_MIXED &&
      mode != BH_MODE_SURROGATE)
    return bh_fail(BH_E_UNSUPPORTED, "bh_autotune: FP64, FP32, MIXED and SURROGATE modes only");
  if (opts->spp > 1)
    return bh_fail(BH_E_UNSUPPORTED, "bh_autotune: one sample per pixel");
  DeviceGuard g(scene->device);
  cudaStream_t stream = (cudaStream_t)opts->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t ce = cudaEventCreate(&e0);
  if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) return bh_cuda_fail(ce, "bh_autotune: events");

  int trials = 0;
  auto time_shape = [&](const TunedShape& s, float* best) -> int {
    bh_render_opts o = *opts;
    o.block_size = s.block;
    o.blocks_per_sm = s.blocks_per_sm;
    o.tile_w = s.tile_w;
    o.tile_h = s.tile_h;
    o.queue_chunk = s.chunk;
    o.budget = s.budget;
    *best = 1e30f;
    ++trials;
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
  const TunedShape def = default_shape(mode);
  float ms_default = 0.0f;
  rc = time_shape(def, &ms_default);
  TunedShape best_s = def;
  float best_ms = ms_default;
  auto consider = [&](const TunedShape& s) {
    if (rc) return;
    float ms = 0.0f;
    rc = time_shape(s, &ms);
    if (!rc && ms < best_ms) {
      best_ms = ms;
      best_s = s;
    }
  };
  // stage 1: (block, resident blocks per SM; 0 = as many as fit) x tile
  const int tiles[4][2] = {{8, 4}, {4, 8}, {8, 8}, {16, 16}};
  std::vector<std::pair<int, int>> res;
  if (mode == BH_MODE_MIXED)
    res = {{128, 8}, {128, 7}, {256, 4}, {512, 2}};
  else if (mode == BH_MODE_SURROGATE)
    res = {{def.block, def.blocks_per_sm}};
  else
    res = {{128, 0}, {256, 0}, {512, 0}};
  for (const auto& rb : res)
    for (const auto& t : tiles) {
      TunedShape s = def;
      s.block = rb.first;
      s.blocks_per_sm = rb.second;
      s.tile_w = t[0];
      s.tile_h = t[1];
      if (s.block == def.block && s.blocks_per_sm == def.blocks_per_sm && s.tile_w == def.tile_w &&
          s.tile_h == def.tile_h)
        continue;  // timed above
      consider(s);
    }
  // stage 2: queue chunk
  {
    const TunedShape base = best_s;
    for (int c = 64; c <= 1024; c *= 2) {
      TunedShape s = base;
      s.chunk = c;
      consider(s);
    }
  }
  // stage 3: step budget of the coherent pass
  {
    const TunedShape base = best_s;
    const int b32[2] = {48, 256}, b64[2] = {128, 512};
    for (int i = 0; i < 2; ++i) {
      TunedShape s = base;
      s.budget = mode == BH_MODE_FP64 ? b64[i] : b32[i];
      consider(s);
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
  result->queue_chunk = best_s.chunk;
  result->ms_best = best_ms;
  result->ms_default = ms_default;
  result->trials = trials;
  return BH_OK;
}

extern "C" int bh_autotune_reset(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned.clear();
  return BH_OK;
}
