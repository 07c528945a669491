// A render captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include "runtime.h"

using namespace bhk;

struct bh_graph {
  bh_scene* scene = nullptr;
  CamK* d_cams = nullptr;  // the graph's own camera table
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int mode = 0;
};

extern "C" void bh_graph_destroy(bh_graph* g) {
  if (!g) return;
  {
    DeviceGuard dg(g->scene ? g->scene->device : 0);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->d_cams) cudaFree(g->d_cams);
  }
  delete g;
}

extern "C" int bh_graph_create(bh_scene* scene, const bh_camera* cams, int n_cams, const int* w,
                               const int* h, void* out_dirs, uint16_t* out_flags,
                               uint32_t* out_rgba8, const bh_render_opts* opts, bh_graph** out) {
  if (!out) return bh_fail(BH_E_INVALID, "bh_graph_create: null output");
  *out = nullptr;
  int rc = check_render_args(scene, cams, n_cams, w, h, opts);
  if (rc) return rc;
  DeviceGuard dg(scene->device);
  bh_graph* g = new (std::nothrow) bh_graph();
  if (!g) return bh_fail(BH_E_NOMEM, "bh_graph_create: host allocation");
  g->scene = scene;
  g->mode = opts->mode;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaMalloc((void**)&g->d_cams, n_cams * sizeof(CamK));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    bh_graph_destroy(g);
    return bh_cuda_fail(e, "bh_graph_create: setup");
  }
  PreparedRender pr;
  rc = opts->mode == BH_MODE_SURROGATE
           ? surrogate_prepare(scene, cams, n_cams, w, h, out_dirs, out_flags, out_rgba8, opts, cs,
                               g->d_cams, &pr)
           : prepare_render(scene, cams, n_cams, w, h, out_dirs, out_flags, out_rgba8, opts, cs,
                            g->d_cams, &pr);
  if (!rc) {
    e = cudaStreamSynchronize(cs);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = bh_cuda_fail(e, "bh_graph_create: begin capture");
  }
  if (!rc) {
    const int erc = enqueue_render(scene, pr, cs);
    e = cudaStreamEndCapture(cs, &g->graph);
    if (erc) rc = erc;
    else if (e != cudaSuccess) rc = bh_cuda_fail(e, "bh_graph_create: end capture");
  }
  if (!rc) {
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) rc = bh_cuda_fail(e, "bh_graph_create: instantiate");
  }
  cudaStreamDestroy(cs);
  if (rc) {
    bh_graph_destroy(g);
    return rc;
  }
  *out = g;
  return BH_OK;
}

extern "C" int bh_graph_launch(bh_graph* g, void* stream) {
  if (!g || !g->exec) return bh_fail(BH_E_INVALID, "bh_graph_launch: null graph");
  DeviceGuard dg(g->scene->device);
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return bh_cuda_fail(e, "bh_graph_launch");
  g->scene->last_stream = (cudaStream_t)stream;
  g->scene->timed = true;
  // the surrogate's FP64 band pass runs on the scene's side stream, timed
  // by its own events
  g->scene->band_used = g->mode == BH_MODE_SURROGATE;
  return BH_OK;
}
