// MLP surrogate (not yet trained in this build).
#include "runtime.h"

int surrogate_render(bh_scene* sc, const bh_camera* cams, int n_cams, const int* w, const int* h,
                     void* dirs, uint16_t* flags, uint32_t* rgba, const bh_render_opts* opts,
                     const RenderConfig& cfg) {
  (void)sc; (void)cams; (void)n_cams; (void)w; (void)h; (void)dirs; (void)flags; (void)rgba;
  (void)opts; (void)cfg;
  return bh_fail(BH_E_NO_SURROGATE, "surrogate mode: no trained weights on this scene");
}

void surrogate_release(bh_scene* sc) { (void)sc; }
