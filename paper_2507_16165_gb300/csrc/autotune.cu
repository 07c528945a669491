// Launch-shape selection.
#include "runtime.h"

TunedShape tuned_shape(const bh_scene* sc, int mode) {
  (void)sc;
  TunedShape t;
  t.block = 256;
  t.blocks_per_sm = 0;
  t.tile_w = 8;
  t.tile_h = 4;
  t.budget = (mode == BH_MODE_FP64) ? 256 : 48;
  return t;
}
