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
  // MIXED: leave room on every SM for the band pass that runs alongside
  if (mode == BH_MODE_MIXED) t.blocks_per_sm = 3;
  t.band_lanes = 32;
  t.band_warps = 4;
  return t;
}
