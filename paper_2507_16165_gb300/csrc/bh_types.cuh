// Plain-data types shared by the host runtime and the kernels.
#pragma once

#include <stdint.h>

#include "bh.h"

namespace bhk {

constexpr int kMaxSph = BH_MAX_SPHERES;

// Scene constants, passed by value in every kernel's parameter block.
struct SceneK {
  double M, M3;        // mass and 3M
  double u_capt;       // capture threshold on u: 1/(3M) when every object lies
                       // outside r = 3M (early-out inside the photon sphere), else 1/(2M)
  double b_crit;       // 3 sqrt(3) M
  int disk_on;
  double r_in, r_out;
  int n_sph;
  double c[kMaxSph][3];
  double c2[kMaxSph];  // |c|^2
  double R[kMaxSph];
  double K[kMaxSph];   // |c|^2 - R^2
  float alb[kMaxSph][3];
  unsigned long long seed;
  int ic;
};

// One camera in device memory.  Its rays occupy queue slots
// [q_off, q_off + tiles_x * tiles_y * 32): one 32-ray tile per warp grab,
// padded where w or h is not a multiple of the tile.
struct CamK {
  double pos[3], fwd[3], right[3], up[3];
  double sx, sy;       // tan(fov/2) and tan(fov/2) * h / w
  double r_obs;
  int w, h, tiles_x, tiles_y;
  long long q_off, out_off;
};

enum StatId {
  ST_RAYS, ST_STEPS, ST_REJ, ST_ESC, ST_CAPT, ST_DISK, ST_SPH, ST_LIM, ST_BAND, ST_LONG,
  ST_SURR, ST_FALLBACK, ST_GRABS, ST_PERI, ST_EVENTS, ST_STEPS64, ST_N
};

// Device workspace: queue counters, list lengths, status and statistics.
// Cleared before every render.
struct WorkK {
  unsigned long long q_next;      // coherent-pass queue (slots)
  unsigned long long long_count;  // rays moved to the long-ray list
  unsigned long long long_next;   // long-ray consumer position
  unsigned long long band_count;  // rays deferred to the FP64 band list
  unsigned long long band_next;
  unsigned long long surr_count;  // surrogate fallback list
  unsigned long long surr_next;
  unsigned int status;            // BH_STATUS_* bits
  unsigned int pad;
  unsigned long long stats[ST_N];
};

// Saved state of a ray moved from the coherent pass to the long-ray list.
template <typename R>
struct Spill {
  int q;       // queue slot
  int steps;
  unsigned aux;
  int pad;
  R u, v, phi, h;
};

enum Mode { MODE_FP64 = 0, MODE_FP32 = 1, MODE_MIXED = 2, MODE_BAND64 = 3 };

// Kernel parameter block.
struct Params {
  SceneK s;
  const CamK* cams;
  int n_cams;
  int tile_w, tile_h;
  int budget;
  long long n_queue;  // queue slots
  long long n_rays;   // output rays
  double rtol, atol;            // integrator tolerances of the main pass
  double rtol64, atol64;        // FP64 band tolerances (MIXED)
  double band;                  // |b - b_c| below which MIXED defers to FP64
  double phi_max;
  double h_max;                 // step-size cap of the main pass (FP64 band: none)
  int max_steps;
  int peri_reset;
  unsigned long long abort_after;  // stop grabbing work past this slot (0 = off)
  void* dirs;
  uint16_t* flags;
  uint32_t* rgba;
  WorkK* ws;
  void* spill;        // Spill<R>[n_queue]
  int* band_list;     // queue slots deferred to FP64 [n_queue]
};

}  // namespace bhk
