// Plain-data types shared by the host runtime and the kernels.
#pragma once

#include <stdint.h>

#include <cmath>

#include "bh.h"

namespace bhk {

constexpr int kMaxSph = BH_MAX_SPHERES;

// Scene constants in the kernel's arithmetic type (a float copy for the
// FP32 kernels, so they convert nothing from double on the slow FP64 pipe).
template <typename R>
struct SceneR {
  R M, M3, u_capt, b_crit, r_in, r_out;
  R c[kMaxSph][3], c2[kMaxSph], rad[kMaxSph], K[kMaxSph];
  // Rays with impact parameter b > cull_b[k] never meet sphere k: an
  // unbound orbit (b > 3 sqrt(3) M) stays at r >= r_p, its periastron, and
  // b = r_p sqrt(r_p / (r_p - 2M)) exceeds r_p by at most 3 sqrt(3) M - 3M
  // = 2.196M (at r_p = 3M; the excess falls to M as r_p grows), so
  // r_p >= b - 2.2M; the ball |x - c_k| <= R_k lies within r <= |c_k| + R_k.
  // cull_b = (|c_k| + R_k)(1 + 1e-5) + 2.25M, the margins covering the
  // rounding of b; +inf when that is not above 3 sqrt(3) M (a sphere
  // reaching inside about 3M, which captured orbits may meet).
  R cull_b[kMaxSph];
  R cnorm[kMaxSph];  // |c_k|
};

// Camera constants in the kernel's arithmetic type.  A camera looks at the
// hole (fwd = -pos / r_obs), so the ray through image-plane point (sx, sy)
// has tan(alpha) = rho = |(sx, sy)| with alpha its angle from the direction
// of the hole, its orbital plane holds e1 = pos / r_obs and
// e2 = (sx right + sy up) / rho, and its normal is n = (sx up - sy right) / rho.
template <typename R>
struct CamR {
  R pos[3], fwd[3], right[3], up[3];
  R sx, sy, r_obs;
  R ir;              // 1 / r_obs
  R px_scale;        // 2 sx / w: image-plane step per pixel column
  R py_scale;        // 2 sy / h
  R inv_tiles_x;     // 1 / tiles_x (a first guess for the tile row)
  R pdiag;           // sqrt(px_scale^2 + py_scale^2): one pixel's diagonal
  R kb;              // b = kb sin(alpha): r_obs / sqrt(1 - 2M / r_obs) (static observer)
  R kv;              // u'0 = kv / rho: u0 sqrt(1 - 2M u0) (static) or u0 (Euclidean)
  R ec[kMaxSph];     // e1 . c_k
  R rc[kMaxSph];     // right . c_k
  R uc[kMaxSph];     // up . c_k
};

// Tolerances and caps in the kernel's arithmetic type.
template <typename R>
struct TolR {
  R rtol, atol, phi_max, h_max, band;
  R h_far;  // step cap of rays with |b - b_c| >= kFarB (FP32 passes)
  R far_e2; // (rtol / rtol_far)^2: their squared error norm is scaled by it
  R near_e2; // FP32 form: (rtol / rtol_near)^2 for rays with |b - b_c| < band
};

// Rays at least this far from the critical impact parameter (units of M)
// take the relaxed step cap h_far and tolerance rtol_far in the FP32 passes.
constexpr double kFarB = 2.0;

// Tile shapes: tile_w * tile_h slots, a power of two from 32 to 256, tile_w
// a power of two.
inline bool tile_shape_ok(int tw, int th) {
  const int t = tw * th;
  return tw >= 1 && th >= 1 && t >= 32 && t <= 256 && (t & (t - 1)) == 0 && (tw & (tw - 1)) == 0;
}
inline int ilog2(int x) {
  int k = 0;
  while ((1 << (k + 1)) <= x) ++k;
  return k;
}

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
  const uint32_t* sky_tex;  // equirectangular RGBA8 sky image, or null: checker
  const float4* sky_lut;    // checker: the 512 cell colours (rgb), or null
  int sky_w, sky_h;
  SceneR<float> f;
  SceneR<double> d;
};

// One camera in device memory.  Its rays occupy queue slots
// [q_off, q_off + tiles_x * tiles_y * tile_w * tile_h): tile after tile,
// row-major within a tile, padded where w or h is not a multiple of the
// tile; a warp takes its 32-slot groups in turn.
struct CamK {
  double pos[3], fwd[3], right[3], up[3];
  double sx, sy;       // tan(fov/2) and tan(fov/2) * h / w
  double r_obs;
  int w, h, tiles_x, tiles_y;
  long long q_off, out_off;
  CamR<float> f;
  CamR<double> d;
  // u0^2 (1 - 2M u0) of the FP32 state u0 = f.ir and the FP32 mass: the
  // u0 part of the first integral, for the MIXED periastron solve
  double peri_k0;
  float peri_k0f;
  // MIXED band as bounds on the squared image-plane radius (band_pixel)
  float band_rho2_lo, band_rho2_hi;
  // 1/b^2 of the ray through image-plane radius rho: peri_A + peri_B / rho^2
  // (FP64, u0 = 1/r_obs; MIXED turning point with periastron_reset = 2)
  double peri_A, peri_B;
  int row_off;  // first row of this camera among all cameras' rows
};

// Fill a camera's MIXED band bounds: rays with |b - b_c| < band are those
// whose image-plane radius rho = tan(alpha) satisfies rho^2 in (lo, hi),
// from b(alpha) = r sin(alpha) / sqrt(1 - 2M/r) (static observer) or
// r sin(alpha) / sqrt(1 - 2M sin^2(alpha) / r) (Euclidean), both increasing
// in alpha.  band <= 0: an empty band.
inline double band_rho2_of_b(double b, double r, double M, int ic) {
  if (!(b > 0.0)) return 0.0;
  double s = ic == 0 ? b * std::sqrt(1.0 - 2.0 * M / r) / r : b / std::sqrt(r * r + 2.0 * M * b * b / r);
  if (!(s < 1.0)) return INFINITY;
  return s * s / (1.0 - s * s);
}
inline void fill_cam_band(CamK& c, double M, int ic, double band) {
  const double bc = 3.0 * std::sqrt(3.0) * M;
  // 1/b^2 = u0^2 (1 - 2M u0) / sin^2(alpha) (static observer) or
  // u0^2 / sin^2(alpha) - 2M u0^3 (Euclidean), with 1/sin^2 = 1 + 1/rho^2
  const double u0 = 1.0 / c.r_obs;
  c.peri_A = u0 * u0 * (1.0 - 2.0 * M * u0);
  c.peri_B = ic == 0 ? c.peri_A : u0 * u0;
  if (!(band > 0.0) || !(M > 0.0)) {
    c.band_rho2_lo = c.band_rho2_hi = -1.0f;
    return;
  }
  c.band_rho2_lo = (float)band_rho2_of_b(bc - band, c.r_obs, M, ic);
  c.band_rho2_hi = (float)band_rho2_of_b(bc + band, c.r_obs, M, ic);
}

// Fill the periastron constant of a camera (after fill_cam_r).
inline void fill_cam_peri(CamK& c, float M) {
  const double u0 = (double)c.f.ir;
  c.peri_k0 = u0 * u0 * (1.0 - 2.0 * (double)M * u0);
  c.peri_k0f = (float)c.peri_k0;
}

enum StatId {
  ST_RAYS, ST_STEPS, ST_REJ, ST_ESC, ST_CAPT, ST_DISK, ST_SPH, ST_LIM, ST_BAND, ST_LONG,
  ST_SURR, ST_FALLBACK, ST_GRABS, ST_PERI, ST_EVENTS, ST_STEPS64, ST_MLP, ST_N
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

enum Mode { MODE_FP64 = 0, MODE_FP32 = 1, MODE_MIXED = 2, MODE_BAND64 = 3, MODE_PAPER32 = 4,
            MODE_PAPER64 = 5 };

// Kernel parameter block.
struct Params {
  SceneK s;
  const CamK* cams;
  int n_cams;
  int tile_w, tile_h;
  int tile_shift;     // log2(tile_w * tile_h): slots per tile, a power of two >= 32
  int tile_wshift;    // log2(tile_w)
  int chunk;          // queue slots a warp takes per grab (a multiple of 32)
  int budget;
  long long n_queue;  // queue slots: the pass takes slots [q_begin, n_queue)
  long long q_begin;  // first slot (0; a later window when a render is split into strips)
  long long n_rays;   // output rays
  double rtol, atol;            // integrator tolerances of the main pass
  double rtol64, atol64;        // FP64 band tolerances (MIXED)
  double band;                  // |b - b_c| below which MIXED defers to FP64
  double phi_max;
  double h_max;                 // step-size cap of the main pass (FP64 band: none)
  double h_max_far;             // FP32 step cap of rays with |b - b_c| >= kFarB
  double rtol_far;              // FP32 rtol of those rays (atol scaled alike)
  double rtol_near;             // FP32 form: rtol of rays with |b - b_c| < band
  double paper_eps;             // fixed step of the polyline modes
  int spp_n;                    // samples per pixel side (n x n), 1 = one centre ray
  int doppler;                  // Keplerian disk shading
  int max_steps;
  int peri_reset;
  unsigned long long abort_after;  // stop grabbing work past this slot (0 = off)
  void* dirs;
  uint16_t* flags;
  uint32_t* rgba;
  WorkK* ws;
  void* spill;        // Spill<R>[n_queue]
  int* band_list;     // queue slots deferred to FP64 [n_queue]
  int band_trim;      // MIXED: band-pass warps beyond the list's need leave at once
  // surrogate mode
  const uint16_t* mlp_w;       // FP16 W^T tiles of the tensor-core path (bhs::TC_NW)
  const float* mlp_bias;       // bhs::NBIAS
  const unsigned char* surr_table;  // served (1) / fallback (0) per calibration bin
  int surr_nb_lb, surr_nb_r;   // table dimensions: ln(b - b_c) bins x r_obs bins
  int* surr_list;              // queue slots the surrogate hands back to the integrator
  TolR<float> tf;     // main pass, FP32 kernels
  TolR<double> td;    // main pass, FP64 mode
  TolR<double> tb;    // FP64 band pass of the MIXED mode
};

template <typename R> __host__ __device__ __forceinline__ const SceneR<R>& SR(const SceneK& s);
template <> __host__ __device__ __forceinline__ const SceneR<float>& SR<float>(const SceneK& s) { return s.f; }
template <> __host__ __device__ __forceinline__ const SceneR<double>& SR<double>(const SceneK& s) { return s.d; }
template <typename R> __host__ __device__ __forceinline__ const CamR<R>& CR(const CamK& c);
template <> __host__ __device__ __forceinline__ const CamR<float>& CR<float>(const CamK& c) { return c.f; }
template <> __host__ __device__ __forceinline__ const CamR<double>& CR<double>(const CamK& c) { return c.d; }

// Fill the typed copies of the scene, camera and tolerance constants.
template <typename R>
inline void fill_scene_r(const SceneK& s, SceneR<R>* o) {
  o->M = R(s.M);
  o->M3 = R(s.M3);
  o->u_capt = R(s.u_capt);
  o->b_crit = R(s.b_crit);
  o->r_in = R(s.r_in);
  o->r_out = R(s.r_out);
  for (int k = 0; k < kMaxSph; ++k) {
    for (int j = 0; j < 3; ++j) o->c[k][j] = R(s.c[k][j]);
    o->c2[k] = R(s.c2[k]);
    o->rad[k] = R(s.R[k]);
    o->K[k] = R(s.K[k]);
    o->cnorm[k] = R(std::sqrt(s.c2[k]));
    const double cb = (std::sqrt(s.c2[k]) + s.R[k]) * (1.0 + 1e-5) + 2.25 * s.M;
    o->cull_b[k] = cb > 1.001 * s.b_crit ? R(cb) : R(INFINITY);
  }
}
// Typed camera constants; the scene gives the mass, the initial-condition
// convention and the sphere centres.
template <typename R>
inline void fill_cam_r(const CamK& c, const SceneK& s, CamR<R>* o) {
  for (int j = 0; j < 3; ++j) {
    o->pos[j] = R(c.pos[j]);
    o->fwd[j] = R(c.fwd[j]);
    o->right[j] = R(c.right[j]);
    o->up[j] = R(c.up[j]);
  }
  o->sx = R(c.sx);
  o->sy = R(c.sy);
  o->r_obs = R(c.r_obs);
  o->ir = R(1.0 / c.r_obs);
  const double pxs = 2.0 * c.sx / c.w, pys = 2.0 * c.sy / c.h;
  o->px_scale = R(pxs);
  o->py_scale = R(pys);
  o->inv_tiles_x = R(1.0 / c.tiles_x);
  o->pdiag = R(std::sqrt(pxs * pxs + pys * pys));
  const double u0 = 1.0 / c.r_obs;
  o->kb = R(c.r_obs / std::sqrt(1.0 - 2.0 * s.M * u0));
  o->kv = R(s.ic == 0 ? u0 * std::sqrt(1.0 - 2.0 * s.M * u0) : u0);
  for (int k = 0; k < kMaxSph; ++k) {
    double e = 0.0, rr = 0.0, uu = 0.0;
    for (int j = 0; j < 3; ++j) {
      e += c.pos[j] * u0 * s.c[k][j];
      rr += c.right[j] * s.c[k][j];
      uu += c.up[j] * s.c[k][j];
    }
    o->ec[k] = R(e);
    o->rc[k] = R(rr);
    o->uc[k] = R(uu);
  }
}

}  // namespace bhk
