// Persistent render kernels.
//
// The image is cut into tiles of tile_w x tile_h pixels (32 to 256, camera-
// major, row-major inside a tile); a warp grabs `chunk` queue slots at a time
// from a global atomic counter and takes them 32 at a time.  It integrates
// its 32 neighbouring rays in lock step (coherent pass); a ray that needs more than
// `budget` attempted steps -- near the photon sphere the step count grows
// like -ln|b - 3 sqrt(3) M| -- is saved to the long-ray list and finished by
// a second persistent kernel whose lanes refill one ray at a time, so one
// slow ray never holds 31 idle lanes.  In MIXED mode rays inside the band
// |b - b_c| < band go to a third list that an FP64 kernel finishes beside
// the FP32 coherent pass.
#include <cuda_runtime.h>
#include <stdint.h>

#include "mlp.cuh"
#include "mlp_tc.cuh"
#include "render.h"
#include "tracer.cuh"

namespace bhk {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Tolerances of a pass: FP32 kernels, FP64 mode, or the MIXED FP64 band.
template <typename R, int MODE> struct TolPick;
template <int MODE> struct TolPick<float, MODE> {
  static __device__ __forceinline__ const TolR<float>& get(const Params& p) { return p.tf; }
};
template <int MODE> struct TolPick<double, MODE> {
  static __device__ __forceinline__ const TolR<double>& get(const Params& p) {
    return MODE == MODE_BAND64 ? p.tb : p.td;
  }
};

struct LocalStats {
  unsigned c[ST_N];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < ST_N; ++i) c[i] = 0;
  }
  __device__ __forceinline__ void flush(WorkK* ws) {
#pragma unroll
    for (int i = 0; i < ST_N; ++i) {
      const unsigned s = __reduce_add_sync(kFull, c[i]);
      if ((threadIdx.x & 31) == 0 && s) atomicAdd(&ws->stats[i], (unsigned long long)s);
    }
  }
  __device__ __forceinline__ void count_flag(unsigned fl) {
    const unsigned f = fl & 0xFFu;
    c[ST_RAYS]++;
    if (f & BH_FLAG_ESC) c[ST_ESC]++;
    if (f & BH_FLAG_CAPT) c[ST_CAPT]++;
    if (f & BH_FLAG_DISK) c[ST_DISK]++;
    if (f & BH_FLAG_SPHERE) c[ST_SPH]++;
    if (f & BH_FLAG_STEP_LIMIT) c[ST_LIM]++;
  }
};

// Queue slot -> camera, pixel and output index.  Returns false for padding.
__device__ __forceinline__ bool slot_pixel(const Params& p, long long q, int* cam, int* px,
                                           int* py, int* out) {
  int lo = 0, hi = p.n_cams - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.cams[mid].q_off <= q)
      lo = mid;
    else
      hi = mid - 1;
  }
  const CamK& c = p.cams[lo];
  const long long l = q - c.q_off;
  const int tile = (int)(l >> p.tile_shift), i = (int)(l & ((1 << p.tile_shift) - 1));
  // tile row from an FP32 estimate, corrected to the exact quotient (the
  // estimate is off by a few at most, for tile counts beyond 2^24)
  int ty = (int)((float)tile * c.f.inv_tiles_x);
  int tx = tile - ty * c.tiles_x;
  while (tx < 0) {
    --ty;
    tx += c.tiles_x;
  }
  while (tx >= c.tiles_x) {
    ++ty;
    tx -= c.tiles_x;
  }
  // tile_w and the tile's slot count are powers of two
  const int x = tx * p.tile_w + (i & (p.tile_w - 1));
  const int y = ty * p.tile_h + (i >> p.tile_wshift);
  *cam = lo;
  *px = x;
  *py = y;
  *out = (int)(c.out_off + (long long)y * c.w + x);
  return x < c.w && y < c.h;
}

// Straight radial ray (|P x d| ~ 0): spheres by exact ray-sphere
// intersection, otherwise capture (ingoing) or escape along d.  At most a
// pixel or two per image, but inlined: an out-of-line call inside the
// persistent loop makes the caller keep values live across it in local
// memory (measured 1% slower FP32, 7% slower mixed).  Returns the ray's
// flags; the caller counts them.
template <typename R, typename OutR, bool SPP = false>
__device__ __forceinline__ unsigned radial_ray(const Params& p, const R P[3], const R d[3], R cos_a,
                                            int out, unsigned aux, SppAcc* acc = nullptr) {
  const SceneK& s = p.s;
  const SceneR<R>& S = SR<R>(s);
  R best = R(INFINITY);
  int bk = -1;
  for (int k = 0; k < s.n_sph; ++k) {
    const R o0 = P[0] - S.c[k][0], o1 = P[1] - S.c[k][1], o2 = P[2] - S.c[k][2];
    const R bq = o0 * d[0] + o1 * d[1] + o2 * d[2];
    const R cq = o0 * o0 + o1 * o1 + o2 * o2 - S.rad[k] * S.rad[k];
    const R disc = bq * bq - cq;
    if (disc < R(0)) continue;
    const R t = -bq - m_sqrt(disc);
    if (t > R(0) && t < best) {
      best = t;
      bk = k;
    }
  }
  const R r0 = m_sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
  const bool ingoing = cos_a < R(0);
  const R t_hole = ingoing ? r0 - R(2) * S.M : R(INFINITY);
  unsigned flags;
  if (bk >= 0 && best < t_hole) {
    const R x0 = P[0] + best * d[0], x1 = P[1] + best * d[1], x2 = P[2] + best * d[2];
    const R iR = R(1) / S.rad[bk];
    const R N0 = (x0 - S.c[bk][0]) * iR, N1 = (x1 - S.c[bk][1]) * iR,
            N2 = (x2 - S.c[bk][2]) * iR;
    const float lam = 0.25f + 0.75f * fmaxf(0.0f, (float)(-(N0 * d[0] + N1 * d[1] + N2 * d[2])));
    const R ix = R(1) / m_sqrt(x0 * x0 + x1 * x1 + x2 * x2);
    R th, ph;
    dir_angles(x0 * ix, x1 * ix, x2 * ix, &th, &ph);
    flags = BH_FLAG_SPHERE | ((unsigned)bk << 8) | aux;
    const float c[3] = {s.alb[bk][0] * lam, s.alb[bk][1] * lam, s.alb[bk][2] * lam};
    emit_ray<OutR, SPP>(p, out, OutR(th), OutR(ph), flags, c, acc);
  } else if (ingoing && S.M > R(0)) {
    flags = BH_FLAG_CAPT | aux;
    const float c[3] = {0.0f, 0.0f, 0.0f};
    emit_ray<OutR, SPP>(p, out, OutR(NAN), OutR(NAN), flags, c, acc);
  } else {
    R th, ph;
    dir_angles(d[0], d[1], d[2], &th, &ph);
    flags = BH_FLAG_ESC | aux;
    float c[3];
    if (s.sky_tex)
      sky_image_rgb<R>(s, th, ph, c);
    else
      sky_rgb<R>(s, th, ph, c);
    emit_ray<OutR, SPP>(p, out, OutR(th), OutR(ph), flags, c, acc);
  }
  return flags;
}

// Periastron of the orbit through the FP32 initial state (u0, v0): the
// middle root u_p of P(u) = 2M u^3 - u^2 + E0, E0 = v0^2 + u0^2 (1 - 2M u0).
// u0 = 1/r_obs is the same for every ray of a camera, so the camera table
// holds k0 = u0^2 (1 - 2M u0) exactly in FP64 (and rounded to FP32); E0 is
// then one FP64 fused multiply-add of the ray's v0.  FP32 start from the
// trigonometric form of the cubic's roots,
//   u_p = cos(acos(1 - 54 M^2 E0) / 3 - 2 pi / 3) / (3M) + 1/(6M),
// one FP32 Newton step, then one Newton step whose residual P(u) is
// evaluated in FP64 (the slope only scales the small correction and stays
// in FP32).  Seven operations on the FP64 pipe per ray.  NaN when there is
// no turning point (b <= 3 sqrt(3) M).  Solved once per ray at set-up,
// where a warp's lanes run it together.
// arccos on [-1, 1] to 6.7e-5 rad (Abramowitz & Stegun 4.4.45); only the
// starting guess of the periastron uses it, which two Newton steps refine.
__device__ __forceinline__ float acos_guess(float x) {
  const float a = fabsf(x);
  const float p = fmaf(fmaf(fmaf(-0.0187293f, a, 0.0742610f), a, -0.2121144f), a, 1.5707288f);
  const float r = sqrtf(fmaxf(0.0f, 1.0f - a)) * p;
  return x >= 0.0f ? r : 3.14159265f - r;
}

// Middle root of 2M u^3 - u^2 + E0 from E0 given in FP64 (and its FP32
// rounding E): the FP32 start and Newton step, then the Newton step whose
// residual is FP64.
__device__ __forceinline__ float periastron_of_e(float M, double m2, float E, double E0) {
  if (!(M > 0.0f)) return sqrtf(E);
  const float x = fmaf(-54.0f * M * M, E, 1.0f);
  if (!(x > -1.0f)) return NAN;
  const float im = 1.0f / M;
  float u = fmaf(0.33333334f * im, __cosf(acos_guess(x) * 0.33333334f - 2.0943951f), 0.16666667f * im);
  const float m2f = 2.0f * M;
  u -= fmaf(u * u, fmaf(m2f, u, -1.0f), E) / (u * fmaf(3.0f * m2f, u, -2.0f));
  const double ud = u;
  const double f = fma(ud * ud, fma(m2, ud, -1.0), E0);
  return fmaf(-(float)f, 1.0f / (u * fmaf(3.0f * m2f, u, -2.0f)), u);
}

__device__ __forceinline__ float periastron64(float M, double m2, float v0f, double k0, float k0f) {
  const double vd = v0f;
  return periastron_of_e(M, m2, fmaf(v0f, v0f, k0f), fma(vd, vd, k0));
}

// The same periastron for the ray through image point (px + ox, py + oy) of
// camera c with 1/b^2 itself in FP64: rho^2 = sx^2 + sy^2 from the camera's
// FP64 constants, 1/rho^2 from the FP32 reciprocal and one FP64 Newton step
// (relative error about 1e-14), 1/b^2 = peri_A + peri_B / rho^2 (fill_cam_band).
// Eleven operations on the FP64 pipe.
__device__ __forceinline__ float periastron_b64(float M, const CamK& c, double px, double py) {
  const double sx = fma(px, c.d.px_scale, -c.d.sx);
  const double sy = fma(-py, c.d.py_scale, c.d.sy);
  const double rho2 = fma(sx, sx, sy * sy);
  const double y0 = (double)rcp_approx((float)rho2);
  const double y = fma(y0, fma(-rho2, y0, 1.0), y0);
  const double E0 = fma(c.peri_B, y, c.peri_A);
  return periastron_of_e(M, 2.0 * (double)M, (float)E0, E0);
}

// Photon-sphere band of the MIXED mode as a test on the pixel: a camera
// looks at the hole, so the ray through image-plane point (sx, sy) makes the
// angle alpha with tan(alpha) = rho = |(sx, sy)| with the direction of the
// hole, and its impact parameter grows with alpha.  The band
// |b - 3 sqrt(3) M| < band is then rho^2 in (band_rho2_lo, band_rho2_hi),
// bounds the host derives per camera in FP64.  The list builder and the
// passes that skip band rays evaluate this same function, so they agree on
// every pixel.  The comparison is in FP32: the band's edge is a policy, not a
// physical boundary, and a pixel within the FP32 rounding of rho^2 (about
// 1e-7 relative) of it is integrated by either pass within the bar.
__device__ __forceinline__ bool band_pixel(const CamK& c, int px, int py) {
  const float sx = fmaf((float)px + 0.5f, c.f.px_scale, -c.f.sx);
  const float sy = fmaf(-((float)py + 0.5f), c.f.py_scale, c.f.sy);
  const float rho2 = fmaf(sx, sx, sy * sy);
  return rho2 > c.band_rho2_lo && rho2 < c.band_rho2_hi;
}

// Queue slot of pixel (px, py) of camera c (the inverse of slot_pixel).
__device__ __forceinline__ long long pixel_slot(const Params& p, const CamK& c, int px, int py) {
  const int tx = px / p.tile_w, ty = py / p.tile_h;
  const int i = (py - ty * p.tile_h) * p.tile_w + (px - tx * p.tile_w);
  return c.q_off + (((long long)ty * c.tiles_x + tx) << p.tile_shift) + i;
}

// Set up the ray of queue slot q.  Returns true when the ray is to be
// integrated by the caller; false when it was padding, finished directly
// (radial) or deferred to the FP64 band list.
// WCULL: the 32 lanes of the warp call it together for a group of 32 slots
// (one camera) and share one sphere cull (warp_sphere_candidates); else each
// ray tests every sphere.  SURR: the surrogate pass's set-up, which needs the
// plane, b, the first disk node and whether a sphere is cut, and none of the
// integrator's state (sphere windows, turning point, tolerance tier).
template <typename R, int MODE, typename OutR, bool SPP = false, bool WCULL = false,
          bool SURR = false>
__device__ bool setup_slot(const Params& p, long long q, Ray<R>& r, LocalStats& st, R* b_out,
                           R ox = R(0.5), R oy = R(0.5), SppAcc* acc = nullptr) {
  int cam, px, py, out;
  const bool in_image = slot_pixel(p, q, &cam, &px, &py, &out);
  const CamK& c = p.cams[cam];
  const CamR<R>& C = CR<R>(c);
  // image-plane point of the ray (pixel centre, or a sub-pixel sample)
  const R sx = m_fma(R(px) + ox, C.px_scale, -C.sx);
  const R sy = m_fma(-(R(py) + oy), C.py_scale, C.sy);
  unsigned cand = (1u << p.s.n_sph) - 1u;
  if (WCULL) cand = warp_sphere_candidates<R>(p.s, c, sx, sy);
  if (q >= p.n_queue || !in_image) return false;
  // band rays belong to the FP64 pass (listed by k_band_list)
  if (MODE == MODE_MIXED && band_pixel(c, px, py)) return false;
  r.out = out;
  r.aux = (MODE == MODE_FP64 || MODE == MODE_BAND64) ? BH_FLAG_FP64 : 0u;
  if (MODE == MODE_BAND64) r.aux |= BH_FLAG_BAND;
  R b, cos_a;
  if (plane_setup<R, !SURR>(p.s, c, sx, sy, cand, r, &b, &cos_a)) {
    R P[3], d[3];
    camera_ray<R>(c, px, py, P, d, ox, oy);
    st.count_flag(radial_ray<R, OutR, SPP>(p, P, d, cos_a, out, r.aux, acc));
    return false;
  }
  *b_out = b;
  if (SURR) return true;
  const TolR<R>& tol = TolPick<R, MODE>::get(p);
  const bool d64 = (MODE == MODE_FP64 || MODE == MODE_BAND64);
  // rays at least kFarB from the critical impact parameter, whose exit
  // directions amplify stepping errors far less
  const R db = m_abs(b - SR<R>(p.s).b_crit);
  const bool far = !d64 && db >= R(kFarB) * SR<R>(p.s).M;
  if (MODE == MODE_MIXED) {
    // the FP64 turning point of near-critical rays (all rays with
    // peri_reset == 2); the others step through it in FP32
    if (p.peri_reset == 2 && r.v > R(0)) {
      // every ray with a turning point, 1/b^2 from the FP64 image radius
      r.up = R(periastron_b64(p.s.f.M, c, (double)px + (double)ox, (double)py + (double)oy));
      r.tp = R(0);
    } else if (p.peri_reset == 1 && !far && r.v > R(0)) {
      r.up = R(periastron64(p.s.f.M, 2.0 * (double)p.s.f.M, float(r.v), c.peri_k0, c.peri_k0f));
      r.tp = R(0);
    } else {
      r.up = R(NAN);
      r.tp = R(-INFINITY);
      r.aux |= kAuxPeriDone;
    }
  }
  r.phi_evt = m_min(m_min(r.phi_node, r.phi_sph), tol.phi_max);
  r.steps = 0;
  // FP64 mirrors the oracle's starting step; FP32 starts at the ray's step
  // cap, h_far for far rays (the controller shrinks it when the first
  // attempt is rejected; near the observer u is small and the long first
  // step is accepted: 5.27 -> 4.84 attempted steps per ray at 4096^2)
  r.h = d64 ? initial_step<R>(SR<R>(p.s).M3, r.u, r.v, tol.rtol, tol.atol, R(0.01))
            : (far ? tol.h_far : tol.h_max);
  if (far) r.aux |= kAuxFar;
  // the FP32 form's near-critical rays, which the other forms integrate in
  // FP64, are held to rtol_near
  if (MODE == MODE_FP32 && db < tol.band) r.aux |= kAuxNear;
  // the tier as two per-ray constants, so a step multiplies and clamps
  // instead of testing the tier bits
  r.es = far ? tol.far_e2 : ((MODE == MODE_FP32 && db < tol.band) ? tol.near_e2 : R(1));
  r.hc = far ? tol.h_far : tol.h_max;
  return true;
}

// Band list of the MIXED mode: one warp per image row finds the columns
// where the row meets the band annulus (two x intervals from the bounds on
// rho^2), its lanes test band_pixel on them and two pixels beyond each end,
// and the warp appends the band rays' queue slots to the FP64 list with one
// atomic per 32 columns.
__global__ void __launch_bounds__(256) k_band_list(const __grid_constant__ Params p, int row0,
                                                   int n_rows) {
  // the FP64 band pass may be scheduled now; it waits for this grid's list
  pdl_launch_dependents();
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.x * (blockDim.x >> 5);
  LocalStats st;
  st.zero();
  for (int row = row0 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); row < row0 + n_rows;
       row += warps) {
    int lo = 0, hi = p.n_cams - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (p.cams[mid].row_off <= row)
        lo = mid;
      else
        hi = mid - 1;
    }
    const CamK& c = p.cams[lo];
    const int py = row - c.row_off;
    if (!(c.band_rho2_hi > c.band_rho2_lo)) continue;
    const float sy = fmaf(-((float)py + 0.5f), c.f.py_scale, c.f.sy);
    const float out2 = c.band_rho2_hi - sy * sy;
    if (!(out2 > 0.0f)) continue;
    const float a = sqrtf(fmaxf(0.0f, c.band_rho2_lo - sy * sy)), bnd = sqrtf(out2);
    // columns x with |sx| in (a, bnd), sx = (x + 1/2) px_scale - sx_half
    const float ip = 1.0f / c.f.px_scale;
    const float xl[2] = {(-bnd + c.f.sx) * ip - 0.5f, (a + c.f.sx) * ip - 0.5f};
    const float xh[2] = {(-a + c.f.sx) * ip - 0.5f, (bnd + c.f.sx) * ip - 0.5f};
    int from[2], to[2];
    for (int k = 0; k < 2; ++k) {
      from[k] = max(0, (int)floorf(xl[k]) - 2);
      to[k] = min(c.w - 1, (int)ceilf(xh[k]) + 2);
    }
    if (from[1] <= to[0] + 1) {  // the two intervals touch: one scan
      to[0] = max(to[0], to[1]);
      from[1] = 1;
      to[1] = 0;
    }
    for (int k = 0; k < 2; ++k) {
      for (int x0 = from[k]; x0 <= to[k]; x0 += 32) {
        const int px = x0 + lane;
        const bool in = px <= to[k] && band_pixel(c, px, py);
        const unsigned bits = __ballot_sync(kFull, in);
        if (!bits) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&p.ws->band_count, (unsigned long long)__popc(bits));
        base = __shfl_sync(kFull, base, 0);
        if (in) {
          p.band_list[base + __popc(bits & ((1u << lane) - 1u))] = (int)pixel_slot(p, c, px, py);
          st.c[ST_BAND]++;
        }
      }
    }
  }
  st.flush(p.ws);
}

// Periastron reset of the MIXED mode.  An accepted FP32 step has just
// passed the turning point (v went from > 0 to <= 0), so its end lies a
// distance d past the periastron of the orbit through (u_p, 0), u_p from the
// FP64 cubic.  The end state is put on that orbit, so no FP32 drift of the
// incoming leg is carried into the outgoing one.  The orbit is even about
// the turning point (its odd derivatives vanish there), so with
// F(u) = 3Mu^2 - u and F' = 6Mu - 1 taken at u_p,
//   u(d) = u_p + F d^2/2 + F' F d^4/24 + (18M F^2 + F'^2 F) d^6/720,
// the d^8 term below 2e-8 u_p for d <= 0.4 rad, and v(d) = du/dd.  d is the
// root of v(d) = v_end (two Newton steps from d = v_end / F); outside the
// FP64 band |F| >= 0.02 / M, so d follows from the end velocity with the
// velocity's own relative accuracy.  The end velocity is kept; u and the
// FSAL derivative are replaced.  NaN u_p (no turning point): no change.
template <typename R>
__device__ __forceinline__ void periastron_reset(R M3, R up, R h, R& un, R& vn, R& fn) {
  if (!(up == up)) return;
  const R F0 = accel(M3, up);
  const R F1 = m_fma(R(2) * M3, up, R(-1));
  const R c2 = R(0.5) * F0;
  const R c4 = F1 * F0 * R(1.0 / 24.0);
  const R c6 = m_fma(R(6) * M3 * F0, F0, F1 * F1 * F0) * R(1.0 / 720.0);
  R d = vn * m_rcp(F0);
  for (int it = 0; it < 2; ++it) {
    const R d2 = d * d;
    const R g = m_fma(d, m_fma(d2, m_fma(d2, R(6) * c6, R(4) * c4), R(2) * c2), -vn);
    const R dg = m_fma(d2, m_fma(d2, R(30) * c6, R(12) * c4), R(2) * c2);
    d -= g * m_rcp(dg);
  }
  d = m_min(m_max(d, R(0)), h);
  const R d2 = d * d;
  un = m_fma(d2, m_fma(d2, m_fma(d2, c6, c4), c2), up);
  vn = d * m_fma(d2, m_fma(d2, R(6) * c6, R(4) * c4), R(2) * c2);
  fn = accel(M3, un);
}

template <typename R, typename E>
__device__ __forceinline__ void consider(int type, R ph, unsigned id, int& bt, R& bp, unsigned& bid) {
  const R tie = R(Num<E>::tie);
  if (bt < 0 || ph < bp - tie ||
      (m_abs(ph - bp) <= tie && (type < bt || (type == bt && id < bid)))) {
    bt = type;
    bp = ph;
    bid = id;
  }
}

enum { EV_CAPT = 0, EV_SPHERE = 1, EV_DISK = 2, EV_ESC = 3 };

// Arithmetic type of event location.  The FP64 band pass of the MIXED mode
// steps in FP64 (the orbit's sensitivity near the photon sphere needs it)
// but locates events in FP32: its results are stored in FP32 against a
// 1e-4 rad budget, and FP32 root searches cost a small fraction of FP64 ones
// on the narrow FP64 pipe.  Every other pass uses its stepping type.
template <typename R, int MODE> struct EventT { using type = R; };
template <> struct EventT<double, MODE_BAND64> { using type = float; };

// Event handling for an accepted step [pa, pa + h] that may hold an event:
// locate capture / escape roots, disk-node crossings and sphere entries on
// the quintic Hermite interpolant and keep the earliest (ties within
// Num<E>::tie: capture > sphere (lower index) > disk > escape).  With a
// narrower event type E the interpolant's angles are taken relative to
// shift = 2 pi floor(pa / 2 pi), so they stay small in FP32.
template <typename R, int MODE>
__device__ bool step_events(const Params& p, Ray<R>& r, R& un, R& vn, R& fn, R& pb, R h,
                            Hit<R>& hit, LocalStats& st) {
  using E = typename EventT<R, MODE>::type;
  constexpr bool narrow = sizeof(E) < sizeof(R);
  const SceneK& s = p.s;
  const SceneR<E>& S = SR<E>(s);
  const E M3 = S.M3;
  const R pa = r.phi;
  const R shift = narrow ? Num<R>::two_pi * m_floor(pa * R(0.15915494309189535)) : R(0);
  const E pa_e = E(pa - shift);
  Hermite<E> H;
  H.make(pa_e, E(h), E(r.u), E(r.v), E(r.f), E(un), E(vn), E(fn));
  const R hs = R(H.h);
  int bt = -1;
  R bp = R(0);
  unsigned bid = 0;
  // A disk or sphere hit in a step that ends captured lies before the
  // capture radius is crossed (its radius is finite and outside it), and
  // captured rays output no direction: capture is entered at the step's end
  // without locating its root.
  if (un >= SR<R>(s).u_capt) consider<R, E>(EV_CAPT, pb, 0u, bt, bp, bid);
  if (un <= R(0))
    consider<R, E>(EV_ESC, pa + hs * R(hermite_root<E>(H, E(0), E(0), E(1))), 0u, bt, bp, bid);
  for (int it = 0; it < 8 && r.phi_node <= pb; ++it) {
    const E uk = H.val_t(E((r.phi_node - pa) * R(H.ih)));
    if (uk > E(0)) {
      const E rk = m_quot(E(1), uk);
      if (rk >= S.r_in && rk <= S.r_out) {
        consider<R, E>(EV_DISK, r.phi_node, 0u, bt, bp, bid);
        break;
      }
    }
    r.phi_node += Num<R>::pi;
  }
  if (pb >= r.phi_sph) {
    const E pb_e = E(pb - shift);
    unsigned m = r.sph_mask;
    while (m) {
      const int k = __ffs(m) - 1;
      m &= m - 1;
      E ph;
      if (sphere_entry<E, R>(s, r, k, H, pa_e, pb_e, &ph))
        consider<R, E>(EV_SPHERE, shift + R(ph), (unsigned)k, bt, bp, bid);
    }
    r.phi_sph = next_sphere_window<R>(r, pb);
  }
  r.phi_evt = m_min(m_min(r.phi_node, r.phi_sph), TolPick<R, MODE>::get(p).phi_max);
  if (bt < 0) return false;
  const E tb = E((bp - pa) * R(H.ih));
  hit.phi = bp;
  hit.u = R(H.val_t(tb));
  hit.v = R(H.dval_t(tb) * H.ih);
  hit.flags = bt == EV_CAPT     ? BH_FLAG_CAPT
              : bt == EV_SPHERE ? (BH_FLAG_SPHERE | (bid << 8))
              : bt == EV_DISK   ? BH_FLAG_DISK
                                : BH_FLAG_ESC;
  return true;
}

// One attempted step.  Returns true when the ray ended (hit filled in).
template <typename R, int MODE>
__device__ __forceinline__ bool advance(const Params& p, Ray<R>& r, Hit<R>& hit, LocalStats& st) {
  const SceneR<R>& S = SR<R>(p.s);
  const TolR<R>& tol = TolPick<R, MODE>::get(p);
  R un, vn, fn;
  float err2;
  dp5_attempt<R>(S.M3, r.u, r.v, r.f, r.h, tol.rtol, tol.atol, un, vn, fn, err2);
  // rays far from the critical impact parameter (FP32 passes) are held to
  // rtol_far, the FP32 form's near-critical rays to rtol_near, atol scaled
  // alike: their squared error norm scales by (rtol / rtol_tier)^2.  The FP32
  // form keeps the tier in two per-ray constants; the MIXED pass, whose
  // registers are fuller, tests the far bit (it has no near tier).
  constexpr bool d64 = sizeof(R) == 8;
  if (MODE == MODE_FP32) err2 *= r.es;
  else if (!d64 && (r.aux & kAuxFar)) err2 *= tol.far_e2;
  r.steps++;
  st.c[ST_STEPS]++;
  if (sizeof(R) == 8) st.c[ST_STEPS64]++;
  const R h = r.h;
  r.h = h * step_factor<R>(err2);
  r.h = m_min(r.h, MODE == MODE_FP32 ? r.hc : ((!d64 && (r.aux & kAuxFar)) ? tol.h_far : tol.h_max));
  if (!(err2 <= 1.0f)) {
    st.c[ST_REJ]++;
    if (r.steps >= p.max_steps) {
      hit.flags = BH_FLAG_STEP_LIMIT;
      hit.phi = r.phi;
      hit.u = r.u;
      hit.v = r.v;
      return true;
    }
    return false;
  }
  R pb = r.phi + h;
  // u <= 0 (escape) or u >= u_capt (capture) in one test: |u - c| >= c with
  // c = u_capt / 2; node, sphere window and the phi cap through phi_evt;
  // in MIXED the first step past the turning point (vn <= tp)
  const R c = R(0.5) * S.u_capt;
  bool slow = (m_abs(un - c) >= c) | (pb >= r.phi_evt);
  if (MODE == MODE_MIXED) slow |= vn <= r.tp;
  if (__builtin_expect(slow, 0)) {
    if (MODE == MODE_MIXED && vn <= r.tp) {
      periastron_reset<R>(S.M3, r.up, h, un, vn, fn);
      r.aux |= kAuxPeriDone;
      r.tp = R(-INFINITY);
      st.c[ST_PERI]++;
    }
    if ((m_abs(un - c) >= c) | (pb >= r.phi_evt)) {
      st.c[ST_EVENTS]++;
      if (step_events<R, MODE>(p, r, un, vn, fn, pb, h, hit, st)) return true;
    }
  }
  r.u = un;
  r.v = vn;
  r.f = fn;
  r.phi = pb;
  if (r.steps >= p.max_steps || (slow && pb >= tol.phi_max)) {
    hit.flags = BH_FLAG_STEP_LIMIT;
    hit.phi = pb;
    hit.u = un;
    hit.v = vn;
    return true;
  }
  return false;
}

// Persistent work loop of a warp: each grab of the global counter takes
// p.chunk queue slots, handed to body() 32 at a time (lane i gets slot
// g + i of each 32-slot group g); the loop ends with the queue or at the
// host's abort slot.  Queue windows and lengths are multiples of 32.
template <typename F>
__device__ __forceinline__ void for_each_grab(const Params& p, LocalStats& st, F&& body) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0)
      base = (unsigned long long)p.q_begin + atomicAdd(&p.ws->q_next, (unsigned long long)p.chunk);
    base = __shfl_sync(kFull, base, 0);
    if (base >= (unsigned long long)p.n_queue) break;
    if (p.abort_after && base >= p.abort_after) {
      if (lane == 0) atomicOr(&p.ws->status, (unsigned)BH_STATUS_ABORTED);
      break;
    }
    if (lane == 0) st.c[ST_GRABS]++;
    const unsigned long long end =
        base + (unsigned long long)p.chunk < (unsigned long long)p.n_queue
            ? base + (unsigned long long)p.chunk : (unsigned long long)p.n_queue;
    for (unsigned long long g = base; g < end; g += 32) body((long long)g + lane);
  }
}

// Coherent pass: 32 rays of a grab at a time, lanes in lock step, rays
// over the step budget moved to the long-ray list.
// The lanes of a warp integrate their rays in lock step until each has
// ended (finished and stored) or used its step budget (moved to the
// long-ray list).
// In FP64 a lane whose ray ends keeps the event in registers the ended ray
// no longer needs (phi, u and v in its state, the flags in its step count),
// and the warp maps back, shades and stores its ended rays together after
// the loop: the FP64 map-back runs once per warp instead of once per step
// at which some lane ended (1.4% faster at 4096^2).  FP32 rays finish at
// once (deferred, the FP32 passes measured 3.5% slower).
template <typename R, int MODE, typename OutR, bool SPP = false>
__device__ __forceinline__ void integrate_warp(const Params& p, Ray<R>& r, bool active, long long q,
                                               LocalStats& st, SppAcc* acc = nullptr) {
  constexpr bool defer = sizeof(R) == 8;
  bool ended = false;
  while (__any_sync(kFull, active)) {
    if (active) {
      Hit<R> hit;
      if (advance<R, MODE>(p, r, hit, st)) {
        if (defer) {
          r.phi = hit.phi;
          r.u = hit.u;
          r.v = hit.v;
          r.steps = (int)hit.flags;
          ended = true;
        } else {
          finish_ray<R, OutR, SPP>(p, r, hit, acc);
          st.count_flag(hit.flags | r.aux);
        }
        active = false;
      } else if (r.steps >= p.budget) {
        const unsigned long long k = atomicAdd(&p.ws->long_count, 1ull);
        Spill<R> sp;
        sp.q = (int)q;
        sp.steps = r.steps;
        sp.aux = r.aux;
        sp.pad = 0;
        sp.u = r.u;
        sp.v = r.v;
        sp.phi = r.phi;
        sp.h = r.h;
        reinterpret_cast<Spill<R>*>(p.spill)[k] = sp;
        st.c[ST_LONG]++;
        active = false;
      }
    }
  }
  if (defer && ended) {
    Hit<R> hit;
    hit.flags = (unsigned)r.steps;
    hit.phi = r.phi;
    hit.u = r.u;
    hit.v = r.v;
    finish_ray<R, OutR, SPP>(p, r, hit, acc);
    st.count_flag(hit.flags | r.aux);
  }
}

// Resident 512-thread blocks per SM the register allocation must allow:
// 2 (64 registers) for FP32, 1 (128 registers) for FP64; blocks of up to 512
// threads may be launched.  At 64 registers the FP32 kernels spill a few
// words but run 2% faster than at 80 with three 256-thread blocks.
template <typename R> constexpr int kMinBlocks = sizeof(R) == 4 ? 2 : 1;

// Re-create a ray from its queue slot and, for a long ray, its saved state.
template <typename R, int MODE, typename OutR>
__device__ bool restore_ray(const Params& p, long long q, const Spill<R>* sp, Ray<R>& r,
                            LocalStats& st) {
  R b;
  if (!setup_slot<R, MODE, OutR>(p, q, r, st, &b)) return false;
  if (sp) {
    r.steps = sp->steps;
    r.aux = sp->aux;
    r.u = sp->u;
    r.v = sp->v;
    r.phi = sp->phi;
    r.h = sp->h;
    r.f = accel(SR<R>(p.s).M3, r.u);
    if (r.aux & kAuxPeriDone) r.tp = R(-INFINITY);
    for (int it = 0; it < 64 && r.phi_node <= r.phi; ++it) r.phi_node += Num<R>::pi;
    if (r.sph_mask) r.phi_sph = next_sphere_window<R>(r, r.phi);
    r.phi_evt = m_min(m_min(r.phi_node, r.phi_sph), TolPick<R, MODE>::get(p).phi_max);
  }
  return true;
}

// Sources of the list-driven pass.
enum { SRC_SPILL = 0, SRC_BAND = 1, SRC_SURR = 2 };

// Long-ray pass: every lane refills on its own from a list (saved long
// rays, FP64 band rays, or rays the surrogate sends back to the integrator),
// warp-aggregated: one atomic per refill round.
template <typename R, int MODE, typename OutR, int SRC>
__device__ __forceinline__ void list_pass(const Params& p, LocalStats& st) {
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  constexpr bool FROM_SPILL = SRC == SRC_SPILL;
  unsigned long long* next = SRC == SRC_SPILL ? &p.ws->long_next
                             : SRC == SRC_BAND ? &p.ws->band_next
                                               : &p.ws->surr_next;
  const unsigned long long total =
      SRC == SRC_SPILL  ? *(volatile unsigned long long*)&p.ws->long_count
      : SRC == SRC_BAND ? *(volatile unsigned long long*)&p.ws->band_count
                        : *(volatile unsigned long long*)&p.ws->surr_count;
  Ray<R> r;
  SphWin win;
  r.win = &win;
  bool active = false, exhausted = false;
  for (long long guard = 0; guard < (1ll << 40); ++guard) {
    if (!exhausted) {
      const unsigned need = __ballot_sync(kFull, !active);
      if (need) {
        unsigned long long base = 0;
        if (lane == 0) {
          base = atomicAdd(next, (unsigned long long)__popc(need));
          st.c[ST_GRABS]++;
        }
        base = __shfl_sync(kFull, base, 0);
        if (base + __popc(need) >= total) exhausted = true;
        if (!active) {
          const unsigned long long idx = base + __popc(need & lt_mask);
          if (idx < total) {
            if (FROM_SPILL) {
              const Spill<R> sp = reinterpret_cast<const Spill<R>*>(p.spill)[idx];
              active = restore_ray<R, MODE, OutR>(p, sp.q, &sp, r, st);
            } else {
              const int* list = SRC == SRC_BAND ? p.band_list : p.surr_list;
              active = restore_ray<R, MODE, OutR>(p, list[idx], nullptr, r, st);
            }
          }
        }
      }
    }
    if (!__any_sync(kFull, active)) {
      if (exhausted) break;
      continue;
    }
    if (active) {
      Hit<R> hit;
      if (advance<R, MODE>(p, r, hit, st)) {
        finish_ray<R, OutR>(p, r, hit);
        st.count_flag(hit.flags | r.aux);
        active = false;
      }
    }
  }
}

// The FP64 band pass is held to 64 registers, so one band warp and seven
// 128-thread FP32 blocks fill an SM sub-partition's register file; it lets
// the dependent coherent pass launch at once (see k_coherent).  Of its
// one-warp blocks (band_warps per SM), only as many stay as the band list
// needs for about 1.7 rays a lane, and never fewer than half: the others
// leave at once and give their registers to the coherent pass beside it
// (MIXED only).  At 4096^2 (config 3: 16,172 band rays) two warps per SM
// (1.66 rays a lane) made the mixed frame 0.712 -> 0.700 ms; one (3.3 rays
// a lane) made the band pass the frame's tail (0.96 ms).  Beside the
// surrogate pass, whose shared memory fixes its residency, the band pass
// keeps all its warps (two per SM measured 0.4% slower there).
// The long-ray pass over spilled rays is launched as the programmatic
// dependent of the pass that spills them, so its blocks are scheduled while
// that pass drains; it waits for the pass to complete (and its spill list
// to be visible) before reading the list.
template <typename R, int MODE, typename OutR, int SRC>
__global__ void __launch_bounds__(512, MODE == MODE_BAND64 ? 2 : kMinBlocks<R>)
    k_longrays(const __grid_constant__ Params p) {
  if (SRC == SRC_BAND) pdl_launch_dependents();
  // the pass that fills the list may still run (a programmatic launch):
  // wait for it to complete and its writes to be visible
  pdl_wait_primary();
  if (SRC == SRC_BAND && p.band_trim) {
    const unsigned long long n = *(volatile unsigned long long*)&p.ws->band_count;
    const unsigned long long warps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long want = (n * 10ull + 32ull * 17ull - 1ull) / (32ull * 17ull);
    const unsigned long long keep = want < warps / 2 ? warps / 2 : (want < warps ? want : warps);
    if ((unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5) >= keep) return;
  }
  LocalStats st;
  st.zero();
  list_pass<R, MODE, OutR, SRC>(p, st);
  st.flush(p.ws);
}

// Lock-step pass over the surrogate's fallback list: a warp takes 32
// consecutive list entries at a time -- rays a surrogate warp listed
// together, neighbours in the image -- and integrates them as the coherent
// pass does, rays over the step budget moving to the long-ray list.
template <typename R, int MODE, typename OutR>
__global__ void __launch_bounds__(512, kMinBlocks<R>) k_listwarp(const __grid_constant__ Params p) {
  const int lane = threadIdx.x & 31;
  const unsigned long long total = *(volatile unsigned long long*)&p.ws->surr_count;
  LocalStats st;
  st.zero();
  for (long long guard = 0; guard < (1ll << 40); ++guard) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&p.ws->surr_next, 32ull);
    base = __shfl_sync(kFull, base, 0);
    if (base >= total) break;
    if (lane == 0) st.c[ST_GRABS]++;
    const unsigned long long idx = base + lane;
    const long long q = idx < total ? (long long)p.surr_list[idx] : -1;
    Ray<R> r;
    SphWin win;
    r.win = &win;
    const bool active = q >= 0 && restore_ray<R, MODE, OutR>(p, q, nullptr, r, st);
    integrate_warp<R, MODE, OutR>(p, r, active, q, st);
  }
  st.flush(p.ws);
}

// In MIXED mode the pass is launched as a programmatic dependent of the
// FP64 band pass, so its blocks fill the SMs beside the resident band warps
// (and take the band warps' places as they leave); each block waits for the
// band pass to complete before it exits, so the render ends after both.
template <typename R, int MODE, typename OutR, bool SPP = false>
__global__ void __launch_bounds__(512, kMinBlocks<R>) k_coherent(const __grid_constant__ Params p) {
  // the long-ray pass may be scheduled now; it waits for this grid to end
  pdl_launch_dependents();
  LocalStats st;
  st.zero();
  for_each_grab(p, st, [&](long long q) {
    if (!SPP) {
      Ray<R> r;
      SphWin win;
      r.win = &win;
      R b;
      bool active = setup_slot<R, MODE, OutR, false, true>(p, q, r, st, &b);
      integrate_warp<R, MODE, OutR>(p, r, active, q, st);
    } else {
      // n x n stratified samples per pixel, then the ray through the centre
      // (directions and flags); every ray of the pixel stays in this lane,
      // and the lanes take sample k of their pixels together
      const int n = p.spp_n, ns = n * n;
      const R inv_n = R(1) / R(n);
      SppAcc acc;
      acc.c[0] = acc.c[1] = acc.c[2] = 0.0f;
      SphWin win;
      int out = -1;
      for (int k = 0; k <= ns; ++k) {
        acc.centre = (k == ns);
        const R ox = acc.centre ? R(0.5) : (R(k % n) + R(0.5)) * inv_n;
        const R oy = acc.centre ? R(0.5) : (R(k / n) + R(0.5)) * inv_n;
        Ray<R> r;
        r.win = &win;
        R b;
        r.out = -1;
        bool active = setup_slot<R, MODE, OutR, true, true>(p, q, r, st, &b, ox, oy, &acc);
        if (r.out >= 0) out = r.out;
        integrate_warp<R, MODE, OutR, true>(p, r, active, q, st, &acc);
      }
      if (out >= 0 && p.rgba) {
        const float w = 1.0f / (float)ns;
        p.rgba[out] = pack_rgba(acc.c[0] * w, acc.c[1] * w, acc.c[2] * w);
      }
    }
  });
  st.flush(p.ws);
  if (MODE == MODE_MIXED) pdl_wait_primary();
}

// Surrogate pass.  A CTA of four warps takes 128 queue slots at a time (warp
// w the 32-slot group g + 32w, one tile row of one camera): each thread sets
// up its ray as the MIXED coherent pass does (FP32 camera, orbital plane,
// impact parameter, first disk-node angle psi0, periastron; band rays
// belong to the FP64 pass, radial rays finish at once) and decides whether
// the MLP may answer it -- no sphere cut by the orbital plane, inside the
// training domain, and a calibration bin whose measured 99.9th-percentile
// error is within the threshold.  When any of the 128 may, the CTA
// evaluates the network for all of them on the tensor cores (mlp_cta_tc:
// tcgen05.mma into tensor memory) and shades the rays it answers: a served
// ray escapes at phi_inf = alpha + delta unless the disk is met at psi0 or
// psi0 + pi first (u b from the MLP gives the crossing radius).  The rays it
// does not answer go to a list that the FP32 integrator's list pass
// finishes after this pass.
// 128-thread CTAs, four per SM (54 KB of shared memory and 128 tensor-memory
// columns each), at most 112 registers a thread: the four CTAs (57,344
// registers) and the FP64 band pass's four 64-register warps (8,192) fill
// an SM's 65,536 together, so the band pass runs beside this pass.  A layer
// that does not complete within its poll limit sets BH_STATUS_WATCHDOG and
// ends the pass.
__global__ void __maxnreg__(112) k_surrogate(const __grid_constant__ Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bhs::TcSmem& s = *reinterpret_cast<bhs::TcSmem*>(smem_raw);
  __shared__ unsigned long long s_grab;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  for (int i = tid; i < bhs::TC_NW / 8; i += 128)
    reinterpret_cast<uint4*>(s.w)[i] = reinterpret_cast<const uint4*>(p.mlp_w)[i];
  for (int i = tid; i < bhs::NBIAS; i += 128) s.bias[i] = p.mlp_bias[i];
  if (tid < 32) bhs::tmem_alloc(bhs::smem_u32(&s.tmem), bhs::TC_COLS);
  if (tid == 0) bhs::mbar_init(bhs::smem_u32(&s.mbar), 1);
  bhs::tc_fence_before();
  __syncthreads();
  bhs::tc_fence_after();
  const uint32_t tmem = s.tmem;
  uint32_t phase = 0;
  const SceneR<float>& S = p.s.f;
  const float M = S.M, iM = 1.0f / M;
  const float bc_m = 5.19615242270663188f;  // 3 sqrt 3: b_crit / M
  // slots per CTA grab: the queue chunk rounded up to whole 128-slot groups
  const unsigned long long grab = (unsigned long long)((p.chunk + 127) / 128 * 128);
  LocalStats st;
  st.zero();
  bool failed = false;
  for (;;) {
    if (tid == 0) {
      s_grab = (unsigned long long)p.q_begin + atomicAdd(&p.ws->q_next, grab);
      st.c[ST_GRABS]++;
    }
    __syncthreads();
    const unsigned long long base = s_grab;
    __syncthreads();
    if (base >= (unsigned long long)p.n_queue) break;
    if (p.abort_after && base >= p.abort_after) {
      if (tid == 0) atomicOr(&p.ws->status, (unsigned)BH_STATUS_ABORTED);
      break;
    }
    const unsigned long long end =
        base + grab < (unsigned long long)p.n_queue ? base + grab : (unsigned long long)p.n_queue;
    for (unsigned long long g = base; g < end; g += 128) {
      const long long q = (long long)g + tid;
      Ray<float> r;
      SphWin win;
      r.win = &win;
      float b = 0.0f;
      bool active = setup_slot<float, MODE_MIXED, float, false, true, true>(p, q, r, st, &b);
      bool serve = false;
      float r_obs = 0.0f;
      float f[bhs::K0];
#pragma unroll
      for (int k = 0; k < bhs::K0; ++k) f[k] = 0.0f;
      if (active) {
        r_obs = 1.0f / r.u;  // the set-up state is u = 1 / r_obs
        const float bm = b * iM, rm = r_obs * iM;
        bool ok = r.sph_mask == 0 && bm > bc_m + 1e-4f && rm >= 15.0f && rm <= 100.0f &&
                  (!p.s.disk_on || r.phi_node < 4.0f);
        if (ok) {
          bhs::surrogate_features<float>(bm, rm, p.s.disk_on ? r.phi_node : bhs::P_C, f);
          const int ib = min(p.surr_nb_lb - 1, max(0, (int)((f[0] + 1.0f) * 0.5f * p.surr_nb_lb)));
          const int ir = min(p.surr_nb_r - 1, max(0, (int)((rm - 15.0f) * (1.0f / 85.0f) * p.surr_nb_r)));
          ok = p.surr_table[ib * p.surr_nb_r + ir] != 0;
        }
        serve = ok;
      }
      if (__syncthreads_or(serve)) {
        if (tid == 0) st.c[ST_MLP] += 128;
        float o[3];
        const bool done = bhs::mlp_cta_tc(s, tmem, phase, f, o);
        if (__syncthreads_or(!done)) {
          failed = true;
          serve = false;
        }
        if (serve) {
          // the hardware reciprocal (a few ulp) throughout: far inside the
          // form's 1e-3 rad bound and its 6e-2 M disk-edge ambiguity
          const float ib = rcp_approx(b), iro = rcp_approx(r_obs);
          const float delta = fmaf(o[0], bhs::D_S, bhs::D_C) * 4.0f * M * ib;
          const float alpha =
              3.14159265358979f - asinf(fminf(1.0f, b * sqrtf(1.0f - 2.0f * M * iro) * iro));
          const float phi_inf = alpha + delta;
          Hit<float> hit;
          hit.flags = BH_FLAG_ESC;
          hit.phi = phi_inf;
          hit.u = 0.0f;
          hit.v = 0.0f;
          if (p.s.disk_on) {
            const float pa = r.phi_node, pb = pa + 3.14159265358979f;
            const float ua = o[1] * ib, ub = o[2] * ib;
            const float ra = rcp_approx(ua), rb = rcp_approx(ub);
            if (pa < phi_inf && ua > 0.0f && ra >= S.r_in && ra <= S.r_out) {
              hit.flags = BH_FLAG_DISK;
              hit.phi = pa;
              hit.u = ua;
            } else if (pb < phi_inf && ub > 0.0f && rb >= S.r_in && rb <= S.r_out) {
              hit.flags = BH_FLAG_DISK;
              hit.phi = pb;
              hit.u = ub;
            } else if (phi_inf > pa + 6.2831853f) {
              serve = false;  // a third node crossing: beyond what the MLP predicts
            }
          }
          if (serve) {
            r.aux |= BH_FLAG_SURR;
            finish_ray<float, float>(p, r, hit);
            st.count_flag(hit.flags | r.aux);
            st.c[ST_SURR]++;
            active = false;
          }
        }
      }
      // the rest go to the integrator's list: one atomic per warp
      const unsigned fb = __ballot_sync(kFull, active);
      if (fb) {
        unsigned long long lb = 0;
        if (lane == 0) lb = atomicAdd(&p.ws->surr_count, (unsigned long long)__popc(fb));
        lb = __shfl_sync(kFull, lb, 0);
        if (active) {
          p.surr_list[lb + __popc(fb & ((1u << lane) - 1u))] = (int)q;
          st.c[ST_FALLBACK]++;
        }
      }
      if (failed) break;
    }
    if (failed) break;
  }
  if (failed && tid == 0) atomicOr(&p.ws->status, (unsigned)BH_STATUS_WATCHDOG);
  st.flush(p.ws);
  bhs::tc_fence_before();
  __syncthreads();
  if (tid < 32) {
    bhs::tc_fence_after();
    bhs::tmem_dealloc(tmem, bhs::TC_COLS);
  }
}

// ---------------------------------------------------------------------------
// The paper's own stepping (Sec. 2.1-2.2, Fig. 1), kept as a mode to measure
// it against the adaptive path: points of the ray at fixed steps eps in phi
// from the classical fourth-order Runge-Kutta method, joined by straight
// segments; objects are found by intersecting each segment with them.  The
// segments lie in the orbital plane, so the work is done in its 2-D
// coordinates (x, y) = (cos phi, sin phi) / u.  A step whose end has u <= 0
// escapes along the angle where the line between the last two (phi, u)
// reaches u = 0; a segment ending at u >= 1/(2M) that meets no object is
// captured.  The points are only formed for steps that may meet an object
// (a disk node or a sphere's angular window inside the step).
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void rk4_step(R M3, R h, R& u, R& v) {
  const R hh = R(0.5) * h;
  const R k1 = accel(M3, u);
  const R v2 = m_fma(hh, k1, v);
  const R k2 = accel(M3, m_fma(hh, v, u));
  const R v3 = m_fma(hh, k2, v);
  const R k3 = accel(M3, m_fma(hh, v2, u));
  const R v4 = m_fma(h, k3, v);
  const R k4 = accel(M3, m_fma(h, v3, u));
  const R h6 = h * R(1.0 / 6.0);
  const R un = m_fma(h6, v + R(2) * (v2 + v3) + v4, u);
  v = m_fma(h6, k1 + R(2) * (k2 + k3) + k4, v);
  u = un;
}

template <typename R>
__device__ __forceinline__ void plane_xy(R phi, R u, R* x, R* y) {
  R s, c;
  m_sincos_evt(phi, &s, &c);
  const R ir = m_div(R(1), u);
  *x = c * ir;
  *y = s * ir;
}

// Objects met by the segment from (xa, ya) to (xb, yb): the smallest
// parameter s in [0, 1] of a disk crossing (z = x e1z + y e2z changes sign,
// radius inside the annulus) or a sphere entry (the sphere's circle in the
// plane).  Returns the event type (-1 for none), *s and the sphere id.
template <typename R>
__device__ int segment_objects(const Params& p, const Ray<R>& r, R xa, R ya, R xb, R yb,
                               bool disk, unsigned sph, R* s_out, unsigned* id_out) {
  const SceneR<R>& S = SR<R>(p.s);
  int best = -1;
  R best_s = R(INFINITY);
  const R dx = xb - xa, dy = yb - ya;
  if (disk) {
    const R za = xa * r.e1z + ya * r.e2z, zb = xb * r.e1z + yb * r.e2z;
    if ((za > R(0) && zb <= R(0)) || (za < R(0) && zb >= R(0))) {
      const R s = m_div(za, za - zb);
      const R X = m_fma(s, dx, xa), Y = m_fma(s, dy, ya);
      const R rr = m_sqrt(m_fma(X, X, Y * Y));
      if (rr >= S.r_in && rr <= S.r_out) {
        best = EV_DISK;
        best_s = s;
      }
    }
  }
  const R dd = m_fma(dx, dx, dy * dy);
  while (sph) {
    const int k = __ffs(sph) - 1;
    sph &= sph - 1;
    const R c0 = S.c[k][0], c1 = S.c[k][1], c2 = S.c[k][2];
    const R cx = c0 * r.e1x + c1 * r.e1y + c2 * r.e1z;
    const R cy = c0 * r.e2x + c1 * r.e2y + c2 * r.e2z;
    const R rp2 = S.rad[k] * S.rad[k] - (S.c2[k] - (cx * cx + cy * cy));  // circle radius^2
    const R ox = xa - cx, oy = ya - cy;
    const R bq = m_fma(ox, dx, oy * dy);
    const R cq = m_fma(ox, ox, oy * oy) - rp2;
    const R disc = bq * bq - dd * cq;
    if (!(disc >= R(0))) continue;
    const R s = m_div(-bq - m_sqrt(disc), dd);
    if (s < R(0) || s > R(1)) continue;
    if (s < best_s || (s == best_s && best != EV_SPHERE)) {
      best = EV_SPHERE;
      best_s = s;
      *id_out = (unsigned)k;
    }
  }
  *s_out = best_s;
  return best;
}

// One fixed step of the polyline method.  Returns true when the ray ended
// (hit filled in for finish_ray: the hit point's plane angle, u = 1/|X| and
// a u' that makes finish_ray's tangent the segment's direction).
template <typename R>
__device__ __forceinline__ bool paper_step(const Params& p, Ray<R>& r, R eps, R u_capt, Hit<R>& hit,
                                           LocalStats& st) {
  const SceneR<R>& S = SR<R>(p.s);
  R un = r.u, vn = r.v;
  rk4_step<R>(S.M3, eps, un, vn);
  r.steps++;
  st.c[ST_STEPS]++;
  if (sizeof(R) == 8) st.c[ST_STEPS64]++;
  // the points lie at phi = k eps: formed from the step count, since a sum
  // of hundreds of FP32 additions of eps drifts by 1e-4 rad
  const R pa = r.phi, pb = R(r.steps) * eps;
  if (un <= R(0)) {
    hit.flags = BH_FLAG_ESC;
    hit.phi = m_fma(eps, m_div(r.u, r.u - un), pa);
    hit.u = R(0);
    hit.v = R(0);
    return true;
  }
  const bool disk = p.s.disk_on && r.phi_node <= pb;
  unsigned sph = 0;
  if (pb >= r.phi_sph) {
    unsigned m = r.sph_mask;
    while (m) {
      const int k = __ffs(m) - 1;
      m &= m - 1;
      float we;
      const float ws = sphere_window(r, k, (float)pa, &we);
      if (R(ws) <= pb && R(we) >= pa) sph |= 1u << k;
    }
  }
  if (disk || sph) {
    st.c[ST_EVENTS]++;
    R xa, ya, xb, yb;
    plane_xy<R>(pa, r.u, &xa, &ya);
    plane_xy<R>(pb, un, &xb, &yb);
    R s;
    unsigned id = 0;
    const int ev = segment_objects<R>(p, r, xa, ya, xb, yb, disk, sph, &s, &id);
    while (r.phi_node <= pb) r.phi_node += Num<R>::pi;
    if (sph) r.phi_sph = next_sphere_window<R>(r, pb);
    if (ev >= 0) {
      const R dx = xb - xa, dy = yb - ya;
      const R X = m_fma(s, dx, xa), Y = m_fma(s, dy, ya);
      const R rr = m_sqrt(m_fma(X, X, Y * Y));
      // the hit angle, continued from pa so that phi mod 2 pi is exact
      const R ph = pa + m_atan2(xa * Y - ya * X, xa * X + ya * Y);
      const R u = m_div(R(1), rr);
      const R cr = m_div(X, rr), sr = m_div(Y, rr);
      const R along = m_fma(dx, cr, dy * sr), across = m_fma(dy, cr, -dx * sr);
      hit.flags = ev == EV_DISK ? BH_FLAG_DISK : (BH_FLAG_SPHERE | (id << 8));
      hit.phi = ph;
      hit.u = u;
      hit.v = across != R(0) ? -u * m_div(along, across) : R(0);
      return true;
    }
  }
  if (un >= u_capt) {
    hit.flags = BH_FLAG_CAPT;
    hit.phi = pb;
    hit.u = un;
    hit.v = vn;
    return true;
  }
  r.u = un;
  r.v = vn;
  r.phi = pb;
  if (r.steps >= p.max_steps || pb >= TolPick<R, sizeof(R) == 8 ? MODE_FP64 : MODE_FP32>::get(p).phi_max) {
    hit.flags = BH_FLAG_STEP_LIMIT;
    hit.phi = pb;
    hit.u = un;
    hit.v = vn;
    return true;
  }
  return false;
}

template <typename R, typename OutR>
__global__ void __launch_bounds__(512, kMinBlocks<R>) k_paper(const __grid_constant__ Params p) {
  constexpr int MODE = sizeof(R) == 8 ? MODE_FP64 : MODE_FP32;
  const R eps = R(p.paper_eps);
  const R u_capt = SR<R>(p.s).M > R(0) ? R(0.5) / SR<R>(p.s).M : R(INFINITY);
  LocalStats st;
  st.zero();
  for_each_grab(p, st, [&](long long q) {
    Ray<R> r;
    SphWin win;
    r.win = &win;
    R b;
    bool active = setup_slot<R, MODE, OutR, false, true>(p, q, r, st, &b);
    if (active) r.steps = 0;
    while (__any_sync(kFull, active)) {
      if (active) {
        Hit<R> hit;
        if (paper_step<R>(p, r, eps, u_capt, hit, st)) {
          finish_ray<R, OutR>(p, r, hit);
          st.count_flag(hit.flags | r.aux);
          active = false;
        }
      }
    }
  });
  st.flush(p.ws);
}

__global__ void k_sky_lut(unsigned long long seed, float4* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= 512) return;
  float rgb[3];
  sky_cell_rgb(seed, c >> 5, c & 31, rgb);
  out[c] = make_float4(rgb[0], rgb[1], rgb[2], 0.0f);
}

// ---------------------------------------------------------------------------
// Host-side launch.
// ---------------------------------------------------------------------------
cudaError_t fill_sky_lut(unsigned long long seed, float4* out, cudaStream_t stream) {
  k_sky_lut<<<4, 128, 0, stream>>>(seed, out);
  return cudaGetLastError();
}

template <typename K>
static int occupancy(K kernel, int block) {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, 0);
  return n > 0 ? n : 1;
}

// Launch `kernel` as the programmatic dependent of the previous kernel on
// `stream` (it must call pdl_wait_primary before reading that kernel's
// results).
template <typename K>
static void launch_dependent(K kernel, int grid, int block, cudaStream_t stream, const Params& p) {
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)grid);
  lc.blockDim = dim3((unsigned)block);
  lc.dynamicSmemBytes = 0;
  lc.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  lc.attrs = attr;
  lc.numAttrs = 1;
  cudaLaunchKernelEx(&lc, kernel, p);
}

cudaError_t launch_render(const Params& p, int mode, const LaunchShape& ls, cudaStream_t stream,
                          cudaEvent_t* ev) {
  // a failure left by earlier, unrelated runtime calls is not this launch's
  cudaGetLastError();
  // while the stream is captured into a graph, timing events must be
  // recorded as external event nodes to carry timestamps at replay
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(stream, &cap);
  const bool capturing = cap == cudaStreamCaptureStatusActive;
  auto record = [&](cudaEvent_t e, cudaStream_t s) {
    if (capturing)
      cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
      cudaEventRecord(e, s);
  };
  const int block = ls.block;
  auto grid_of = [&](auto kernel) {
    const int per_sm = ls.blocks_per_sm > 0 ? ls.blocks_per_sm : occupancy(kernel, block);
    return ls.num_sms * per_sm;
  };
  auto rec = [&](int i) {
    if (ev && ev[i]) record(ev[i], stream);
  };
  rec(0);
  if (mode == MODE_PAPER32 || mode == MODE_PAPER64) {
    if (mode == MODE_PAPER64) {
      auto k = k_paper<double, double>;
      k<<<grid_of(k), block, 0, stream>>>(p);
    } else {
      auto k = k_paper<float, float>;
      k<<<grid_of(k), block, 0, stream>>>(p);
    }
    rec(1);
    rec(2);
    rec(3);
  } else if (p.spp_n > 1) {
    // several samples per pixel: every ray finishes in the tile pass
    if (mode == MODE_FP64) {
      auto k = k_coherent<double, MODE_FP64, double, true>;
      k<<<grid_of(k), block, 0, stream>>>(p);
    } else {
      auto k = k_coherent<float, MODE_FP32, float, true>;
      k<<<grid_of(k), block, 0, stream>>>(p);
    }
    rec(1);
    rec(2);
    rec(3);
  } else if (mode == MODE_FP64) {
    auto k1 = k_coherent<double, MODE_FP64, double>;
    k1<<<grid_of(k1), block, 0, stream>>>(p);
    auto k2 = k_longrays<double, MODE_FP64, double, SRC_SPILL>;
    launch_dependent(k2, grid_of(k2), block, stream, p);
    rec(1);
    rec(2);
    rec(3);
  } else if (mode == MODE_FP32) {
    auto k1 = k_coherent<float, MODE_FP32, float>;
    k1<<<grid_of(k1), block, 0, stream>>>(p);
    auto k2 = k_longrays<float, MODE_FP32, float, SRC_SPILL>;
    launch_dependent(k2, grid_of(k2), block, stream, p);
    rec(1);
    rec(2);
    rec(3);
  } else if (ls.mixed_part == 1) {
    // MIXED band only: the band list and the FP64 band pass
    k_band_list<<<(ls.band_rows + 7) / 8, 256, 0, stream>>>(p, ls.band_row0, ls.band_rows);
    auto k3 = k_longrays<double, MODE_BAND64, float, SRC_BAND>;
    k3<<<ls.band_warps * ls.num_sms, 32, 0, stream>>>(p);
    rec(1);
    rec(2);
    rec(3);
  } else if (ls.mixed_part == 2) {
    // MIXED without the band: the FP32 coherent pass (band pixels skipped)
    // and the long rays, in stream order: the band pass runs on another
    // stream here, and a programmatic dependent's waiting blocks would take
    // the SM room it runs in (measured 11% slower end to end)
    auto k1 = k_coherent<float, MODE_MIXED, float>;
    k1<<<grid_of(k1), block, 0, stream>>>(p);
    auto k2 = k_longrays<float, MODE_MIXED, float, SRC_SPILL>;
    k2<<<grid_of(k2), block, 0, stream>>>(p);
    rec(1);
    rec(2);
    rec(3);
  } else {
    // MIXED: the band list; the FP64 band pass (one-warp blocks, band_warps
    // per SM) as its programmatic dependent, waiting for the list inside; the
    // FP32 coherent pass as the band pass's programmatic dependent, which
    // runs beside it from the frame's start (0.722 -> 0.716 ms at 4096^2,
    // the band list no longer running alone first); then the long rays
    k_band_list<<<(ls.band_rows + 7) / 8, 256, 0, stream>>>(p, ls.band_row0, ls.band_rows);
    auto k3 = k_longrays<double, MODE_BAND64, float, SRC_BAND>;
    launch_dependent(k3, ls.band_warps * ls.num_sms, 32, stream, p);
    auto k1 = k_coherent<float, MODE_MIXED, float>;
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)grid_of(k1));
    lc.blockDim = dim3((unsigned)block);
    lc.dynamicSmemBytes = 0;
    lc.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = 1;
    cudaLaunchKernelEx(&lc, k1, p);
    auto k2 = k_longrays<float, MODE_MIXED, float, SRC_SPILL>;
    launch_dependent(k2, grid_of(k2), block, stream, p);
    rec(1);
    rec(2);
    rec(3);
  }
  return cudaGetLastError();
}

cudaError_t launch_surrogate(const Params& p, const LaunchShape& ls, cudaStream_t stream,
                             cudaEvent_t* ev) {
  cudaGetLastError();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(stream, &cap);
  const bool capturing = cap == cudaStreamCaptureStatusActive;
  auto record = [&](cudaEvent_t e, cudaStream_t s) {
    if (!e) return;
    if (capturing)
      cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
      cudaEventRecord(e, s);
  };
  if (ev) record(ev[0], stream);
  k_band_list<<<(ls.band_rows + 7) / 8, 256, 0, stream>>>(p, ls.band_row0, ls.band_rows);
  cudaEventRecord(ls.fork, stream);
  cudaStreamWaitEvent(ls.side, ls.fork, 0);
  if (ls.band_ev) record(ls.band_ev[0], ls.side);
  auto kb = k_longrays<double, MODE_BAND64, float, SRC_BAND>;
  kb<<<ls.band_warps * ls.num_sms, 32, 0, ls.side>>>(p);
  if (ls.band_ev) record(ls.band_ev[1], ls.side);
  cudaEventRecord(ls.join, ls.side);
  k_surrogate<<<ls.num_sms * 4, 128, sizeof(bhs::TcSmem), stream>>>(p);
  // the integrator finishes the rays the network did not answer; it follows
  // in stream order (as a programmatic dependent its waiting blocks would
  // take the SM room the FP64 band pass runs in)
  if (ev) record(ev[1], stream);
  auto kw = k_listwarp<float, MODE_MIXED, float>;
  kw<<<ls.num_sms * occupancy(kw, ls.block), ls.block, 0, stream>>>(p);
  auto kl = k_longrays<float, MODE_MIXED, float, SRC_SPILL>;
  launch_dependent(kl, ls.num_sms * occupancy(kl, ls.block), ls.block, stream, p);
  if (ev) record(ev[2], stream);
  cudaStreamWaitEvent(stream, ls.join, 0);
  if (ev) record(ev[3], stream);
  return cudaGetLastError();
}

cudaError_t surrogate_kernel_setup() {
  return cudaFuncSetAttribute(k_surrogate, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(bhs::TcSmem));
}

cudaError_t launch_coherent_only(const Params& p, int mode, const LaunchShape& ls,
                                 cudaStream_t stream) {
  const int block = ls.block;
  if (mode == MODE_FP64) {
    auto k = k_coherent<double, MODE_FP64, double>;
    const int per_sm = ls.blocks_per_sm > 0 ? ls.blocks_per_sm : occupancy(k, block);
    k<<<ls.num_sms * per_sm, block, 0, stream>>>(p);
  } else if (mode == MODE_FP32) {
    auto k = k_coherent<float, MODE_FP32, float>;
    const int per_sm = ls.blocks_per_sm > 0 ? ls.blocks_per_sm : occupancy(k, block);
    k<<<ls.num_sms * per_sm, block, 0, stream>>>(p);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace bhk
