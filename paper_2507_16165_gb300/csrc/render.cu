// Persistent render kernels.
//
// The image is cut into 32-ray tiles (tile_w x tile_h pixels, camera-major),
// one tile per warp grab from a global atomic queue.  A warp integrates its 32
// neighbouring rays in lock step (coherent pass); a ray that needs more than
// `budget` attempted steps -- near the photon sphere the step count grows
// like -ln|b - 3 sqrt(3) M| -- is saved to the long-ray list and finished by
// a second persistent kernel whose lanes refill one ray at a time, so one
// slow ray never holds 31 idle lanes.  In MIXED mode rays inside the band
// |b - b_c| < band go to a third list that an FP64 kernel finishes.
#include <cuda_runtime.h>
#include <stdint.h>

#include "render.h"
#include "tracer.cuh"

namespace bhk {

constexpr unsigned kFull = 0xFFFFFFFFu;

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
  const int tile = (int)(l >> 5), i = (int)(l & 31);
  const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
  const int x = tx * p.tile_w + i % p.tile_w;
  const int y = ty * p.tile_h + i / p.tile_w;
  *cam = lo;
  *px = x;
  *py = y;
  *out = (int)(c.out_off + (long long)y * c.w + x);
  return x < c.w && y < c.h;
}

// Straight radial ray (|P x d| ~ 0): spheres by exact ray-sphere
// intersection, otherwise capture (ingoing) or escape along d.
template <typename R, typename OutR>
__device__ void radial_ray(const Params& p, const R P[3], const R d[3], R cos_a, int out,
                           unsigned aux, LocalStats& st) {
  const SceneK& s = p.s;
  R best = R(INFINITY);
  int bk = -1;
  for (int k = 0; k < s.n_sph; ++k) {
    const R o0 = P[0] - R(s.c[k][0]), o1 = P[1] - R(s.c[k][1]), o2 = P[2] - R(s.c[k][2]);
    const R bq = o0 * d[0] + o1 * d[1] + o2 * d[2];
    const R cq = o0 * o0 + o1 * o1 + o2 * o2 - R(s.R[k]) * R(s.R[k]);
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
  const R t_hole = ingoing ? r0 - R(2) * R(s.M) : R(INFINITY);
  unsigned flags;
  if (bk >= 0 && best < t_hole) {
    const R x0 = P[0] + best * d[0], x1 = P[1] + best * d[1], x2 = P[2] + best * d[2];
    const R iR = R(1) / R(s.R[bk]);
    const R N0 = (x0 - R(s.c[bk][0])) * iR, N1 = (x1 - R(s.c[bk][1])) * iR,
            N2 = (x2 - R(s.c[bk][2])) * iR;
    const float lam = 0.25f + 0.75f * fmaxf(0.0f, (float)(-(N0 * d[0] + N1 * d[1] + N2 * d[2])));
    const R ix = R(1) / m_sqrt(x0 * x0 + x1 * x1 + x2 * x2);
    R th, ph;
    dir_angles(x0 * ix, x1 * ix, x2 * ix, &th, &ph);
    flags = BH_FLAG_SPHERE | ((unsigned)bk << 8) | aux;
    store_ray<OutR>(p, out, OutR(th), OutR(ph), flags,
                    pack_rgba(s.alb[bk][0] * lam, s.alb[bk][1] * lam, s.alb[bk][2] * lam));
  } else if (ingoing && s.M > 0.0) {
    flags = BH_FLAG_CAPT | aux;
    store_ray<OutR>(p, out, OutR(NAN), OutR(NAN), flags, 255u << 24);
  } else {
    R th, ph;
    dir_angles(d[0], d[1], d[2], &th, &ph);
    flags = BH_FLAG_ESC | aux;
    store_ray<OutR>(p, out, OutR(th), OutR(ph), flags, sky_rgba<R>(s.seed, th, ph));
  }
  st.count_flag(flags);
}

// Set up the ray of queue slot q.  Returns true when the ray is to be
// integrated by the caller; false when it was padding, finished directly
// (radial) or deferred to the FP64 band list.
template <typename R, int MODE, typename OutR>
__device__ bool setup_slot(const Params& p, long long q, Ray<R>& r, LocalStats& st, R* b_out) {
  int cam, px, py, out;
  if (!slot_pixel(p, q, &cam, &px, &py, &out)) return false;
  const CamK& c = p.cams[cam];
  R P[3], d[3];
  camera_ray<R>(c, px, py, P, d);
  r.out = out;
  r.aux = (MODE == MODE_FP64 || MODE == MODE_BAND64) ? BH_FLAG_FP64 : 0u;
  if (MODE == MODE_BAND64) r.aux |= BH_FLAG_BAND;
  R b, cos_a;
  if (plane_setup<R>(p.s, P, d, R(c.r_obs), r, &b, &cos_a)) {
    radial_ray<R, OutR>(p, P, d, cos_a, out, r.aux, st);
    return false;
  }
  *b_out = b;
  if (MODE == MODE_MIXED) {
    if (m_abs(b - R(p.s.b_crit)) < R(p.band)) {
      const unsigned long long k = atomicAdd(&p.ws->band_count, 1ull);
      p.band_list[k] = (int)q;
      st.c[ST_BAND]++;
      return false;
    }
  }
  r.steps = 0;
  const bool d64 = (MODE == MODE_FP64 || MODE == MODE_BAND64);
  const R rtol = R(d64 && MODE == MODE_BAND64 ? p.rtol64 : p.rtol);
  const R atol = R(d64 && MODE == MODE_BAND64 ? p.atol64 : p.atol);
  r.h = initial_step<R>(R(p.s.M3), r.u, r.v, rtol, atol, R(d64 ? 0.01 : m_min(1.0, p.h_max)));
  return true;
}

// Turning point of the FP32 orbit: v changes sign inside [0, 1] of H.
// Newton on v(t) with dv/dt = h^2 accel(u), from the linear guess.
template <typename R>
__device__ __forceinline__ R turning_t(const Hermite<R>& H, R M3) {
  const R va = H.d0, vb = H.d1;  // h-scaled derivatives at the ends
  R t = va / (va - vb);
  t = m_min(R(1), m_max(R(0), t));
  for (int it = 0; it < 4; ++it) {
    const R g = H.dval_t(t);
    const R dg = H.h * H.h * accel(M3, H.val_t(t));
    if (dg == R(0)) break;
    const R tn = t - g / dg;
    t = m_min(R(1), m_max(R(0), tn));
  }
  return t;
}

// Periastron u_p in FP64: Newton on 2M u^3 - u^2 + E0 = 0 with
// E0 = v0^2 + u0^2 - 2M u0^3 from the FP32 initial state, started at the
// interpolated u (two steps; the reciprocal slope in single precision).
__device__ __forceinline__ double periastron64(double M, double u0, double v0, double ug) {
  const double E0 = v0 * v0 + u0 * u0 - 2.0 * M * u0 * u0 * u0;
  double u = ug;
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const double f = fma(2.0 * M * u, u * u, fma(-u, u, E0));
    const double df = u * fma(6.0 * M, u, -2.0);
    u -= f * (double)(1.0f / (float)df);
  }
  return u;
}

template <typename R>
__device__ __forceinline__ void consider(int type, R ph, unsigned id, int& bt, R& bp, unsigned& bid) {
  const R tie = Num<R>::tie;
  if (bt < 0 || ph < bp - tie ||
      (m_abs(ph - bp) <= tie && (type < bt || (type == bt && id < bid)))) {
    bt = type;
    bp = ph;
    bid = id;
  }
}

enum { EV_CAPT = 0, EV_SPHERE = 1, EV_DISK = 2, EV_ESC = 3 };

// Event handling for an accepted step [pa, pa + h] that may hold an event:
// locate capture / escape roots, disk-node crossings and sphere entries on
// the quintic Hermite interpolant and keep the earliest (ties within
// Num<R>::tie: capture > sphere (lower index) > disk > escape).
template <typename R, int MODE>
__device__ bool step_events(const Params& p, Ray<R>& r, R& un, R& vn, R& fn, R& pb, R h,
                            bool peri, Hit<R>& hit, LocalStats& st) {
  const SceneK& s = p.s;
  const R M3 = R(s.M3);
  const R pa = r.phi;
  Hermite<R> H;
  H.make(pa, h, r.u, r.v, r.f, un, vn, fn);
  if (MODE == MODE_MIXED && peri) {
    // periastron reset: truncate the step at the turning point and put the
    // state back on the orbit of the initial conditions, (u_p, 0) with u_p
    // from the FP64 cubic
    const R tp = turning_t<R>(H, M3);
    const R ug = H.val_t(tp);
    const double up = periastron64(s.M, (double)r.u0, (double)r.v0, (double)ug);
    if (tp > R(0)) {
      const R hp = tp * h;
      pb = pa + hp;
      un = R(up);
      vn = R(0);
      fn = accel(M3, un);
      H.make(pa, hp, r.u, r.v, r.f, un, vn, fn);
    }
    r.aux |= kAuxPeriDone;
    st.c[ST_PERI]++;
  }
  int bt = -1;
  R bp = R(0);
  unsigned bid = 0;
  if (un >= R(s.u_capt)) consider<R>(EV_CAPT, pa + H.h * hermite_root<R>(H, R(s.u_capt), R(0), R(1)), 0u, bt, bp, bid);
  if (un <= R(0)) consider<R>(EV_ESC, pa + H.h * hermite_root<R>(H, R(0), R(0), R(1)), 0u, bt, bp, bid);
  for (int it = 0; it < 8 && r.phi_node <= pb; ++it) {
    const R uk = H.u_at(r.phi_node);
    if (uk > R(0)) {
      const R rk = R(1) / uk;
      if (rk >= R(s.r_in) && rk <= R(s.r_out)) {
        consider<R>(EV_DISK, r.phi_node, 0u, bt, bp, bid);
        break;
      }
    }
    r.phi_node += Num<R>::pi;
  }
  if (pb >= r.phi_sph) {
    unsigned m = r.sph_mask;
    while (m) {
      const int k = __ffs(m) - 1;
      m &= m - 1;
      R ph;
      if (sphere_entry<R>(s, r, k, H, pa, pb, &ph)) consider<R>(EV_SPHERE, ph, (unsigned)k, bt, bp, bid);
    }
    r.phi_sph = next_sphere_window<R>(s, r, pb);
  }
  if (bt < 0) return false;
  hit.phi = bp;
  hit.u = H.u_at(bp);
  hit.v = H.v_at(bp);
  hit.flags = bt == EV_CAPT     ? BH_FLAG_CAPT
              : bt == EV_SPHERE ? (BH_FLAG_SPHERE | (bid << 8))
              : bt == EV_DISK   ? BH_FLAG_DISK
                                : BH_FLAG_ESC;
  return true;
}

// One attempted step.  Returns true when the ray ended (hit filled in).
template <typename R, int MODE>
__device__ __forceinline__ bool advance(const Params& p, Ray<R>& r, Hit<R>& hit, LocalStats& st) {
  const R M3 = R(p.s.M3);
  const R rtol = R(MODE == MODE_BAND64 ? p.rtol64 : p.rtol);
  const R atol = R(MODE == MODE_BAND64 ? p.atol64 : p.atol);
  R un, vn, fn, err2;
  dp5_attempt<R>(M3, r.u, r.v, r.f, r.h, rtol, atol, un, vn, fn, err2);
  r.steps++;
  st.c[ST_STEPS]++;
  if (sizeof(R) == 8) st.c[ST_STEPS64]++;
  const R h = r.h;
  r.h = h * step_factor<R>(err2);
  if (MODE != MODE_BAND64) r.h = m_min(r.h, R(p.h_max));
  if (!(err2 <= R(1))) {
    st.c[ST_REJ]++;
    if (r.steps >= p.max_steps) {
      hit.flags = BH_FLAG_STEP_LIMIT;
      return true;
    }
    return false;
  }
  R pb = r.phi + h;
  bool slow = (un <= R(0)) | (un >= R(p.s.u_capt)) | (pb >= r.phi_node) | (pb >= r.phi_sph);
  bool peri = false;
  if (MODE == MODE_MIXED) {
    peri = p.peri_reset && (r.v > R(0)) && (vn <= R(0)) && !(r.aux & kAuxPeriDone);
    slow |= peri;
  }
  if (slow) {
    st.c[ST_EVENTS]++;
    if (step_events<R, MODE>(p, r, un, vn, fn, pb, h, peri, hit, st)) return true;
  }
  r.u = un;
  r.v = vn;
  r.f = fn;
  r.phi = pb;
  if (r.steps >= p.max_steps || pb >= R(p.phi_max)) {
    hit.flags = BH_FLAG_STEP_LIMIT;
    return true;
  }
  return false;
}

// Coherent pass: one 32-ray tile per warp grab, lanes in lock step, rays
// over the step budget moved to the long-ray list.
template <typename R, int MODE, typename OutR>
__global__ void __launch_bounds__(256) k_coherent(Params p) {
  const int lane = threadIdx.x & 31;
  LocalStats st;
  st.zero();
  for (;;) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&p.ws->q_next, 32ull);
    base = __shfl_sync(kFull, base, 0);
    if (base >= (unsigned long long)p.n_queue) break;
    if (p.abort_after && base >= p.abort_after) {
      if (lane == 0) atomicOr(&p.ws->status, (unsigned)BH_STATUS_ABORTED);
      break;
    }
    if (lane == 0) st.c[ST_GRABS]++;
    const long long q = (long long)base + lane;
    Ray<R> r;
    R b;
    bool active = (q < p.n_queue) && setup_slot<R, MODE, OutR>(p, q, r, st, &b);
    while (__any_sync(kFull, active)) {
      if (active) {
        Hit<R> hit;
        if (advance<R, MODE>(p, r, hit, st)) {
          finish_ray<R, OutR>(p, r, hit);
          st.count_flag(hit.flags | r.aux);
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
  }
  st.flush(p.ws);
}

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
    r.f = accel(R(p.s.M3), r.u);
    for (int it = 0; it < 64 && r.phi_node <= r.phi; ++it) r.phi_node += Num<R>::pi;
    if (r.sph_mask) r.phi_sph = next_sphere_window<R>(p.s, r, r.phi);
  }
  return true;
}

// Long-ray pass: every lane refills on its own from a list (saved long
// rays, or FP64 band rays), warp-aggregated: one atomic per refill round.
template <typename R, int MODE, typename OutR, bool FROM_SPILL>
__global__ void __launch_bounds__(256) k_longrays(Params p) {
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned long long* next = FROM_SPILL ? &p.ws->long_next : &p.ws->band_next;
  const unsigned long long total =
      FROM_SPILL ? *(volatile unsigned long long*)&p.ws->long_count
                 : *(volatile unsigned long long*)&p.ws->band_count;
  LocalStats st;
  st.zero();
  Ray<R> r;
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
              active = restore_ray<R, MODE, OutR>(p, p.band_list[idx], nullptr, r, st);
              if (active) st.c[ST_BAND] += 0;
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
  st.flush(p.ws);
}

// ---------------------------------------------------------------------------
// Host-side launch.
// ---------------------------------------------------------------------------
template <typename K>
static int occupancy(K kernel, int block) {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, 0);
  return n > 0 ? n : 1;
}

cudaError_t launch_render(const Params& p, int mode, const LaunchShape& ls, cudaStream_t stream,
                          cudaEvent_t* ev) {
  const int block = ls.block;
  auto grid_of = [&](auto kernel) {
    const int per_sm = ls.blocks_per_sm > 0 ? ls.blocks_per_sm : occupancy(kernel, block);
    return ls.num_sms * per_sm;
  };
  auto rec = [&](int i) {
    if (ev && ev[i]) cudaEventRecord(ev[i], stream);
  };
  rec(0);
  if (mode == MODE_FP64) {
    auto k1 = k_coherent<double, MODE_FP64, double>;
    k1<<<grid_of(k1), block, 0, stream>>>(p);
    rec(1);
    auto k2 = k_longrays<double, MODE_FP64, double, true>;
    k2<<<grid_of(k2), block, 0, stream>>>(p);
    rec(2);
    rec(3);
  } else if (mode == MODE_FP32) {
    auto k1 = k_coherent<float, MODE_FP32, float>;
    k1<<<grid_of(k1), block, 0, stream>>>(p);
    rec(1);
    auto k2 = k_longrays<float, MODE_FP32, float, true>;
    k2<<<grid_of(k2), block, 0, stream>>>(p);
    rec(2);
    rec(3);
  } else {
    auto k1 = k_coherent<float, MODE_MIXED, float>;
    k1<<<grid_of(k1), block, 0, stream>>>(p);
    rec(1);
    auto k2 = k_longrays<float, MODE_MIXED, float, true>;
    k2<<<grid_of(k2), block, 0, stream>>>(p);
    rec(2);
    auto k3 = k_longrays<double, MODE_BAND64, float, false>;
    k3<<<grid_of(k3), block, 0, stream>>>(p);
    rec(3);
  }
  return cudaGetLastError();
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
