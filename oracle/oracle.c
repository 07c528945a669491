/*
 * Plain FP64 CPU oracle for the Schwarzschild light-ray renderer.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no source, header, table or helper
 * with the CUDA path.
 *
 * What it computes (paper: Naddell & Ponce, "Parallel Ray Tracing of Black
 * Hole Images Using the Schwarzschild Metric", PEARC '25):
 *   - one ray per pixel of a pinhole camera (Sec. 1, last paragraph);
 *   - the ray is reduced to its orbital plane through the hole and the
 *     photon-orbit equation in u = 1/r against the azimuth phi (Sec. 1, Eq. 1)
 *     is integrated from initial conditions at the camera (Sec. 2.2).
 *     Eq. 1 is printed as u'' - u = 3Mu^2; differentiating the first integral
 *     (u')^2 + u^2 - 2Mu^3 = 1/b^2 gives u'' = 3Mu^2 - u, which is the form
 *     used here (the printed sign would give cosh-type, not straight, rays at
 *     M = 0);
 *   - the paper's fixed step epsilon with an unnamed GSL stepper (Sec. 2.2)
 *     is replaced by adaptive Dormand-Prince 5(4) with the Hairer-Norsett-
 *     Wanner error norm and step controller; the paper's piecewise-linear
 *     segments (Sec. 2.1) are replaced by exact event location on the
 *     quintic Hermite interpolant of each accepted step;
 *   - the paper's own fixed-step polyline is kept as method 1 (classical
 *     Runge-Kutta at a fixed step eps, segment intersection), to measure
 *     that approach against the adaptive one;
 *   - events: escape (u -> 0), capture (u >= 1/(2M)), thin equatorial disk
 *     annulus, opaque spheres; the result is mapped back to 3-D and shaded
 *     against a procedural checkerboard sky.
 * Every step below is written plainly: no blocking, no fusion, bisection
 * for every root, 64-bit floating point throughout.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_MAX_SPHERES 8

/* outcome flags (bit layout shared with the renderer's documented C-ABI) */
#define OR_ESC 1u
#define OR_CAPT 2u
#define OR_DISK 4u
#define OR_SPHERE 8u
#define OR_STEP_LIMIT 128u

/* ambiguity mask bits: outputs that a correct renderer at a given precision
 * may legitimately decide the other way */
#define OR_AMB_CAPT 1u    /* |b - 3 sqrt(3) M| < eps_b                      */
#define OR_AMB_DISK 2u    /* a node crossing within eps_r of r_in or r_out  */
#define OR_AMB_SPHERE 4u  /* a sphere passage grazing within eps_r          */
#define OR_AMB_SKY 8u     /* exit direction within eps_ang of a cell edge   */
#define OR_AMB_DEGEN 16u  /* radial ray or orbit lying in the disk plane    */

typedef struct {
  double c[3];
  double radius;
  double albedo[3];
} or_sphere;

typedef struct {
  double mass;
  int disk_enabled;
  double disk_r_in, disk_r_out;
  int n_spheres;
  or_sphere spheres[OR_MAX_SPHERES];
  uint64_t sky_seed;
  int ic; /* 0 = static observer, 1 = Euclidean ("linear direction") */
  /* optional sky image (Sec. 3.1 renders photographs as the background):
   * equirectangular RGBA8, row j at theta = (j + 1/2) pi / h from the +z
   * pole, column i at phi = (i + 1/2) 2 pi / w; NULL: procedural checker */
  const uint32_t *sky_tex;
  int sky_w, sky_h;
} or_scene;

typedef struct {
  double r_obs, incl_deg, azim_deg, fov_deg;
  int w, h;
} or_camera;

typedef struct {
  double rtol, atol;
  double phi_max;
  long max_steps;
  double eps_r, eps_ang, eps_b; /* ambiguity thresholds */
  int method;  /* 0: Dormand-Prince 5(4) with exact events; 1: the paper's
                  fixed-step polyline (Sec. 2.1-2.2) */
  double eps;  /* step in phi of method 1 */
  int spp_n;   /* samples per pixel side: n x n stratified samples (<= 1: one) */
  int doppler; /* 1: Keplerian disk with Doppler and gravitational shift */
} or_opts;

typedef struct {
  unsigned flags;
  unsigned sphere_id;
  unsigned ambig;
  double theta, phi; /* output direction (NaN when captured) */
  double rgb[3];
  double b;
  long steps; /* attempted steps */
} or_pixel;

/* ------------------------------------------------------------------ */
/* Small 3-vector helpers                                              */
/* ------------------------------------------------------------------ */
static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void cross3(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------ */
/* The ODE: Eq. 1 with the sign fixed by the first integral            */
/*   y = (u, v = du/dphi),  y' = (v, 3 M u^2 - u)                     */
/* ------------------------------------------------------------------ */
static double accel(double M, double u) { return 3.0 * M * u * u - u; }

/* ------------------------------------------------------------------ */
/* Dormand-Prince 5(4) coefficients (Dormand & Prince 1980, RK5(4)7M). */
/* ------------------------------------------------------------------ */
static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};
/* fifth-order weights = last row of A (first-same-as-last) */
static const double DP_B5[7] = {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192,
                                -2187.0 / 6784, 11.0 / 84, 0};
/* embedded fourth-order weights */
static const double DP_B4[7] = {5179.0 / 57600, 0, 7571.0 / 16695, 393.0 / 640,
                                -92097.0 / 339200, 187.0 / 2100, 1.0 / 40};

/* One Dormand-Prince attempt from (u, v) with step h.  Returns the
 * fifth-order solution, the Hairer error norm and the derivative at the new
 * point (stage 7, reused as stage 1 of the next step). */
static void dp5_attempt(double M, double u, double v, double h, double rtol,
                        double atol, double *un, double *vn, double *err) {
  double ku[7], kv[7];
  for (int s = 0; s < 7; ++s) {
    double us = u, vs = v;
    for (int j = 0; j < s; ++j) {
      us += h * DP_A[s][j] * ku[j];
      vs += h * DP_A[s][j] * kv[j];
    }
    ku[s] = vs;
    kv[s] = accel(M, us);
    (void)DP_C;
  }
  double u5 = u, v5 = v, u4 = u, v4 = v;
  for (int s = 0; s < 7; ++s) {
    u5 += h * DP_B5[s] * ku[s];
    v5 += h * DP_B5[s] * kv[s];
    u4 += h * DP_B4[s] * ku[s];
    v4 += h * DP_B4[s] * kv[s];
  }
  double scu = atol + rtol * fmax(fabs(u), fabs(u5));
  double scv = atol + rtol * fmax(fabs(v), fabs(v5));
  double eu = (u5 - u4) / scu, ev = (v5 - v4) / scv;
  *err = sqrt(0.5 * (eu * eu + ev * ev));
  *un = u5;
  *vn = v5;
}

/* Starting step: Hairer, Norsett & Wanner, Solving ODEs I, Sec. II.4,
 * capped at 0.01 rad. */
static double initial_step(double M, double u, double v, double rtol,
                           double atol) {
  double scu = atol + rtol * fabs(u), scv = atol + rtol * fabs(v);
  double fu = v, fv = accel(M, u);
  double d0 = sqrt(0.5 * ((u / scu) * (u / scu) + (v / scv) * (v / scv)));
  double d1 = sqrt(0.5 * ((fu / scu) * (fu / scu) + (fv / scv) * (fv / scv)));
  double h0 = (d0 < 1e-5 || d1 < 1e-5) ? 1e-6 : 0.01 * d0 / d1;
  double u1 = u + h0 * fu, v1 = v + h0 * fv;
  double gu = v1 - fu, gv = accel(M, u1) - fv;
  double d2 = sqrt(0.5 * ((gu / scu) * (gu / scu) + (gv / scv) * (gv / scv))) / h0;
  double dm = fmax(d1, d2);
  double h1 = (dm <= 1e-15) ? fmax(1e-6, h0 * 1e-3) : pow(0.01 / dm, 1.0 / 5.0);
  double h = fmin(100.0 * h0, h1);
  return fmin(h, 0.01);
}

/* Step-size update: h <- h * min(10, max(0.2, 0.9 err^(-1/5))); after a
 * rejection the factor is also capped at 1. */
static double next_step(double h, double err, int accepted) {
  double fac = (err > 0.0) ? 0.9 * pow(err, -0.2) : 10.0;
  if (fac > 10.0) fac = 10.0;
  if (fac < 0.2) fac = 0.2;
  if (!accepted && fac > 1.0) fac = 1.0;
  return h * fac;
}

/* ------------------------------------------------------------------ */
/* Quintic Hermite interpolant of u on an accepted step [pa, pa + h],  */
/* built from u, u' = v and u'' = 3Mu^2 - u at both ends.              */
/* ------------------------------------------------------------------ */
typedef struct {
  double pa, h;
  double u0, d0, s0, u1, d1, s1; /* values, h*u', h^2*u'' */
} hermite5;

static void hermite_make(hermite5 *H, double M, double pa, double h, double ua,
                         double va, double ub, double vb) {
  H->pa = pa;
  H->h = h;
  H->u0 = ua;
  H->d0 = h * va;
  H->s0 = h * h * accel(M, ua);
  H->u1 = ub;
  H->d1 = h * vb;
  H->s1 = h * h * accel(M, ub);
}

static double hermite_u(const hermite5 *H, double phi) {
  double t = (phi - H->pa) / H->h;
  double t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
  double h0 = 1 - 10 * t3 + 15 * t4 - 6 * t5;
  double h1 = t - 6 * t3 + 8 * t4 - 3 * t5;
  double h2 = 0.5 * (t2 - 3 * t3 + 3 * t4 - t5);
  double h3 = 10 * t3 - 15 * t4 + 6 * t5;
  double h4 = -4 * t3 + 7 * t4 - 3 * t5;
  double h5 = 0.5 * (t3 - 2 * t4 + t5);
  return H->u0 * h0 + H->d0 * h1 + H->s0 * h2 + H->u1 * h3 + H->d1 * h4 +
         H->s1 * h5;
}

/* du/dphi of the interpolant */
static double hermite_v(const hermite5 *H, double phi) {
  double t = (phi - H->pa) / H->h;
  double t2 = t * t, t3 = t2 * t, t4 = t3 * t;
  double h0 = -30 * t2 + 60 * t3 - 30 * t4;
  double h1 = 1 - 18 * t2 + 32 * t3 - 15 * t4;
  double h2 = 0.5 * (2 * t - 9 * t2 + 12 * t3 - 5 * t4);
  double h3 = 30 * t2 - 60 * t3 + 30 * t4;
  double h4 = -12 * t2 + 28 * t3 - 15 * t4;
  double h5 = 0.5 * (3 * t2 - 8 * t3 + 5 * t4);
  return (H->u0 * h0 + H->d0 * h1 + H->s0 * h2 + H->u1 * h3 + H->d1 * h4 +
          H->s1 * h5) /
         H->h;
}

/* Root of hermite_u(phi) - target on [lo, hi] given a sign change, by plain
 * bisection down to adjacent doubles. */
static double hermite_root(const hermite5 *H, double target, double lo,
                           double hi) {
  double flo = hermite_u(H, lo) - target;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double fm = hermite_u(H, mid) - target;
    if ((fm > 0) == (flo > 0) && fm != 0.0) {
      lo = mid;
      flo = fm;
    } else {
      hi = mid;
    }
  }
  return hi;
}

/* ------------------------------------------------------------------ */
/* Plane geometry of one ray                                            */
/* ------------------------------------------------------------------ */
typedef struct {
  double e1[3], e2[3], n[3];
  double u0, v0, b, sin_a, cos_a;
  int radial;
  /* disk nodes */
  int disk_in_plane; /* orbit plane == disk plane */
  double psi0;       /* first node angle in [0, pi) */
  /* spheres cut by the plane */
  int sph_on[OR_MAX_SPHERES];
  double sph_cx[OR_MAX_SPHERES], sph_cy[OR_MAX_SPHERES];
  double sph_k[OR_MAX_SPHERES]; /* |c|^2 - R^2 */
  double sph_rp[OR_MAX_SPHERES]; /* in-plane circle radius R' */
  double sph_phic[OR_MAX_SPHERES], sph_dphi[OR_MAX_SPHERES];
} or_plane;

/* Pinhole camera: observer at P = r_obs (sin i cos a, sin i sin a, cos i),
 * looking at the hole, up = world +z projected (world +x when looking along
 * z), pixel centres, row 0 at the top, FOV across the full width. */
static void camera_ray(const or_camera *cam, double px, double py, double P[3],
                       double d[3]) {
  double inc = cam->incl_deg * OR_PI / 180.0, az = cam->azim_deg * OR_PI / 180.0;
  P[0] = cam->r_obs * sin(inc) * cos(az);
  P[1] = cam->r_obs * sin(inc) * sin(az);
  P[2] = cam->r_obs * cos(inc);
  double f[3] = {-P[0] / cam->r_obs, -P[1] / cam->r_obs, -P[2] / cam->r_obs};
  double upw[3] = {0, 0, 1}, right[3], up[3];
  cross3(f, upw, right);
  if (norm3(right) < 1e-12) {
    upw[0] = 1;
    upw[1] = 0;
    upw[2] = 0;
    cross3(f, upw, right);
  }
  double nr = norm3(right);
  for (int k = 0; k < 3; ++k) right[k] /= nr;
  cross3(right, f, up);
  double th = tan(0.5 * cam->fov_deg * OR_PI / 180.0);
  double sx = (2.0 * (px + 0.5) / cam->w - 1.0) * th;
  double sy = (1.0 - 2.0 * (py + 0.5) / cam->h) * th * ((double)cam->h / cam->w);
  double dd[3];
  for (int k = 0; k < 3; ++k) dd[k] = f[k] + sx * right[k] + sy * up[k];
  double nd = norm3(dd);
  for (int k = 0; k < 3; ++k) d[k] = dd[k] / nd;
}

/* Orbital-plane reduction: e1 along the observer, e2 completing the plane
 * of (P, d), impact parameter b and initial (u, u'). */
static void plane_reduce(const or_scene *sc, const double P[3],
                         const double d[3], or_plane *pl) {
  double M = sc->mass;
  double r = norm3(P);
  for (int k = 0; k < 3; ++k) pl->e1[k] = P[k] / r;
  double cr[3];
  cross3(P, d, cr);
  double s = norm3(cr);
  pl->cos_a = dot3(d, pl->e1);
  pl->u0 = 1.0 / r;
  pl->radial = (s < 1e-12 * r);
  if (pl->radial) {
    pl->sin_a = 0.0;
    pl->b = 0.0;
    pl->v0 = 0.0;
    return;
  }
  for (int k = 0; k < 3; ++k) pl->n[k] = cr[k] / s;
  cross3(pl->n, pl->e1, pl->e2);
  pl->sin_a = dot3(d, pl->e2);
  double cot = pl->cos_a / pl->sin_a;
  if (sc->ic == 0) {
    /* static observer: sin(alpha) = b sqrt(1 - 2M/r) / r */
    pl->b = r * pl->sin_a / sqrt(1.0 - 2.0 * M / r);
    pl->v0 = -pl->u0 * cot * sqrt(1.0 - 2.0 * M * pl->u0);
  } else {
    /* Euclidean: successor point along the straight camera direction */
    pl->b = r * pl->sin_a / sqrt(1.0 - 2.0 * M * pl->sin_a * pl->sin_a / r);
    pl->v0 = -pl->u0 * cot;
  }
  /* disk nodes: z(phi) proportional to cos(phi) e1z + sin(phi) e2z */
  double a = pl->e1[2], c = pl->e2[2];
  pl->disk_in_plane = (a * a + c * c < 1e-24);
  if (!pl->disk_in_plane) {
    double p0 = atan2(-a, c);
    if (p0 < 0) p0 += OR_PI;
    if (p0 >= OR_PI) p0 -= OR_PI;
    pl->psi0 = p0;
  } else {
    pl->psi0 = 0.0;
  }
  for (int k = 0; k < sc->n_spheres; ++k) {
    const or_sphere *S = &sc->spheres[k];
    double sd = dot3(pl->n, S->c);
    pl->sph_on[k] = fabs(sd) < S->radius;
    if (!pl->sph_on[k]) continue;
    double rp = sqrt(S->radius * S->radius - sd * sd);
    double cx = dot3(S->c, pl->e1), cy = dot3(S->c, pl->e2);
    double rho = sqrt(cx * cx + cy * cy);
    double pc = atan2(cy, cx);
    if (pc < 0) pc += 2 * OR_PI;
    pl->sph_cx[k] = cx;
    pl->sph_cy[k] = cy;
    pl->sph_rp[k] = rp;
    pl->sph_k[k] = dot3(S->c, S->c) - S->radius * S->radius;
    pl->sph_phic[k] = pc;
    pl->sph_dphi[k] = asin(fmin(1.0, rp / rho));
  }
}

/* g < 0 inside the sphere's in-plane circle: u^2 (|p - c'|^2 - R'^2) */
static double sphere_g(const or_plane *pl, int k, double phi, double u) {
  return 1.0 - 2.0 * u * (pl->sph_cx[k] * cos(phi) + pl->sph_cy[k] * sin(phi)) +
         pl->sph_k[k] * u * u;
}

/* First entry into sphere k's in-plane circle during the accepted step,
 * restricted to the step's overlap with the sphere's angular window
 * [phi_c - dphi, phi_c + dphi] (mod 2 pi).  g is sampled at 17 points, its
 * minimum refined by golden-section search, and the entry located by
 * bisection.  Returns 1 and the entry angle if entered. */
static int sphere_entry(const or_plane *pl, int k, const hermite5 *H, double pa,
                        double pb, double eps_r, unsigned *ambig,
                        double *phi_hit) {
  double pc = pl->sph_phic[k], dp = pl->sph_dphi[k];
  double two_pi = 2 * OR_PI;
  double m = ceil((pa - pc - dp) / two_pi);
  double ws = pc - dp + two_pi * m, we = pc + dp + two_pi * m;
  if (ws > pb || we < pa) return 0;
  double lo = fmax(pa, ws), hi = fmin(pb, we);
  if (!(hi > lo)) return 0;
  enum { NS = 16 };
  double ph[NS + 1], g[NS + 1];
  for (int i = 0; i <= NS; ++i) {
    ph[i] = lo + (hi - lo) * i / NS;
    g[i] = sphere_g(pl, k, ph[i], hermite_u(H, ph[i]));
  }
  /* minimum of g over the interval */
  int j = 0;
  for (int i = 1; i <= NS; ++i)
    if (g[i] < g[j]) j = i;
  double x0 = ph[j > 0 ? j - 1 : 0], x3 = ph[j < NS ? j + 1 : NS];
  const double gr = 0.6180339887498949;
  double x1 = x3 - gr * (x3 - x0), x2 = x0 + gr * (x3 - x0);
  double g1 = sphere_g(pl, k, x1, hermite_u(H, x1));
  double g2 = sphere_g(pl, k, x2, hermite_u(H, x2));
  for (int it = 0; it < 200 && (x3 - x0) > 1e-15 * (1 + fabs(x3)); ++it) {
    if (g1 < g2) {
      x3 = x2;
      x2 = x1;
      g2 = g1;
      x1 = x3 - gr * (x3 - x0);
      g1 = sphere_g(pl, k, x1, hermite_u(H, x1));
    } else {
      x0 = x1;
      x1 = x2;
      g1 = g2;
      x2 = x0 + gr * (x3 - x0);
      g2 = sphere_g(pl, k, x2, hermite_u(H, x2));
    }
  }
  double xm = 0.5 * (x0 + x3);
  double gm = sphere_g(pl, k, xm, hermite_u(H, xm));
  if (g[j] < gm) {
    xm = ph[j];
    gm = g[j];
  }
  {
    /* closest approach minus R' from g = u^2 (d^2 - R'^2) */
    double um = hermite_u(H, xm);
    double gap = fabs(gm) / (um * um * 2.0 * pl->sph_rp[k]);
    if (gap < eps_r) *ambig |= OR_AMB_SPHERE;
  }
  if (gm > 0) return 0;
  int first_in = -1;
  for (int i = 0; i <= NS; ++i)
    if (g[i] <= 0) {
      first_in = i;
      break;
    }
  if (first_in == 0) {
    *phi_hit = ph[0];
    return 1;
  }
  double a_lo, a_hi; /* bracket with g(a_lo) > 0 >= g(a_hi) */
  if (first_in > 0) {
    a_lo = ph[first_in - 1];
    a_hi = ph[first_in];
  } else {
    /* all samples outside, the refined minimum inside: the sample left of
     * the minimum is outside */
    int jl = 0;
    for (int i = 0; i <= NS; ++i)
      if (ph[i] < xm) jl = i;
    a_lo = ph[jl];
    a_hi = xm;
  }
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (a_lo + a_hi);
    if (mid <= a_lo || mid >= a_hi) break;
    if (sphere_g(pl, k, mid, hermite_u(H, mid)) > 0)
      a_lo = mid;
    else
      a_hi = mid;
  }
  *phi_hit = a_hi;
  return 1;
}

/* ------------------------------------------------------------------ */
/* Trace one ray in its plane                                           */
/* ------------------------------------------------------------------ */
typedef struct {
  unsigned flags, sphere_id, ambig;
  double phi_evt, u_evt, v_evt;
  long steps;
} or_event;

enum { EV_CAPT = 0, EV_SPHERE = 1, EV_DISK = 2, EV_ESC = 3 };

static void trace_plane(const or_scene *sc, const or_opts *o,
                        const or_plane *pl, or_event *ev) {
  double M = sc->mass;
  double u = pl->u0, v = pl->v0, phi = 0.0;
  double u_capt = (M > 0) ? 1.0 / (2.0 * M) : INFINITY;
  double h = initial_step(M, u, v, o->rtol, o->atol);
  long steps = 0;
  int disk_k = 0; /* index of the next node: phi_k = psi0 + k pi > 0 */
  if (sc->disk_enabled && !pl->disk_in_plane && !(pl->psi0 > 0)) disk_k = 1;
  ev->ambig = 0;
  ev->sphere_id = 0;
  for (;;) {
    if (steps >= o->max_steps || phi >= o->phi_max) {
      ev->flags = OR_STEP_LIMIT;
      ev->phi_evt = phi;
      ev->u_evt = u;
      ev->v_evt = v;
      ev->steps = steps;
      return;
    }
    double un, vn, err;
    dp5_attempt(M, u, v, h, o->rtol, o->atol, &un, &vn, &err);
    ++steps;
    if (!(err <= 1.0)) {
      h = next_step(h, err, 0);
      continue;
    }
    double pa = phi, pb = phi + h;
    hermite5 H;
    hermite_make(&H, M, pa, h, u, v, un, vn);
    /* candidate events in this step */
    int best = -1;
    double best_phi = INFINITY;
    unsigned best_id = 0;
#define OR_CONSIDER(type, ph, id)                                            \
  do {                                                                       \
    double _p = (ph);                                                        \
    if (best < 0 || _p < best_phi - 1e-12 ||                                 \
        (fabs(_p - best_phi) <= 1e-12 &&                                     \
         ((type) < best || ((type) == best && (id) < best_id)))) {           \
      best = (type);                                                         \
      best_phi = _p;                                                         \
      best_id = (id);                                                        \
    }                                                                        \
  } while (0)
    if (un >= u_capt) OR_CONSIDER(EV_CAPT, hermite_root(&H, u_capt, pa, pb), 0u);
    if (un <= 0.0) OR_CONSIDER(EV_ESC, hermite_root(&H, 0.0, pa, pb), 0u);
    if (sc->disk_enabled && !pl->disk_in_plane) {
      for (;;) {
        double pk = pl->psi0 + disk_k * OR_PI;
        if (pk > pb) break;
        double uk = hermite_u(&H, pk);
        if (uk > 0) {
          double rk = 1.0 / uk;
          if (fabs(rk - sc->disk_r_in) < o->eps_r ||
              fabs(rk - sc->disk_r_out) < o->eps_r)
            ev->ambig |= OR_AMB_DISK;
          if (rk >= sc->disk_r_in && rk <= sc->disk_r_out) {
            OR_CONSIDER(EV_DISK, pk, 0u);
            break;
          }
        }
        ++disk_k;
      }
    }
    for (int k = 0; k < sc->n_spheres; ++k) {
      if (!pl->sph_on[k]) continue;
      double ph;
      if (sphere_entry(pl, k, &H, pa, pb, o->eps_r, &ev->ambig, &ph))
        OR_CONSIDER(EV_SPHERE, ph, (unsigned)k);
    }
#undef OR_CONSIDER
    if (best >= 0) {
      ev->phi_evt = best_phi;
      ev->u_evt = hermite_u(&H, best_phi);
      ev->v_evt = hermite_v(&H, best_phi);
      ev->steps = steps;
      ev->sphere_id = best_id;
      ev->flags = best == EV_CAPT     ? OR_CAPT
                  : best == EV_SPHERE ? OR_SPHERE
                  : best == EV_DISK   ? OR_DISK
                                      : OR_ESC;
      return;
    }
    u = un;
    v = vn;
    phi = pb;
    h = next_step(h, err, 1);
  }
}

/* ------------------------------------------------------------------ */
/* Shading                                                              */
/* ------------------------------------------------------------------ */
/* splitmix64 (Steele, Lea & Flood 2014): output for state x */
static uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* 16 x 32 checkerboard in (theta, phi), two base colours, per-cell tint */
static void sky_rgb(uint64_t seed, double theta, double phi, double rgb[3]) {
  int i = (int)floor(16.0 * theta / OR_PI);
  int j = (int)floor(32.0 * phi / (2.0 * OR_PI));
  if (i > 15) i = 15;
  if (i < 0) i = 0;
  if (j > 31) j = 31;
  if (j < 0) j = 0;
  static const double base[2][3] = {{0.9, 0.9, 0.9}, {0.1, 0.1, 0.25}};
  const double *bc = base[(i + j) & 1];
  uint64_t hsh = splitmix64(seed * 2654435761ull + (uint64_t)(32 * i + j));
  for (int c = 0; c < 3; ++c) {
    double slice = (double)((hsh >> (16 * c)) & 0xFFFFFFull);
    rgb[c] = bc[c] * (0.75 + 0.25 * slice / 16777216.0);
  }
}

/* Background colour in direction (theta, phi): the sky image, bilinear in
 * linear colour between the four nearest texel centres (wrapping in phi,
 * clamped at the poles), or the procedural checker. */
static void sky_colour(const or_scene *sc, double theta, double phi, double rgb[3]) {
  if (!sc->sky_tex) {
    sky_rgb(sc->sky_seed, theta, phi, rgb);
    return;
  }
  int W = sc->sky_w, H = sc->sky_h;
  double x = phi / (2.0 * OR_PI) * W - 0.5, y = theta / OR_PI * H - 0.5;
  double fx0 = floor(x), fy0 = floor(y);
  double fx = x - fx0, fy = y - fy0;
  long i0 = (long)fx0, j0 = (long)fy0;
  long ia = ((i0 % W) + W) % W, ib = (((i0 + 1) % W) + W) % W;
  long ja = j0 < 0 ? 0 : (j0 > H - 1 ? H - 1 : j0);
  long jb = j0 + 1 < 0 ? 0 : (j0 + 1 > H - 1 ? H - 1 : j0 + 1);
  uint32_t t00 = sc->sky_tex[ja * W + ia], t10 = sc->sky_tex[ja * W + ib];
  uint32_t t01 = sc->sky_tex[jb * W + ia], t11 = sc->sky_tex[jb * W + ib];
  for (int c = 0; c < 3; ++c) {
    double c00 = ((t00 >> (8 * c)) & 255) / 255.0, c10 = ((t10 >> (8 * c)) & 255) / 255.0;
    double c01 = ((t01 >> (8 * c)) & 255) / 255.0, c11 = ((t11 >> (8 * c)) & 255) / 255.0;
    rgb[c] = (1.0 - fy) * ((1.0 - fx) * c00 + fx * c10) + fy * ((1.0 - fx) * c01 + fx * c11);
  }
}

static int near_cell_edge(double theta, double phi, double eps) {
  double ti = 16.0 * theta / OR_PI;
  double dt = fabs(ti - floor(ti + 0.5)) * OR_PI / 16.0;
  if (dt < eps) return 1;
  double pj = 32.0 * phi / (2.0 * OR_PI);
  double dp = fabs(pj - floor(pj + 0.5)) * (2.0 * OR_PI / 32.0);
  return dp * sin(theta) < eps;
}

static unsigned quant8(double c) {
  double q = floor(255.0 * c + 0.5);
  if (q > 255) q = 255;
  if (q < 0) q = 0;
  return (unsigned)q;
}

static void dir_angles(const double d[3], double *theta, double *phi) {
  double z = d[2];
  if (z > 1) z = 1;
  if (z < -1) z = -1;
  *theta = acos(z);
  double p = atan2(d[1], d[0]);
  if (p < 0) p += 2 * OR_PI;
  *phi = p;
}

/* ------------------------------------------------------------------ */
/* One pixel: the whole path                                            */
/* ------------------------------------------------------------------ */
/* Thin-disk temperature ramp at radius r: t = (r_in / r)^(3/4). */
static void disk_rgb(const or_scene *sc, double r, double rgb[3]) {
  double t = pow(sc->disk_r_in / r, 0.75);
  double k = 0.3 + 0.7 * t;
  rgb[0] = 1.0 * k;
  rgb[1] = (0.35 + 0.65 * t) * k;
  rgb[2] = (0.1 + 0.9 * t * t) * k;
}

/* Keplerian disk seen by the static camera at r_obs: the frequency ratio
 * g = nu_camera / nu_emitted of a photon reaching the camera from the disk
 * point x (r = |x|, in the equatorial plane).  Worked in the local static
 * frame at x: the gas moves on a prograde circular orbit (about +z) with
 * speed beta = sqrt(M / (r - 2M)); the photon arrives along the unit vector
 * kin, minus the traced ray's direction; with local frame components
 * (radial scaled by 1/sqrt(1 - 2M/r)), the emitted energy in the static
 * frame is gamma (1 - beta kin.phi_hat) times the gas frame's, and static
 * energies at r and r_obs differ by sqrt(1 - 2M/r) / sqrt(1 - 2M/r_obs).
 * Inside r = 3M there is no circular orbit: g = 0. */
static double disk_g(double M, double r_obs, const double x[3], const double xr_dir[3],
                     double dr_dphi, const double t_dir[3], double r) {
  if (!(r > 3.0 * M)) return 0.0;
  double f = 1.0 - 2.0 * M / r;
  /* traced direction in the local orthonormal static frame: radial part
   * (dr/dphi) / sqrt(f), tangential part r (per unit dphi) */
  double kr = dr_dphi / sqrt(f), kt = r;
  double nk = sqrt(kr * kr + kt * kt);
  double kin[3];
  for (int k = 0; k < 3; ++k) kin[k] = -(kr * xr_dir[k] + kt * t_dir[k]) / nk;
  /* prograde azimuthal direction about +z at x */
  double ph[3] = {-x[1], x[0], 0.0};
  double nph = norm3(ph);
  for (int k = 0; k < 3; ++k) ph[k] /= nph;
  double beta = sqrt(M / (r - 2.0 * M));
  double gamma = 1.0 / sqrt(1.0 - beta * beta);
  double e_static_over_gas = 1.0 / (gamma * (1.0 - beta * dot3(kin, ph)));
  return e_static_over_gas * sqrt(f) / sqrt(1.0 - 2.0 * M / r_obs);
}

/* Disk colour with the Keplerian shift g: the ramp at the observed
 * temperature factor g t, brightness scaled by g^3. */
static void disk_rgb_doppler(const or_scene *sc, double r, double g, double rgb[3]) {
  double t = g * pow(sc->disk_r_in / r, 0.75);
  double k = 0.3 + 0.7 * t;
  double s = g * g * g;
  rgb[0] = 1.0 * k * s;
  rgb[1] = (0.35 + 0.65 * t) * k * s;
  rgb[2] = (0.1 + 0.9 * t * t) * k * s;
}

/* ------------------------------------------------------------------ */
/* The paper's own stepping (Sec. 2.1-2.2, Fig. 1): points of the ray at   */
/* fixed steps eps in phi, computed with the classical fourth-order        */
/* Runge-Kutta method, joined by straight segments in 3-D; objects are     */
/* found by intersecting each segment with them.  Readings: the point      */
/* beyond which u <= 0 ends the ray, escaping along the angle where the    */
/* straight line between the last two (phi, u) values reaches u = 0; a     */
/* segment whose end has u >= 1/(2M) and that meets no object is captured. */
/* ------------------------------------------------------------------ */
static void rk4_step(double M, double h, double *u, double *v) {
  double u0 = *u, v0 = *v;
  double ku1 = v0, kv1 = accel(M, u0);
  double ku2 = v0 + 0.5 * h * kv1, kv2 = accel(M, u0 + 0.5 * h * ku1);
  double ku3 = v0 + 0.5 * h * kv2, kv3 = accel(M, u0 + 0.5 * h * ku2);
  double ku4 = v0 + h * kv3, kv4 = accel(M, u0 + h * ku3);
  *u = u0 + h / 6.0 * (ku1 + 2.0 * ku2 + 2.0 * ku3 + ku4);
  *v = v0 + h / 6.0 * (kv1 + 2.0 * kv2 + 2.0 * kv3 + kv4);
}

/* 3-D point of the orbit at plane angle phi and u = 1/r */
static void plane_point(const or_plane *pl, double phi, double u, double x[3]) {
  double c = cos(phi), s = sin(phi);
  for (int k = 0; k < 3; ++k) x[k] = (c * pl->e1[k] + s * pl->e2[k]) / u;
}

typedef struct {
  unsigned flags, sphere_id, ambig;
  double phi_esc;   /* escape angle */
  double x[3];      /* hit position */
  double t[3];      /* unit direction of the segment that hit */
  long steps;
} or_poly_event;

static void trace_polyline(const or_scene *sc, const or_opts *o, const or_plane *pl,
                           or_poly_event *ev) {
  double M = sc->mass, eps = o->eps;
  double u = pl->u0, v = pl->v0, phi = 0.0;
  double u_capt = (M > 0) ? 1.0 / (2.0 * M) : INFINITY;
  double xa[3];
  plane_point(pl, 0.0, u, xa);
  ev->ambig = 0;
  ev->sphere_id = 0;
  for (long steps = 0;; ++steps) {
    ev->steps = steps;
    if (steps >= o->max_steps || phi >= o->phi_max) {
      ev->flags = OR_STEP_LIMIT;
      return;
    }
    double un = u, vn = v;
    rk4_step(M, eps, &un, &vn);
    double pb = phi + eps;
    if (un <= 0.0) {
      ev->flags = OR_ESC;
      ev->phi_esc = phi + eps * u / (u - un);
      ev->steps = steps + 1;
      return;
    }
    double xb[3], D[3];
    plane_point(pl, pb, un, xb);
    for (int k = 0; k < 3; ++k) D[k] = xb[k] - xa[k];
    double best_s = INFINITY;
    int best = -1; /* 0 sphere, 1 disk */
    unsigned best_id = 0;
    /* disk: the segment crosses z = 0 */
    if (sc->disk_enabled && !pl->disk_in_plane) {
      double za = xa[2], zb = xb[2];
      if ((za > 0.0 && zb <= 0.0) || (za < 0.0 && zb >= 0.0)) {
        double s = za / (za - zb), X[3];
        for (int k = 0; k < 3; ++k) X[k] = xa[k] + s * D[k];
        double r = norm3(X);
        if (fabs(r - sc->disk_r_in) < o->eps_r || fabs(r - sc->disk_r_out) < o->eps_r)
          ev->ambig |= OR_AMB_DISK;
        if (r >= sc->disk_r_in && r <= sc->disk_r_out) {
          best_s = s;
          best = 1;
        }
      }
    }
    /* spheres: first entry along the segment */
    double dd = dot3(D, D);
    for (int k = 0; k < sc->n_spheres; ++k) {
      const or_sphere *S = &sc->spheres[k];
      double oc[3] = {xa[0] - S->c[0], xa[1] - S->c[1], xa[2] - S->c[2]};
      double bq = dot3(oc, D), cq = dot3(oc, oc) - S->radius * S->radius;
      /* closest approach of the segment to the centre, for the graze mask */
      double sc_ = fmin(1.0, fmax(0.0, -bq / dd));
      double cl[3] = {oc[0] + sc_ * D[0], oc[1] + sc_ * D[1], oc[2] + sc_ * D[2]};
      if (fabs(norm3(cl) - S->radius) < o->eps_r) ev->ambig |= OR_AMB_SPHERE;
      double disc = bq * bq - dd * cq;
      if (disc < 0.0) continue;
      double s = (-bq - sqrt(disc)) / dd;
      if (s < 0.0 || s > 1.0) continue;
      if (s < best_s - 1e-12 || (fabs(s - best_s) <= 1e-12 && (best != 0 || (unsigned)k < best_id))) {
        best_s = s;
        best = 0;
        best_id = (unsigned)k;
      }
    }
    if (best >= 0) {
      double nD = sqrt(dd);
      for (int k = 0; k < 3; ++k) {
        ev->x[k] = xa[k] + best_s * D[k];
        ev->t[k] = D[k] / nD;
      }
      ev->flags = best == 0 ? OR_SPHERE : OR_DISK;
      ev->sphere_id = best_id;
      ev->steps = steps + 1;
      return;
    }
    if (un >= u_capt) {
      ev->flags = OR_CAPT;
      ev->steps = steps + 1;
      return;
    }
    u = un;
    v = vn;
    phi = pb;
    for (int k = 0; k < 3; ++k) xa[k] = xb[k];
  }
}

/* Shade a polyline event into out (direction, colour, mask bits). */
static void shade_polyline(const or_scene *sc, const or_opts *o, const or_plane *pl,
                           const or_poly_event *ev, or_pixel *out) {
  out->ambig |= ev->ambig;
  out->steps = ev->steps;
  out->flags = ev->flags;
  out->sphere_id = ev->sphere_id;
  if (ev->flags == OR_CAPT || ev->flags == OR_STEP_LIMIT) {
    out->theta = out->phi = NAN;
    out->rgb[0] = out->rgb[1] = out->rgb[2] = 0.0;
    return;
  }
  double dirv[3];
  if (ev->flags == OR_ESC) {
    double cp = cos(ev->phi_esc), sp = sin(ev->phi_esc);
    for (int k = 0; k < 3; ++k) dirv[k] = cp * pl->e1[k] + sp * pl->e2[k];
    dir_angles(dirv, &out->theta, &out->phi);
    sky_colour(sc, out->theta, out->phi, out->rgb);
    if (!sc->sky_tex && near_cell_edge(out->theta, out->phi, o->eps_ang)) out->ambig |= OR_AMB_SKY;
    return;
  }
  double r = norm3(ev->x);
  for (int k = 0; k < 3; ++k) dirv[k] = ev->x[k] / r;
  dir_angles(dirv, &out->theta, &out->phi);
  if (ev->flags == OR_DISK) {
    disk_rgb(sc, r, out->rgb);
  } else {
    const or_sphere *S = &sc->spheres[ev->sphere_id];
    double N[3];
    for (int k = 0; k < 3; ++k) N[k] = (ev->x[k] - S->c[k]) / S->radius;
    double lam = 0.25 + 0.75 * fmax(0.0, -dot3(N, ev->t));
    for (int c = 0; c < 3; ++c) out->rgb[c] = S->albedo[c] * lam;
  }
}

static void render_ray(const or_scene *sc, const or_opts *o, const double P[3],
                       const double d[3], or_pixel *out) {
  double M = sc->mass;
  or_plane pl;
  plane_reduce(sc, P, d, &pl);
  out->ambig = 0;
  out->sphere_id = 0;
  out->steps = 0;
  out->b = pl.b;
  double bc = 3.0 * sqrt(3.0) * M;
  if (M > 0 && fabs(pl.b - bc) < o->eps_b) out->ambig |= OR_AMB_CAPT;

  double dirv[3];
  if (pl.radial) {
    /* straight radial line x(t) = P + t d */
    out->ambig |= OR_AMB_DEGEN;
    double best_t = INFINITY;
    int best_k = -1;
    for (int k = 0; k < sc->n_spheres; ++k) {
      const or_sphere *S = &sc->spheres[k];
      double oc[3] = {P[0] - S->c[0], P[1] - S->c[1], P[2] - S->c[2]};
      double bq = dot3(oc, d), cq = dot3(oc, oc) - S->radius * S->radius;
      double disc = bq * bq - cq;
      if (disc < 0) continue;
      double t = -bq - sqrt(disc);
      if (t > 0 && t < best_t) {
        best_t = t;
        best_k = k;
      }
    }
    double r0 = norm3(P);
    int ingoing = pl.cos_a < 0;
    double t_hole = ingoing ? r0 - 2.0 * M : INFINITY;
    if (best_k >= 0 && best_t < t_hole) {
      double x[3] = {P[0] + best_t * d[0], P[1] + best_t * d[1], P[2] + best_t * d[2]};
      const or_sphere *S = &sc->spheres[best_k];
      double N[3] = {(x[0] - S->c[0]) / S->radius, (x[1] - S->c[1]) / S->radius,
                     (x[2] - S->c[2]) / S->radius};
      double lam = 0.25 + 0.75 * fmax(0.0, -dot3(N, d));
      double nx = norm3(x);
      dirv[0] = x[0] / nx;
      dirv[1] = x[1] / nx;
      dirv[2] = x[2] / nx;
      out->flags = OR_SPHERE;
      out->sphere_id = (unsigned)best_k;
      for (int c = 0; c < 3; ++c) out->rgb[c] = S->albedo[c] * lam;
      dir_angles(dirv, &out->theta, &out->phi);
      return;
    }
    if (ingoing && M > 0) {
      out->flags = OR_CAPT;
      out->theta = out->phi = NAN;
      out->rgb[0] = out->rgb[1] = out->rgb[2] = 0.0;
      return;
    }
    out->flags = OR_ESC;
    dir_angles(d, &out->theta, &out->phi);
    sky_colour(sc, out->theta, out->phi, out->rgb);
    if (!sc->sky_tex && near_cell_edge(out->theta, out->phi, o->eps_ang)) out->ambig |= OR_AMB_SKY;
    return;
  }
  if (sc->disk_enabled && pl.disk_in_plane) out->ambig |= OR_AMB_DEGEN;

  if (o->method == 1) {
    or_poly_event pev;
    trace_polyline(sc, o, &pl, &pev);
    shade_polyline(sc, o, &pl, &pev, out);
    return;
  }
  or_event ev;
  trace_plane(sc, o, &pl, &ev);
  out->ambig |= ev.ambig;
  out->steps = ev.steps;
  out->flags = ev.flags;
  out->sphere_id = ev.sphere_id;
  if (ev.flags == OR_CAPT || ev.flags == OR_STEP_LIMIT) {
    out->theta = out->phi = NAN;
    out->rgb[0] = out->rgb[1] = out->rgb[2] = 0.0;
    return;
  }
  double cp = cos(ev.phi_evt), sp = sin(ev.phi_evt);
  for (int k = 0; k < 3; ++k) dirv[k] = cp * pl.e1[k] + sp * pl.e2[k];
  dir_angles(dirv, &out->theta, &out->phi);
  if (ev.flags == OR_ESC) {
    sky_colour(sc, out->theta, out->phi, out->rgb);
    if (!sc->sky_tex && near_cell_edge(out->theta, out->phi, o->eps_ang)) out->ambig |= OR_AMB_SKY;
  } else if (ev.flags == OR_DISK) {
    if (o->doppler) {
      double u = ev.u_evt, r = 1.0 / u, x[3], tdir[3];
      for (int k = 0; k < 3; ++k) {
        x[k] = dirv[k] * r;
        tdir[k] = -sp * pl.e1[k] + cp * pl.e2[k];
      }
      double g = disk_g(M, norm3(P), x, dirv, -ev.v_evt / (u * u), tdir, r);
      disk_rgb_doppler(sc, r, g, out->rgb);
    } else {
      disk_rgb(sc, 1.0 / ev.u_evt, out->rgb);
    }
  } else { /* sphere */
    const or_sphere *S = &sc->spheres[ev.sphere_id];
    double u = ev.u_evt, v = ev.v_evt;
    double x[3], T[3];
    for (int k = 0; k < 3; ++k) {
      x[k] = dirv[k] / u;
      /* d x / d phi scaled by u^2 > 0 */
      T[k] = u * (-sp * pl.e1[k] + cp * pl.e2[k]) - v * dirv[k];
    }
    double nt = norm3(T);
    double N[3];
    for (int k = 0; k < 3; ++k) {
      T[k] /= nt;
      N[k] = (x[k] - S->c[k]) / S->radius;
    }
    double lam = 0.25 + 0.75 * fmax(0.0, -dot3(N, T));
    for (int c = 0; c < 3; ++c) out->rgb[c] = S->albedo[c] * lam;
  }
  (void)M;
}

/* One pixel.  With spp_n = n > 1 the pixel's colour is the mean of the
 * linear colours of n x n stratified samples, at the centres of an n x n
 * grid over the pixel (anti-aliasing, Sec. 3); its direction, flags, impact
 * parameter and step count are those of the ray through the pixel centre,
 * and its mask collects the bits of every sample. */
static void render_pixel(const or_scene *sc, const or_opts *o, const or_camera *cam, int x, int y,
                         or_pixel *out) {
  double P[3], d[3];
  camera_ray(cam, x, y, P, d);
  render_ray(sc, o, P, d, out);
  int n = o->spp_n;
  if (n <= 1) return;
  double acc[3] = {0.0, 0.0, 0.0};
  unsigned amb = out->ambig;
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < n; ++i) {
      /* camera_ray adds half a pixel to its coordinates */
      double sx = x + (i + 0.5) / n - 0.5, sy = y + (j + 0.5) / n - 0.5;
      camera_ray(cam, sx, sy, P, d);
      or_pixel smp;
      render_ray(sc, o, P, d, &smp);
      for (int c = 0; c < 3; ++c) acc[c] += smp.rgb[c];
      amb |= smp.ambig;
    }
  }
  for (int c = 0; c < 3; ++c) out->rgb[c] = acc[c] / (n * n);
  out->ambig = amb;
}

static void store_pixel(const or_pixel *px, long idx, double *theta, double *phi,
                        uint16_t *flags, uint32_t *rgba, uint8_t *ambig,
                        double *b_out, int32_t *steps_out) {
  if (theta) theta[idx] = px->theta;
  if (phi) phi[idx] = px->phi;
  if (flags) flags[idx] = (uint16_t)(px->flags | (px->sphere_id << 8));
  if (rgba)
    rgba[idx] = quant8(px->rgb[0]) | (quant8(px->rgb[1]) << 8) |
                (quant8(px->rgb[2]) << 16) | (255u << 24);
  if (ambig) ambig[idx] = (uint8_t)px->ambig;
  if (b_out) b_out[idx] = px->b;
  if (steps_out) steps_out[idx] = (int32_t)px->steps;
}

static int set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* Exported entry points                                                */
/* ------------------------------------------------------------------ */

/* Number of threads the OpenMP build will use (1 without OpenMP). */
int or_threads(int nthreads) { return set_threads(nthreads); }

/* Render all pixels of all cameras, camera-major then row-major.  OpenMP,
 * when compiled in, splits the scanlines dynamically one at a time (the
 * paper's shared-memory scheme, Sec. 2.4). Any output pointer may be NULL. */
int or_render(const or_scene *sc, const or_camera *cams, int ncams,
              const or_opts *o, int nthreads, double *theta, double *phi,
              uint16_t *flags, uint32_t *rgba, uint8_t *ambig, double *b_out,
              int32_t *steps_out) {
  if (!sc || !cams || !o || ncams < 0) return -1;
  set_threads(nthreads);
  long base = 0;
  for (int c = 0; c < ncams; ++c) {
    const or_camera *cam = &cams[c];
    int W = cam->w, Hh = cam->h;
#pragma omp parallel for schedule(dynamic, 1)
    for (int y = 0; y < Hh; ++y) {
      for (int x = 0; x < W; ++x) {
        or_pixel px;
        render_pixel(sc, o, cam, x, y, &px);
        store_pixel(&px, base + (long)y * W + x, theta, phi, flags, rgba, ambig,
                    b_out, steps_out);
      }
    }
    base += (long)W * Hh;
  }
  return 0;
}

/* Render a list of individual pixels (cam[i], px[i], py[i]); output i is
 * pixel i of the list. */
int or_render_pixels(const or_scene *sc, const or_camera *cams, int ncams,
                     const or_opts *o, int nthreads, long n,
                     const int32_t *cam_idx, const int32_t *px,
                     const int32_t *py, double *theta, double *phi,
                     uint16_t *flags, uint32_t *rgba, uint8_t *ambig,
                     double *b_out, int32_t *steps_out) {
  if (!sc || !cams || !o || n < 0) return -1;
  set_threads(nthreads);
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(| : bad)
  for (long i = 0; i < n; ++i) {
    int c = cam_idx[i];
    if (c < 0 || c >= ncams) {
      bad = 1;
      continue;
    }
    or_pixel pxo;
    render_pixel(sc, o, &cams[c], px[i], py[i], &pxo);
    store_pixel(&pxo, i, theta, phi, flags, rgba, ambig, b_out, steps_out);
  }
  return bad ? -1 : 0;
}

/* Trace an arbitrary world ray from P along unit d (outputs as above). */
int or_render_world_ray(const or_scene *sc, const or_opts *o, const double P[3],
                        const double d[3], double *theta, double *phi,
                        uint16_t *flags, uint32_t *rgba, uint8_t *ambig,
                        double *b_out, int32_t *steps_out) {
  or_pixel px;
  render_ray(sc, o, P, d, &px);
  store_pixel(&px, 0, theta, phi, flags, rgba, ambig, b_out, steps_out);
  return 0;
}

/* Camera ray of one pixel (world position P and unit direction d). */
void or_camera_ray(const or_camera *cam, double px, double py, double *P,
                   double *d) {
  camera_ray(cam, px, py, P, d);
}

/* Plane quantities of one world ray: b, u0, v0, psi0 and the basis. */
void or_plane_of_ray(const or_scene *sc, const double *P, const double *d,
                     double *b, double *u0, double *v0, double *psi0,
                     double *e1, double *e2) {
  or_plane pl;
  plane_reduce(sc, P, d, &pl);
  *b = pl.b;
  *u0 = pl.u0;
  *v0 = pl.v0;
  *psi0 = pl.psi0;
  for (int k = 0; k < 3; ++k) {
    e1[k] = pl.e1[k];
    e2[k] = pl.radial ? 0.0 : pl.e2[k];
  }
}

/* Integrate u(phi) from (u0, v0) at phi = 0 with no scene objects until
 * escape (u = 0), capture (u = 1/(2M)), phi_max or max_steps.  Returns the
 * flag; *phi_exit is the event angle. */
int or_orbit_exit(double M, double u0, double v0, double rtol, double atol,
                  double phi_max, long max_steps, double *phi_exit,
                  long *steps) {
  or_scene sc;
  memset(&sc, 0, sizeof sc);
  sc.mass = M;
  or_opts o = {rtol, atol, phi_max, max_steps, 0.0, 0.0, 0.0};
  or_plane pl;
  memset(&pl, 0, sizeof pl);
  pl.u0 = u0;
  pl.v0 = v0;
  pl.disk_in_plane = 1;
  or_event ev;
  trace_plane(&sc, &o, &pl, &ev);
  *phi_exit = ev.phi_evt;
  if (steps) *steps = ev.steps;
  return (int)ev.flags;
}

/* Integrate with no events up to phi_end and record every accepted step
 * end point (phi, u, v); returns the number recorded (at most cap). */
long or_orbit_steps(double M, double u0, double v0, double rtol, double atol,
                    double phi_end, long cap, double *phi_o, double *u_o,
                    double *v_o) {
  double u = u0, v = v0, phi = 0.0;
  double h = initial_step(M, u, v, rtol, atol);
  long n = 0;
  if (n < cap) {
    phi_o[n] = 0.0;
    u_o[n] = u;
    v_o[n] = v;
    ++n;
  }
  long guard = 0;
  while (phi < phi_end && n < cap && guard < 10000000) {
    ++guard;
    if (phi + h > phi_end) h = phi_end - phi;
    double un, vn, err;
    dp5_attempt(M, u, v, h, rtol, atol, &un, &vn, &err);
    if (!(err <= 1.0)) {
      h = next_step(h, err, 0);
      continue;
    }
    phi += h;
    u = un;
    v = vn;
    phi_o[n] = phi;
    u_o[n] = u;
    v_o[n] = v;
    ++n;
    h = next_step(h, err, 1);
  }
  return n;
}

/* Like or_orbit_steps but reports u and u' at the requested increasing
 * angles phis[0..n) from the quintic Hermite interpolant. */
int or_orbit_sample(double M, double u0, double v0, double rtol, double atol,
                    long n, const double *phis, double *u_o, double *v_o) {
  double u = u0, v = v0, phi = 0.0;
  double h = initial_step(M, u, v, rtol, atol);
  long i = 0;
  while (i < n && phis[i] <= 0.0) {
    u_o[i] = u0;
    v_o[i] = v0;
    ++i;
  }
  long guard = 0;
  while (i < n && guard < 10000000) {
    ++guard;
    double un, vn, err;
    dp5_attempt(M, u, v, h, rtol, atol, &un, &vn, &err);
    if (!(err <= 1.0)) {
      h = next_step(h, err, 0);
      continue;
    }
    hermite5 H;
    hermite_make(&H, M, phi, h, u, v, un, vn);
    while (i < n && phis[i] <= phi + h) {
      u_o[i] = hermite_u(&H, phis[i]);
      v_o[i] = hermite_v(&H, phis[i]);
      ++i;
    }
    phi += h;
    u = un;
    v = vn;
    h = next_step(h, err, 1);
  }
  return i == n ? 0 : -1;
}

/* Sky colour (linear RGB in [0, 1]) of a direction, for unit tests. */
void or_sky_rgb(uint64_t seed, double theta, double phi, double *rgb) {
  sky_rgb(seed, theta, phi, rgb);
}

/* splitmix64 output for state x, for unit tests. */
uint64_t or_splitmix64(uint64_t x) { return splitmix64(x); }

/* Frequency ratio of the Keplerian disk shading (see disk_g), exposed for
 * the tests: disk point x (equatorial, r = |x|), traced direction per unit
 * phi given by dr/dphi and the in-plane unit tangent t. */
double or_disk_g(double M, double r_obs, const double *x, const double *t, double dr_dphi) {
  double r = norm3(x), xr[3];
  for (int k = 0; k < 3; ++k) xr[k] = x[k] / r;
  return disk_g(M, r_obs, x, xr, dr_dphi, t, r);
}
