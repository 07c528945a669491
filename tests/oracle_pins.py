"""Checks that pin the CPU oracle to facts fixed by the physics, not by itself.

Each check takes an oracle library handle (so the same check can run against
deliberately broken builds of the oracle) and returns (ok, detail).  The
expected values come from closed forms (``closed_forms``), textbook
straight-line geometry at M = 0, published test vectors, or scaling laws of
the Dormand-Prince 5(4) pair.  Eq. 1 of the paper is used with the sign fixed
by the first integral: u'' = 3 M u^2 - u.
"""
from __future__ import annotations

import math

import numpy as np

import closed_forms as cf
import oracle
from paper_2507_16165_gb300 import workloads as W

M = 1.0
B_C = cf.B_CRIT


def angle_between(a, b) -> float:
    """Great-circle angle between two directions, accurate near zero."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return math.atan2(float(np.linalg.norm(np.cross(a, b))), float(np.dot(a, b)))


def _ingoing_v0(M, b, u0):
    return math.sqrt(1.0 / (b * b) - u0 * u0 + 2 * M * u0 ** 3)


def first_integral(lib):
    """(u')^2 + u^2 - 2Mu^3 stays 1/b^2 along the accepted steps, to within
    the integration tolerance (rtol = atol = 1e-10; |u|, |u'| < 1, so the
    absolute tolerance governs)."""
    worst = 0.0
    for b, u0, phi_end in [(5.3, 1 / 30, 6.0), (6.0, 1 / 40, 5.0), (12.0, 1 / 50, 3.0),
                           (5.1963, 1 / 30, 10.0), (4.0, 1 / 30, 1.0)]:
        v0 = _ingoing_v0(M, b, u0)
        ph, u, v = oracle.orbit_steps(M, u0, v0, phi_end, lib=lib)
        keep = u < 1.0 / (2 * M)
        E = v[keep] ** 2 + u[keep] ** 2 - 2 * M * u[keep] ** 3
        worst = max(worst, float(np.max(np.abs(E - 1.0 / (b * b)))))
    return worst < 1e-10, f"max absolute drift {worst:.3e}"


def exit_angle(lib, rtol=1e-12):
    """Escape angle phi_inf equals the Carlson elliptic form; error budget
    2e-11 rad scaled by the near-critical amplification 1/(b - b_c)."""
    worst = 0.0
    for b in [5.2, 5.25, 5.5, 6.0, 7.0, 10.0, 20.0, 29.0]:
        u0 = 1 / 30
        v0 = _ingoing_v0(M, b, u0)
        f, ph, _ = oracle.orbit_exit(M, u0, v0, rtol, rtol, lib=lib)
        if f != oracle.ESC:
            return False, f"b={b}: flag {f}, expected escape"
        err = abs(ph - cf.phi_inf(M, b, u0))
        budget = 2e-11 * max(1.0, 1.0 / (b - B_C))
        worst = max(worst, err / budget)
    return worst <= 1.0, f"worst error / budget {worst:.3f}"


def exit_angle_render_tol(lib):
    """At the rendering tolerance rtol = atol = 1e-10 the escape angle is
    within 2e-9 rad x 1/(b - b_c) of the Carlson form."""
    worst = 0.0
    for b in [5.1963, 5.2, 5.5, 8.0, 15.0]:
        u0 = 1 / 40
        v0 = _ingoing_v0(M, b, u0)
        f, ph, _ = oracle.orbit_exit(M, u0, v0, 1e-10, 1e-10, lib=lib)
        if f != oracle.ESC:
            return False, f"b={b}: flag {f}"
        err = abs(ph - cf.phi_inf(M, b, u0))
        worst = max(worst, err / (2e-9 * max(1.0, 1.0 / (b - B_C))))
    return worst <= 1.0, f"worst error / budget {worst:.3f}"


def weak_field(lib):
    """Infinity-to-infinity deflection minus 4M/b + 15 pi M^2/(4b^2) is the
    next series term 128 M^3/(3 b^3) up to O(M^4/b^4) (coefficient 3465 pi/64
    ~ 170); checked for b in [1e2, 1e4]."""
    worst = 0.0
    for b in [1e2, 3e2, 1e3, 3e3, 1e4]:
        f, ph, _ = oracle.orbit_exit(M, 0.0, 1.0 / b, 1e-13, 1e-15 / b, lib=lib)
        if f != oracle.ESC:
            return False, f"b={b}: flag {f}"
        resid = (ph - math.pi) - cf.weak_field_deflection(M, b)
        third = resid * b ** 3
        tol = 200.0 / b + 2e-12 * b ** 3
        worst = max(worst, abs(third - 128.0 / 3.0) / tol)
    return worst <= 1.0, f"worst |b^3 resid - 128/3| / tol = {worst:.3f}"


def capture_iff_subcritical(lib, n=2000):
    """An ingoing ray from r = 1000M is captured iff b < 3 sqrt(3) M, for
    |b - b_c| >= 1e-6 M."""
    rng = np.random.default_rng(1)
    offs = np.exp(rng.uniform(math.log(1e-6), math.log(2.0), n))
    sign = np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    bad = 0
    u0 = 1e-3
    for o, s in zip(offs, sign):
        b = B_C + s * o
        v0 = _ingoing_v0(M, b, u0)
        f, _, _ = oracle.orbit_exit(M, u0, v0, 1e-10, 1e-10, lib=lib)
        want = oracle.CAPT if b < B_C else oracle.ESC
        bad += int(f != want)
    return bad == 0, f"{bad} of {n} misclassified"


def photon_orbit(lib):
    """u = 1/(3M), u' = 0 is the unstable circular orbit; a perturbation eps
    grows like eps cosh(phi) (linearised u'' = (6Mu - 1) du = du)."""
    ph, u, v = oracle.orbit_steps(M, 1.0 / 3.0, 0.0, 8.0, lib=lib)
    stay = float(np.max(np.abs(u - 1.0 / 3.0)))
    eps = 1e-9
    phis = np.linspace(0.5, 5.0, 10)
    up, _ = oracle.orbit_sample(M, 1.0 / 3.0 + eps, 0.0, phis, 1e-13, 1e-15, lib=lib)
    growth = (up - 1.0 / 3.0) / (eps * np.cosh(phis))
    gerr = float(np.max(np.abs(growth - 1.0)))
    return stay < 1e-11 and gerr < 1e-3, f"drift {stay:.2e}, growth error {gerr:.2e}"


def periastron(lib):
    """The largest u along an escaping orbit is the middle root of
    2Mu^3 - u^2 + 1/b^2 (numpy.roots), to 1e-12."""
    worst = 0.0
    for b in [5.4, 6.5, 9.0, 15.0]:
        u0 = 1 / 30
        v0 = _ingoing_v0(M, b, u0)
        u2 = cf.cubic_roots(M, b)[1]
        phi_p = cf.leg_angle(M, b, u0, u2)
        phis = phi_p + np.linspace(-2e-3, 2e-3, 4001)
        u, _ = oracle.orbit_sample(M, u0, v0, phis, 1e-13, 1e-15, lib=lib)
        worst = max(worst, abs(float(u.max()) - u2))
    return worst < 1e-12, f"max |u_max - u_p| = {worst:.2e}"


def step_order(lib):
    """Dormand-Prince 5(4) with an error-per-step controller: accepted step
    sizes scale like tol^(1/5), so a 1e5-fold tighter tolerance shrinks the
    median step over phi in [1, 2.5] about 10-fold (accepted 8..12.5)."""
    worst = 0.0
    for b in (5.5, 8.0, 20.0):
        u0 = 1 / 30
        v0 = _ingoing_v0(M, b, u0)
        med = []
        for tol in (1e-6, 1e-11):
            ph, _, _ = oracle.orbit_steps(M, u0, v0, 3.0, tol, tol, lib=lib)
            h = np.diff(ph)
            mid = (ph[:-1] >= 1.0) & (ph[1:] <= 2.5)
            if mid.sum() < 1:
                return False, "no steps in the window"
            med.append(float(np.median(h[mid])))
        ratio = med[0] / med[1]
        if not 8.0 <= ratio <= 12.5:
            return False, f"b={b}: step ratio {ratio:.2f}"
        worst = max(worst, abs(ratio - 10.0))
    return True, f"max |ratio - 10| = {worst:.2f}"


# straight-line checks run at a tolerance far below the geometry they test
TIGHT = oracle.opts(rtol=1e-13, atol=1e-15)


def _flat_scene(disk=None, spheres=()):
    return W.Scene(mass=0.0, disk=disk, spheres=tuple(spheres), sky_seed=0)


def straight_lines_m0(lib):
    """At M = 0 every escaping ray leaves along its camera direction (1e-11
    rad at rtol 1e-13) and its colour is the sky colour of that direction."""
    cam = W.Camera(30.0, 63.0, 24, 16, azim_deg=20.0)
    sc = _flat_scene()
    out = oracle.render(sc, [cam], TIGHT, lib=lib)
    worst = 0.0
    bad_rgba = 0
    for y in range(cam.h):
        for x in range(cam.w):
            i = y * cam.w + x
            _, d = oracle.camera_ray(cam, x, y, lib=lib)
            th, ph = out["theta"][i], out["phi"][i]
            e = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            worst = max(worst, angle_between(e, d))
            th_d = math.acos(d[2])
            ph_d = math.atan2(d[1], d[0]) % (2 * math.pi)
            rgb = oracle.sky_rgb(0, th_d, ph_d, lib=lib)
            q = np.minimum(255, np.floor(255 * rgb + 0.5)).astype(np.uint32)
            want = int(q[0] | (q[1] << 8) | (q[2] << 16) | (255 << 24))
            bad_rgba += int(want != int(out["rgba"][i]))
            if out["flags"][i] != oracle.ESC:
                return False, f"pixel {x},{y}: flag {out['flags'][i]}"
    return worst < 1e-11 and bad_rgba == 0, f"max angle {worst:.2e}, rgba mismatches {bad_rgba}"


def disk_m0(lib):
    """At M = 0 the thin disk is hit exactly where the straight ray meets
    z = 0 with r in [r_in, r_out]; the reported direction is that of the hit
    point."""
    cam = W.Camera(30.0, 70.0, 32, 32, azim_deg=35.0, fov_deg=90.0)
    sc = _flat_scene(disk=(4.0, 20.0))
    out = oracle.render(sc, [cam], TIGHT, lib=lib)
    worst, wrong = 0.0, 0
    for y in range(cam.h):
        for x in range(cam.w):
            i = y * cam.w + x
            P, d = oracle.camera_ray(cam, x, y, lib=lib)
            hit = False
            if d[2] != 0:
                t = -P[2] / d[2]
                if t > 0:
                    X = P + t * d
                    r = float(np.linalg.norm(X))
                    if abs(r - 4.0) < 1e-9 or abs(r - 20.0) < 1e-9:
                        continue
                    hit = 4.0 <= r <= 20.0
            got = out["flags"][i] == oracle.DISK
            if got != hit:
                wrong += 1
                continue
            if hit:
                n = X / r
                th, ph = out["theta"][i], out["phi"][i]
                e = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph),
                              math.cos(th)])
                worst = max(worst, angle_between(e, n))
    n_hit = int(np.sum(out["flags"] == oracle.DISK))
    return wrong == 0 and worst < 1e-11 and n_hit > 50, \
        f"{wrong} flag mismatches, {n_hit} hits, max angle {worst:.2e}"


def spheres_m0(lib):
    """At M = 0 sphere hits are the first ray-sphere intersections, with the
    sphere index in the high byte and Lambert shading against the ray."""
    sph = [W.Sphere((2.0, 1.0, 0.5), 1.5, (0.9, 0.5, 0.3)),
           W.Sphere((-3.0, -2.0, 1.0), 1.0, (0.4, 0.8, 0.6)),
           W.Sphere((0.0, 3.0, -2.0), 2.0, (0.7, 0.7, 0.9))]
    cam = W.Camera(25.0, 60.0, 32, 32, azim_deg=10.0, fov_deg=40.0)
    sc = _flat_scene(spheres=sph)
    out = oracle.render(sc, [cam], TIGHT, lib=lib)
    wrong = 0
    worst = 0.0
    for y in range(cam.h):
        for x in range(cam.w):
            i = y * cam.w + x
            P, d = oracle.camera_ray(cam, x, y, lib=lib)
            best, bk, graze = math.inf, -1, False
            for k, s in enumerate(sph):
                oc = P - np.array(s.center)
                bq = float(np.dot(oc, d))
                disc = bq * bq - (float(np.dot(oc, oc)) - s.radius ** 2)
                if abs(disc) < 1e-8:
                    graze = True
                if disc < 0:
                    continue
                t = -bq - math.sqrt(disc)
                if 0 < t < best:
                    best, bk = t, k
            if graze:
                continue
            f = int(out["flags"][i])
            if bk < 0:
                wrong += int(f != oracle.ESC)
                continue
            if f != (oracle.SPHERE | (bk << 8)):
                wrong += 1
                continue
            X = P + best * d
            n = X / np.linalg.norm(X)
            th, ph = out["theta"][i], out["phi"][i]
            e = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
            worst = max(worst, angle_between(e, n))
            N = (X - np.array(sph[bk].center)) / sph[bk].radius
            lam = 0.25 + 0.75 * max(0.0, -float(np.dot(N, d)))
            q = np.minimum(255, np.floor(255 * np.array(sph[bk].albedo) * lam + 0.5))
            got = [(int(out["rgba"][i]) >> (8 * c)) & 255 for c in range(3)]
            wrong += int(max(abs(int(q[c]) - got[c]) for c in range(3)) > 1)
    n_hit = int(np.sum((out["flags"] & 0xFF) == oracle.SPHERE))
    return wrong == 0 and worst < 1e-11 and n_hit > 50, \
        f"{wrong} mismatches, {n_hit} hits, max angle {worst:.2e}"


def shadow_edge(lib):
    """Config-1 camera: a pixel is captured iff its off-axis angle is inside
    asin(b_c sqrt(1 - 2M/r)/r) (static observer)."""
    cam = W.Camera(30.0, 90.0, 64, 64)
    sc = W.Scene(mass=1.0, sky_seed=0)
    out = oracle.render(sc, [cam], lib=lib)
    psi_sh = cf.shadow_angle(1.0, 30.0)
    wrong = 0
    for y in range(cam.h):
        for x in range(cam.w):
            P, d = oracle.camera_ray(cam, x, y, lib=lib)
            psi = math.acos(-float(np.dot(d, P)) / np.linalg.norm(P))
            if abs(psi - psi_sh) < 1e-7:
                continue
            want = psi < psi_sh
            wrong += int(want != (out["flags"][y * cam.w + x] == oracle.CAPT))
    n_capt = int(np.sum(out["flags"] == oracle.CAPT))
    return wrong == 0 and n_capt > 100, f"{wrong} mismatches, {n_capt} captured"


def einstein_ring(lib):
    """The off-axis angle whose ray leaves exactly behind the hole (phi_inf
    = pi) matches the Carlson form plus a 1-D root, to 1e-9 rad."""
    from scipy import optimize
    r = 30.0
    u0 = 1.0 / r

    def g(psi):
        b = cf.static_b(1.0, r, math.sin(psi))
        v0 = _ingoing_v0(1.0, b, u0)
        _, ph, _ = oracle.orbit_exit(1.0, u0, v0, 1e-12, 1e-12, lib=lib)
        return ph - math.pi

    want = cf.einstein_ring_angle(1.0, r)
    got = optimize.brentq(g, want - 0.02, want + 0.02, xtol=1e-14)
    return abs(got - want) < 1e-9, f"ring at {got:.12f} vs {want:.12f}"


def disk_radius_m1(lib):
    """With M = 1, u at the node angles sampled from the oracle's trajectory
    agrees with the Carlson form phi(u) (self-consistency of the crossing
    radii the disk test reads)."""
    worst = 0.0
    for b, u0 in [(7.0, 1 / 40), (12.0, 1 / 40), (5.6, 1 / 50)]:
        v0 = _ingoing_v0(1.0, b, u0)
        u2 = cf.cubic_roots(1.0, b)[1]
        phi_p = cf.leg_angle(1.0, b, u0, u2)
        phis = np.array([0.3 * phi_p, 0.8 * phi_p, phi_p + 0.5 * (cf.phi_inf(1.0, b, u0) - phi_p)])
        u, _ = oracle.orbit_sample(1.0, u0, v0, phis, 1e-12, 1e-12, lib=lib)
        for k, (ph, uu) in enumerate(zip(phis, u)):
            back = cf.phi_at_u(1.0, b, u0, float(uu), outgoing=(k == 2))
            worst = max(worst, abs(back - ph))
    return worst < 1e-9, f"max angle mismatch {worst:.2e}"


def splitmix_vector(lib):
    """splitmix64 with state 0: first output 0xE220A8397B1DCDAF (published
    reference vector of the generator)."""
    got = oracle.splitmix64(0, lib=lib)
    return got == 0xE220A8397B1DCDAF, hex(got)


def sky_cells(lib):
    """Sky colour at chosen directions: cell (i, j) = (floor(16 theta/pi),
    floor(32 phi/2pi)); parity picks light (0.9, 0.9, 0.9) or dark
    (0.1, 0.1, 0.25); tint 0.75 + 0.25 h/2^24 from 24-bit slices of
    splitmix64(seed * 2654435761 + 32 i + j) at bits 0, 16, 32."""
    cases = []
    for (i, j) in [(0, 0), (0, 1), (7, 5), (15, 31), (8, 16)]:
        th = (i + 0.5) * math.pi / 16
        ph = (j + 0.5) * 2 * math.pi / 32
        cases.append((i, j, th, ph))
    bad = 0
    h00 = 0xE220A8397B1DCDAF      # splitmix64(0): cell (0,0), seed 0
    rgb00 = oracle.sky_rgb(0, cases[0][2], cases[0][3], lib=lib)
    want00 = [0.9 * (0.75 + 0.25 * ((h00 >> (16 * c)) & 0xFFFFFF) / 2 ** 24) for c in range(3)]
    bad += int(np.max(np.abs(rgb00 - want00)) > 1e-15)
    for i, j, th, ph in cases[1:]:
        rgb = oracle.sky_rgb(0, th, ph, lib=lib)
        light = ((i + j) & 1) == 0
        lo = np.array([0.9, 0.9, 0.9] if light else [0.1, 0.1, 0.25]) * 0.75
        hi = lo / 0.75
        bad += int(np.any(rgb < lo - 1e-15) or np.any(rgb > hi + 1e-15))
    # theta = pi and phi -> 2 pi fall into the last cells
    last = oracle.sky_rgb(0, math.pi, 2 * math.pi - 1e-12, lib=lib)
    bad += int(not np.all(last > 0.0))
    return bad == 0, f"{bad} bad cells"


def camera_convention(lib):
    """Pinhole conventions: the image centre looks at the hole; row 0 is the
    top (world +z side for an equatorial observer); column 0 is the left;
    the rays through the left and right image edges of the centre row span
    exactly the field of view."""
    cam = W.Camera(30.0, 90.0, 40, 30, fov_deg=50.0)
    P, dc = oracle.camera_ray(cam, (cam.w - 1) / 2, (cam.h - 1) / 2, lib=lib)
    fwd = -P / np.linalg.norm(P)
    c0 = angle_between(dc, fwd)
    _, dtop = oracle.camera_ray(cam, (cam.w - 1) / 2, 0, lib=lib)
    _, dleft = oracle.camera_ray(cam, 0, (cam.h - 1) / 2, lib=lib)
    _, dl = oracle.camera_ray(cam, -0.5, (cam.h - 1) / 2, lib=lib)
    _, dr = oracle.camera_ray(cam, cam.w - 0.5, (cam.h - 1) / 2, lib=lib)
    span = angle_between(dl, dr)
    # observer on +x looking at -x with +z up: screen right is world +y
    ok = c0 < 1e-15 and dtop[2] > 0 and dleft[1] < 0 and abs(span - math.radians(50.0)) < 1e-14
    return ok, f"centre {c0:.1e}, top z {dtop[2]:.3f}, left y {dleft[1]:.3f}, span {span:.15f}"


def b_matches_v0(lib):
    """The impact parameter reported for a ray and its initial (u, u') lie on
    the same orbit: 1/b^2 = u'^2 + u^2 - 2Mu^3 (both conventions)."""
    worst = 0.0
    for ic in (0, 1):
        sc = W.Scene(mass=1.0, sky_seed=0, ic=ic)
        cam = W.Camera(20.0, 40.0, 9, 7)
        for y in range(cam.h):
            for x in range(cam.w):
                P, d = oracle.camera_ray(cam, x, y, lib=lib)
                q = oracle.plane_of_ray(sc, P, d, lib=lib)
                if q["b"] == 0.0:      # the radial centre ray has no plane
                    continue
                E = q["v0"] ** 2 + q["u0"] ** 2 - 2 * q["u0"] ** 3
                worst = max(worst, abs(E * q["b"] ** 2 - 1.0))
    return worst < 1e-13, f"max |E b^2 - 1| = {worst:.2e}"


def _hit_position(lib, sc, cam, x, y, out_i):
    """World position of a reported hit: the direction gives the plane angle,
    the oracle's own trajectory gives r there."""
    P, d = oracle.camera_ray(cam, x, y, lib=lib)
    q = oracle.plane_of_ray(sc, P, d, lib=lib)
    th, ph = out_i
    e = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    ang = math.atan2(float(np.dot(e, q["e2"])), float(np.dot(e, q["e1"]))) % (2 * math.pi)
    u, _ = oracle.orbit_sample(sc.mass, q["u0"], q["v0"], np.array([ang]), lib=lib)
    return e / u[0]


def hits_on_surfaces_m1(lib):
    """With M = 1, every reported disk hit lies in z = 0 with r in
    [r_in, r_out] and every sphere hit on its sphere's surface (the position
    rebuilt from the reported direction and the trajectory)."""
    sph = [W.Sphere((9.0, 3.0, 1.0), 1.8, (0.9, 0.5, 0.3)),
           W.Sphere((-6.0, 8.0, -2.0), 1.2, (0.4, 0.8, 0.6))]
    sc = W.Scene(mass=1.0, disk=(6.0, 18.0), spheres=tuple(sph), sky_seed=0)
    cam = W.Camera(35.0, 70.0, 40, 40, azim_deg=15.0, fov_deg=70.0)
    out = oracle.render(sc, [cam], lib=lib)
    worst_disk = worst_sph = 0.0
    nd = ns = 0
    for y in range(cam.h):
        for x in range(cam.w):
            i = y * cam.w + x
            f = int(out["flags"][i])
            if f & 0xFF not in (oracle.DISK, oracle.SPHERE) or out["ambig"][i]:
                continue
            X = _hit_position(lib, sc, cam, x, y, (out["theta"][i], out["phi"][i]))
            if f == oracle.DISK:
                nd += 1
                r = float(np.linalg.norm(X))
                err = abs(X[2]) + max(0.0, 6.0 - r) + max(0.0, r - 18.0)
                worst_disk = max(worst_disk, err)
            else:
                ns += 1
                k = f >> 8
                err = abs(float(np.linalg.norm(X - np.array(sph[k].center))) - sph[k].radius)
                worst_sph = max(worst_sph, err)
    ok = nd > 50 and ns >= 8 and worst_disk < 1e-8 and worst_sph < 1e-8
    return ok, f"disk {nd} hits err {worst_disk:.1e}; spheres {ns} hits err {worst_sph:.1e}"


def disk_colour_ends(lib):
    """Disk ramp t = (r_in/r)^(3/4) (thin-disk temperature law T ~ r^-3/4):
    white at the inner edge; red > green > blue and all channels falling
    with radius outside it (M = 0 face-on camera, hits at known radii)."""
    cam = W.Camera(30.0, 0.0, 33, 33, fov_deg=60.0)
    sc = W.Scene(mass=0.0, disk=(4.0, 16.0), sky_seed=0)
    out = oracle.render(sc, [cam], TIGHT, lib=lib)
    cols = []
    for y in range(cam.h):
        for x in range(cam.w):
            i = y * cam.w + x
            if out["flags"][i] != oracle.DISK:
                continue
            P, d = oracle.camera_ray(cam, x, y, lib=lib)
            t = -P[2] / d[2]
            r = float(np.linalg.norm(P + t * d))
            rgba = int(out["rgba"][i])
            cols.append((r, rgba & 255, (rgba >> 8) & 255, (rgba >> 16) & 255))
    cols.sort()
    if len(cols) < 100:
        return False, f"only {len(cols)} disk pixels"
    inner = cols[0]
    ok = inner[0] < 4.3 and min(inner[1:]) >= 225
    for a, b2 in zip(cols, cols[1:]):
        if b2[0] - a[0] > 1e-6 and any(b2[c] > a[c] + 1 for c in (1, 2, 3)):
            ok = False
    ok = ok and all(c[1] >= c[2] >= c[3] for c in cols)
    outer = cols[-1]
    # at r_out = 4 r_in the ramp is t = 4^(-3/4): clearly dimmer and redder
    ok = ok and outer[0] > 14.0 and outer[1] < 0.7 * inner[1] and outer[3] < 0.5 * outer[1]
    return ok, f"{len(cols)} disk pixels, inner colour {inner[1:]}, outer {outer[1:]}"


ALL = [first_integral, exit_angle, exit_angle_render_tol, weak_field,
       capture_iff_subcritical, photon_orbit, periastron, step_order,
       straight_lines_m0, disk_m0, spheres_m0, shadow_edge, einstein_ring,
       disk_radius_m1, splitmix_vector, sky_cells, camera_convention,
       b_matches_v0, hits_on_surfaces_m1, disk_colour_ends]


# --- the paper's fixed-step polyline (method 1; Sec. 2.1-2.2) ------------

def _gc(t1, p1, t2, p2):
    a = np.stack([np.sin(t1) * np.cos(p1), np.sin(t1) * np.sin(p1), np.cos(t1)], -1)
    b = np.stack([np.sin(t2) * np.cos(p2), np.sin(t2) * np.sin(p2), np.cos(t2)], -1)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, -1))


def polyline_straight_m0(lib):
    """At M = 0 the Runge-Kutta points lie on the straight ray to O(eps^4),
    so do the segments: escapes leave along the camera direction and disk
    hits are the ray-plane intersection (1e-7 rad)."""
    from dataclasses import replace
    w = W.config2(24, "fp64")
    w = replace(w, scene=replace(w.scene, mass=0.0))
    cam = w.cameras[0]
    got = oracle.render(w.scene, w.cameras, oracle.opts(eps=0.01, method=oracle.METHOD_POLYLINE),
                        lib=lib)
    worst, n_disk = 0.0, 0
    for idx in range(cam.w * cam.h):
        P, d = oracle.camera_ray(cam, idx % cam.w, idx // cam.w, lib=lib)
        fl = got["flags"][idx] & 0xFF
        th, ph = got["theta"][idx], got["phi"][idx]
        dd = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
        if fl == oracle.ESC:
            worst = max(worst, angle_between(dd, d))
        elif fl == oracle.DISK:
            X = P - P[2] / d[2] * d
            worst = max(worst, angle_between(dd, X))
            n_disk += 1
    return worst < 1e-7 and n_disk > 20, f"worst {worst:.2e} rad over {n_disk} disk hits"


def polyline_nodes(lib):
    """A segment crosses the disk plane on the line of nodes, so polyline
    disk hits point exactly where the adaptive method's do (1e-9 rad)."""
    w = W.config2(40, "fp64")
    ref = oracle.render(w.scene, w.cameras, oracle.opts(), lib=lib)
    got = oracle.render(w.scene, w.cameras, oracle.opts(eps=0.02, method=oracle.METHOD_POLYLINE),
                        lib=lib)
    both = ((got["flags"] & 0xFF) == oracle.DISK) & ((ref["flags"] & 0xFF) == oracle.DISK)
    ang = _gc(got["theta"][both], got["phi"][both], ref["theta"][both], ref["phi"][both])
    mx = float(ang.max()) if both.any() else 1.0
    return both.sum() > 100 and mx < 1e-9, f"{int(both.sum())} disk hits, max {mx:.2e} rad"


def polyline_escape_order(lib):
    """The escape angle's error against the adaptive method falls at third
    order in eps (classical Runge-Kutta points, linear interpolation of u
    where u'' vanishes with u): median ratios above 5.5 per halving."""
    w = W.config1(32)
    ref = oracle.render(w.scene, w.cameras, oracle.opts(), lib=lib)
    med = []
    for eps in (0.04, 0.02, 0.01):
        got = oracle.render(w.scene, w.cameras, oracle.opts(eps=eps, method=oracle.METHOD_POLYLINE),
                            lib=lib)
        esc = ((got["flags"] & 0xFF) == oracle.ESC) & ((ref["flags"] & 0xFF) == oracle.ESC)
        ang = _gc(got["theta"][esc], got["phi"][esc], ref["theta"][esc], ref["phi"][esc])
        med.append(float(np.median(ang)) if esc.any() else 1.0)
    ok = all(c / f > 5.5 for c, f in zip(med, med[1:])) and med[-1] < 1e-7
    return ok, "medians " + ", ".join(f"{m:.2e}" for m in med)


POLYLINE = [polyline_straight_m0, polyline_nodes, polyline_escape_order]


# --- anti-aliased pixels (n x n stratified samples, box filter) ---------

def spp_mean(lib):
    """A pixel rendered with n x n samples has, to one quantisation level,
    the mean colour of rays traced separately through the centres of an
    n x n grid over the pixel, and the centre ray's direction and flags."""
    w = W.config2(32, "fp64")
    cam = w.cameras[0]
    n = 3
    got = oracle.render(w.scene, w.cameras, oracle.opts(spp_n=n), lib=lib)
    one = oracle.render(w.scene, w.cameras, oracle.opts(), lib=lib)
    if not (np.array_equal(got["flags"], one["flags"])
            and np.array_equal(got["theta"], one["theta"], equal_nan=True)):
        return False, "directions or flags differ from the centre ray's"
    bad = mixed = 0
    for idx in range(0, cam.w * cam.h, 3):
        x, y = idx % cam.w, idx // cam.w
        cols = []
        for j in range(n):
            for i in range(n):
                P, d = oracle.camera_ray(cam, x + (i + 0.5) / n - 0.5, y + (j + 0.5) / n - 0.5,
                                         lib=lib)
                rgba = int(oracle.render_world_ray(w.scene, P, d, lib=lib)["rgba"])
                cols.append([(rgba >> (8 * c)) & 255 for c in range(3)])
        cols = np.array(cols, float)
        mixed += int(np.ptp(cols, axis=0).max() > 2)
        px = np.array([(int(got["rgba"][idx]) >> (8 * c)) & 255 for c in range(3)])
        bad += int(np.any(np.abs(px - cols.mean(axis=0)) > 1.0))
    return bad == 0 and mixed > 10, f"{bad} pixels off the sample mean, {mixed} edge pixels"


# --- Keplerian disk shading (Doppler and gravitational shift) ----------

def doppler_closed_form(lib):
    """The oracle's disk shift, worked in the local static frame with the
    special-relativistic Doppler factor, equals the covariant closed form
    g = sqrt(1 - 3M/r) / (sqrt(1 - 2M/r_obs) (1 + Omega lambda)) with
    Omega = sqrt(M/r^3) and lambda = b n_z the traced ray's angular momentum
    about the disk axis per unit energy (the photon's is -lambda), over
    random disk points, orbital planes and impact parameters (1e-12)."""
    rng = np.random.default_rng(3)
    worst = 0.0
    for _ in range(300):
        r = rng.uniform(6.0, 40.0)
        r_obs = rng.uniform(15.0, 100.0)
        a = rng.uniform(0, 2 * math.pi)
        x = r * np.array([math.cos(a), math.sin(a), 0.0])
        xr = x / r
        # orbital plane through the origin and x: normal n perpendicular to x
        w_ = rng.normal(size=3)
        n = w_ - np.dot(w_, xr) * xr
        n /= np.linalg.norm(n)
        t = np.cross(n, xr)                 # in-plane tangent, phi increasing
        u = 1.0 / r
        b = rng.uniform(B_C + 0.5, 60.0)
        v2 = 1.0 / b ** 2 - u * u + 2 * M * u ** 3
        if v2 < 0:
            continue
        v = math.sqrt(v2) * rng.choice([-1.0, 1.0])
        g = oracle.disk_g(M, r_obs, x, t, -v / (u * u), lib=lib)
        lam = b * n[2]
        want = math.sqrt(1 - 3 * M / r) / (math.sqrt(1 - 2 * M / r_obs)
                                          * (1 + math.sqrt(M / r ** 3) * lam))
        worst = max(worst, abs(g - want) / want)
    return worst < 1e-12, f"worst relative difference {worst:.2e}"


def doppler_approaching_side_bluer(lib):
    """Edge-on disk (camera at i = 90 deg, azimuth 0, prograde rotation about
    +z): disk pixels left of the hole (gas moving toward the camera) are
    shifted to the blue and right of it to the red, and the Doppler render
    is brighter on the approaching side."""
    from dataclasses import replace
    w = W.config2(64, "fp64")
    cam = replace(w.cameras[0], incl_deg=89.0)
    on = oracle.render(w.scene, [cam], oracle.opts(doppler=1), lib=lib)
    off = oracle.render(w.scene, [cam], oracle.opts(), lib=lib)
    disk = ((on["flags"] & 0xFF) == oracle.DISK)
    cols = np.arange(cam.w * cam.h) % cam.w
    left, right = disk & (cols < cam.w // 2 - 4), disk & (cols > cam.w // 2 + 4)
    def bright(im, m):
        rgba = im["rgba"][m].astype(np.int64)
        return float(np.mean(sum(((rgba >> (8 * c)) & 255) for c in range(3))))
    bl, br = bright(on, left), bright(on, right)
    ok = left.sum() > 20 and right.sum() > 20 and bl > 1.2 * br
    # without the shift both sides have the same brightness distribution
    ok = ok and abs(bright(off, left) - bright(off, right)) < 0.2 * bright(off, left)
    return ok, f"approaching {bl:.1f}, receding {br:.1f}"


DOPPLER = [doppler_closed_form, doppler_approaching_side_bluer]


# --- image sky (equirectangular texture, bilinear) -----------------------

def sky_texture_affine(lib):
    """Bilinear interpolation reproduces affine functions exactly: with a
    sky image whose red level is 20 + i and green 30 + 2 j at texel (i, j),
    every escaping ray away from the phi seam and the pole rows has red
    20 + x and green 30 + 2 y, x = phi w / 2 pi - 1/2, y = theta h / pi - 1/2,
    to the quantisation step; a texel-centre direction returns its texel."""
    from dataclasses import replace
    import numpy as np
    w_, h_ = 96, 48
    i = np.arange(w_)[None, :].repeat(h_, 0)
    j = np.arange(h_)[:, None].repeat(w_, 1)
    tex = (20 + i) | ((30 + 2 * j) << 8) | (100 << 16) | (255 << 24)
    tex = tex.astype(np.uint32)
    base = W.config1(40)
    scene = replace(base.scene, mass=0.0, sky_texture=tex)
    cam = replace(base.cameras[0], fov_deg=120.0)
    got = oracle.render(scene, [cam], oracle.opts(), lib=lib)
    esc = (got["flags"] & 0xFF) == oracle.ESC
    x = got["phi"][esc] / (2 * math.pi) * w_ - 0.5
    y = got["theta"][esc] / math.pi * h_ - 0.5
    inner = (x > 0.5) & (x < w_ - 1.5) & (y > 0.5) & (y < h_ - 1.5)
    red = (got["rgba"][esc] & 255).astype(float)
    green = ((got["rgba"][esc] >> 8) & 255).astype(float)
    err = max(float(np.max(np.abs(red[inner] - (20 + x[inner])))),
              float(np.max(np.abs(green[inner] - (30 + 2 * y[inner])))))
    # texel centre: direction of texel (i, j) = (7, 11)
    th, ph = (11 + 0.5) / h_ * math.pi, (7 + 0.5) / w_ * 2 * math.pi
    d = np.array([math.sin(th) * math.cos(ph), math.sin(th) * math.sin(ph), math.cos(th)])
    one = oracle.render_world_ray(scene, -100.0 * d, d, lib=lib)   # straight through the hole
    centre_ok = int(one["rgba"]) == int(tex[11, 7])
    return inner.sum() > 500 and err <= 0.5 + 1e-9 and centre_ok, \
        f"{int(inner.sum())} rays, max level error {err:.3f}, centre texel {'ok' if centre_ok else 'wrong'}"


SKY_TEXTURE = [sky_texture_affine]
