"""Python access to the plain FP64 CPU oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
CPU-baseline leg of the benchmark may import this package.  It shares no code
with the CUDA renderer: its own C source, its own ctypes structures, its own
build line (plain gcc, no fused multiply-add contraction so that x86 and Arm
give the same bits).

Scene and camera values come in as plain Python objects with the attributes
of ``paper_2507_16165_gb300.workloads.Scene`` / ``Camera`` (duck-typed; this
module does not import them).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

MAX_SPHERES = 8
ESC, CAPT, DISK, SPHERE, STEP_LIMIT = 1, 2, 4, 8, 128
AMB_CAPT, AMB_DISK, AMB_SPHERE, AMB_SKY, AMB_DEGEN = 1, 2, 4, 8, 16


def build(out: str = LIB, src: str = SRC, openmp: bool = True) -> str:
    """Compile the oracle into a shared library (gcc, -O2, no FP contraction)."""
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off"]
    if openmp:
        cmd.append("-fopenmp")
    cmd += [src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True)
    return out


class _Sphere(ctypes.Structure):
    _fields_ = [("c", ctypes.c_double * 3), ("radius", ctypes.c_double),
                ("albedo", ctypes.c_double * 3)]


class _Scene(ctypes.Structure):
    _fields_ = [("mass", ctypes.c_double), ("disk_enabled", ctypes.c_int),
                ("disk_r_in", ctypes.c_double), ("disk_r_out", ctypes.c_double),
                ("n_spheres", ctypes.c_int), ("spheres", _Sphere * MAX_SPHERES),
                ("sky_seed", ctypes.c_uint64), ("ic", ctypes.c_int),
                ("sky_tex", ctypes.c_void_p), ("sky_w", ctypes.c_int), ("sky_h", ctypes.c_int)]


class _Camera(ctypes.Structure):
    _fields_ = [("r_obs", ctypes.c_double), ("incl_deg", ctypes.c_double),
                ("azim_deg", ctypes.c_double), ("fov_deg", ctypes.c_double),
                ("w", ctypes.c_int), ("h", ctypes.c_int)]


class _Opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("atol", ctypes.c_double),
                ("phi_max", ctypes.c_double), ("max_steps", ctypes.c_long),
                ("eps_r", ctypes.c_double), ("eps_ang", ctypes.c_double),
                ("eps_b", ctypes.c_double), ("method", ctypes.c_int), ("eps", ctypes.c_double),
                ("spp_n", ctypes.c_int), ("doppler", ctypes.c_int)]


METHOD_DP5 = 0
METHOD_POLYLINE = 1


_lock = threading.Lock()
_libs: dict[str, ctypes.CDLL] = {}

_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


def load(path: str = LIB) -> ctypes.CDLL:
    """Load (building first if needed) an oracle shared library."""
    with _lock:
        if path in _libs:
            return _libs[path]
        if path == LIB and (not os.path.exists(LIB)
                            or os.path.getmtime(LIB) < os.path.getmtime(SRC)):
            build()
        lib = ctypes.CDLL(path)
        lib.or_render.restype = ctypes.c_int
        lib.or_render.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Camera),
                                  ctypes.c_int, ctypes.POINTER(_Opts), ctypes.c_int] + [_VP] * 7
        lib.or_render_pixels.restype = ctypes.c_int
        lib.or_render_pixels.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Camera),
                                         ctypes.c_int, ctypes.POINTER(_Opts), ctypes.c_int,
                                         ctypes.c_long, _VP, _VP, _VP] + [_VP] * 7
        lib.or_render_world_ray.restype = ctypes.c_int
        lib.or_render_world_ray.argtypes = [ctypes.POINTER(_Scene), ctypes.POINTER(_Opts),
                                            _VP, _VP] + [_VP] * 7
        lib.or_camera_ray.restype = None
        lib.or_camera_ray.argtypes = [ctypes.POINTER(_Camera), ctypes.c_double,
                                      ctypes.c_double, _VP, _VP]
        lib.or_plane_of_ray.restype = None
        lib.or_plane_of_ray.argtypes = [ctypes.POINTER(_Scene), _VP, _VP, _D, _D, _D, _D,
                                        _VP, _VP]
        lib.or_orbit_exit.restype = ctypes.c_int
        lib.or_orbit_exit.argtypes = [ctypes.c_double] * 6 + [ctypes.c_long, _D,
                                                               ctypes.POINTER(ctypes.c_long)]
        lib.or_orbit_steps.restype = ctypes.c_long
        lib.or_orbit_steps.argtypes = [ctypes.c_double] * 6 + [ctypes.c_long, _VP, _VP, _VP]
        lib.or_orbit_sample.restype = ctypes.c_int
        lib.or_orbit_sample.argtypes = [ctypes.c_double] * 5 + [ctypes.c_long, _VP, _VP, _VP]
        lib.or_sky_rgb.restype = None
        lib.or_sky_rgb.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_double, _VP]
        lib.or_splitmix64.restype = ctypes.c_uint64
        lib.or_splitmix64.argtypes = [ctypes.c_uint64]
        lib.or_threads.restype = ctypes.c_int
        lib.or_threads.argtypes = [ctypes.c_int]
        lib.or_disk_g.restype = ctypes.c_double
        lib.or_disk_g.argtypes = [ctypes.c_double, ctypes.c_double, _VP, _VP, ctypes.c_double]
        _libs[path] = lib
        return lib


def _scene(scene) -> _Scene:
    s = _Scene()
    s.mass = float(scene.mass)
    disk = getattr(scene, "disk", None)
    s.disk_enabled = 1 if disk is not None else 0
    if disk is not None:
        s.disk_r_in, s.disk_r_out = float(disk[0]), float(disk[1])
    sph = list(getattr(scene, "spheres", ()))
    if len(sph) > MAX_SPHERES:
        raise ValueError("at most 8 spheres")
    s.n_spheres = len(sph)
    for k, sp in enumerate(sph):
        s.spheres[k].c[:] = [float(x) for x in sp.center]
        s.spheres[k].radius = float(sp.radius)
        s.spheres[k].albedo[:] = [float(x) for x in sp.albedo]
    s.sky_seed = int(scene.sky_seed)
    s.ic = int(getattr(scene, "ic", 0))
    tex = getattr(scene, "sky_texture", None)
    if tex is not None:
        tex = np.ascontiguousarray(tex, np.uint32)
        s._tex = tex                     # keeps the texels alive with the struct
        s.sky_tex = tex.ctypes.data
        s.sky_h, s.sky_w = tex.shape
    return s


def _cams(cams) -> ctypes.Array:
    arr = (_Camera * len(cams))()
    for k, c in enumerate(cams):
        arr[k].r_obs, arr[k].incl_deg = float(c.r_obs), float(c.incl_deg)
        arr[k].azim_deg, arr[k].fov_deg = float(c.azim_deg), float(c.fov_deg)
        arr[k].w, arr[k].h = int(c.w), int(c.h)
    return arr


def opts(rtol=1e-10, atol=1e-10, phi_max=64.0, max_steps=100000,
         eps_r=1e-7, eps_ang=1e-9, eps_b=1e-6, method=METHOD_DP5, eps=0.01, spp_n=1,
         doppler=0) -> _Opts:
    """Integration tolerances, caps and ambiguity thresholds; method 1 is the
    paper's fixed-step polyline with step eps (Sec. 2.1-2.2); spp_n > 1
    averages n x n stratified samples per pixel into its colour; doppler = 1
    shades the disk as Keplerian gas with its Doppler and gravitational shift."""
    return _Opts(rtol, atol, phi_max, max_steps, eps_r, eps_ang, eps_b, method, eps, spp_n,
                 doppler)


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _outputs(n: int) -> dict:
    return dict(theta=np.empty(n, np.float64), phi=np.empty(n, np.float64),
                flags=np.empty(n, np.uint16), rgba=np.empty(n, np.uint32),
                ambig=np.empty(n, np.uint8), b=np.empty(n, np.float64),
                steps=np.empty(n, np.int32))


_ORDER = ("theta", "phi", "flags", "rgba", "ambig", "b", "steps")


def render(scene, cams, o: _Opts | None = None, nthreads: int = 1,
           lib: ctypes.CDLL | None = None) -> dict:
    """Render every pixel of every camera (camera-major, row-major)."""
    lib = lib or load()
    o = o or opts()
    n = sum(int(c.w) * int(c.h) for c in cams)
    out = _outputs(n)
    rc = lib.or_render(ctypes.byref(_scene(scene)), _cams(cams), len(cams),
                       ctypes.byref(o), nthreads, *[_ptr(out[k]) for k in _ORDER])
    if rc != 0:
        raise RuntimeError("or_render failed")
    return out


def render_pixels(scene, cams, cam_idx, px, py, o: _Opts | None = None,
                  nthreads: int = 1, lib: ctypes.CDLL | None = None) -> dict:
    """Render an explicit list of pixels (camera index, column, row)."""
    lib = lib or load()
    o = o or opts()
    cam_idx = np.ascontiguousarray(cam_idx, np.int32)
    px = np.ascontiguousarray(px, np.int32)
    py = np.ascontiguousarray(py, np.int32)
    n = len(cam_idx)
    out = _outputs(n)
    rc = lib.or_render_pixels(ctypes.byref(_scene(scene)), _cams(cams), len(cams),
                              ctypes.byref(o), nthreads, n, _ptr(cam_idx), _ptr(px),
                              _ptr(py), *[_ptr(out[k]) for k in _ORDER])
    if rc != 0:
        raise RuntimeError("or_render_pixels failed")
    return out


def render_world_ray(scene, P, d, o: _Opts | None = None,
                     lib: ctypes.CDLL | None = None) -> dict:
    """Trace one world ray from position P along unit direction d."""
    lib = lib or load()
    o = o or opts()
    P = np.ascontiguousarray(P, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    out = _outputs(1)
    lib.or_render_world_ray(ctypes.byref(_scene(scene)), ctypes.byref(o), _ptr(P),
                            _ptr(d), *[_ptr(out[k]) for k in _ORDER])
    return {k: v[0] for k, v in out.items()}


def camera_ray(cam, px: float, py: float, lib=None):
    lib = lib or load()
    P = np.empty(3)
    d = np.empty(3)
    lib.or_camera_ray(ctypes.byref(_cams([cam])[0]), px, py, _ptr(P), _ptr(d))
    return P, d


def plane_of_ray(scene, P, d, lib=None) -> dict:
    lib = lib or load()
    P = np.ascontiguousarray(P, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    b, u0, v0, psi0 = (ctypes.c_double() for _ in range(4))
    e1, e2 = np.empty(3), np.empty(3)
    lib.or_plane_of_ray(ctypes.byref(_scene(scene)), _ptr(P), _ptr(d), ctypes.byref(b),
                        ctypes.byref(u0), ctypes.byref(v0), ctypes.byref(psi0),
                        _ptr(e1), _ptr(e2))
    return dict(b=b.value, u0=u0.value, v0=v0.value, psi0=psi0.value, e1=e1, e2=e2)


def orbit_exit(M, u0, v0, rtol=1e-10, atol=1e-10, phi_max=64.0, max_steps=100000,
               lib=None):
    """(flag, phi_event, attempted steps) of a bare orbit: escape or capture."""
    lib = lib or load()
    phi = ctypes.c_double()
    steps = ctypes.c_long()
    f = lib.or_orbit_exit(M, u0, v0, rtol, atol, phi_max, max_steps, ctypes.byref(phi),
                          ctypes.byref(steps))
    return f, phi.value, steps.value


def orbit_steps(M, u0, v0, phi_end, rtol=1e-10, atol=1e-10, cap=200000, lib=None):
    """Accepted step end points (phi, u, v) of a bare orbit up to phi_end."""
    lib = lib or load()
    ph, u, v = np.empty(cap), np.empty(cap), np.empty(cap)
    n = lib.or_orbit_steps(M, u0, v0, rtol, atol, phi_end, cap, _ptr(ph), _ptr(u), _ptr(v))
    return ph[:n], u[:n], v[:n]


def orbit_sample(M, u0, v0, phis, rtol=1e-10, atol=1e-10, lib=None):
    """u and u' of a bare orbit at increasing angles, from the interpolant."""
    lib = lib or load()
    phis = np.ascontiguousarray(phis, np.float64)
    u, v = np.empty_like(phis), np.empty_like(phis)
    rc = lib.or_orbit_sample(M, u0, v0, rtol, atol, len(phis), _ptr(phis), _ptr(u), _ptr(v))
    if rc != 0:
        raise RuntimeError("or_orbit_sample did not reach the last angle")
    return u, v


def sky_rgb(seed: int, theta: float, phi: float, lib=None) -> np.ndarray:
    lib = lib or load()
    out = np.empty(3)
    lib.or_sky_rgb(seed, theta, phi, _ptr(out))
    return out


def splitmix64(x: int, lib=None) -> int:
    lib = lib or load()
    return int(lib.or_splitmix64(x))


def threads(n: int = 0, lib=None) -> int:
    lib = lib or load()
    return int(lib.or_threads(n))


def disk_g(M: float, r_obs: float, x, t, dr_dphi: float, lib=None) -> float:
    """Frequency ratio camera / emitter of the Keplerian disk at point x for
    a traced ray with in-plane unit tangent t and dr/dphi there."""
    lib = lib or load()
    x = np.ascontiguousarray(x, np.float64)
    t = np.ascontiguousarray(t, np.float64)
    return float(lib.or_disk_g(M, r_obs, _ptr(x), _ptr(t), dr_dphi))
