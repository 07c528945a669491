"""Seeded synthetic inputs: scenes and camera sets for the five workloads.

This module only generates inputs (sphere positions, camera lists, sample
draws).  It holds none of the renderer's arithmetic and is the one module the
CUDA path and the CPU oracle both take values from.  Random draws use
splitmix64 (Steele, Lea & Flood 2014) as a counter-based stream.

The paper renders against NASA/ESA background photographs (Sec. 3.1), which
are not available here; every workload uses the procedural checkerboard sky
instead, which costs the same per ray.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

MASK64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 stream: state advances by the golden gamma each draw."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


@dataclass(frozen=True)
class Sphere:
    center: tuple
    radius: float
    albedo: tuple


@dataclass(frozen=True)
class Scene:
    mass: float = 1.0
    disk: tuple | None = None          # (r_in, r_out) or None
    spheres: tuple = ()
    sky_seed: int = 0
    ic: int = 0                        # 0 static observer, 1 Euclidean
    # optional equirectangular RGBA8 sky image (h x w uint32), None: checker
    sky_texture: object = field(default=None, compare=False, hash=False)


@dataclass(frozen=True)
class Camera:
    r_obs: float
    incl_deg: float
    w: int
    h: int
    azim_deg: float = 0.0
    fov_deg: float = 60.0


@dataclass(frozen=True)
class Workload:
    name: str
    scene: Scene
    cameras: tuple
    mode: str                          # "fp64", "fp32", "mixed", "surrogate"
    rtol: float
    atol: float
    band: float = 0.05
    notes: dict = field(default_factory=dict)

    @property
    def n_rays(self) -> int:
        return sum(c.w * c.h for c in self.cameras)


def seeded_spheres(seed: int = 0, n: int = 8, r_range=(8.0, 25.0),
                   radius_range=(0.5, 2.0), mass: float = 1.0) -> tuple:
    """n non-overlapping spheres: centre distance ~ U[r_range], direction
    uniform on the unit sphere, radius ~ U[radius_range], albedo ~ U[0.3, 1]^3."""
    rng = SplitMix64(seed)
    out: list[Sphere] = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place spheres")
        r = rng.uniform(*r_range)
        z = rng.uniform(-1.0, 1.0)
        a = rng.uniform(0.0, 2.0 * math.pi)
        s = math.sqrt(max(0.0, 1.0 - z * z))
        c = (r * s * math.cos(a), r * s * math.sin(a), r * z)
        R = rng.uniform(*radius_range)
        alb = (rng.uniform(0.3, 1.0), rng.uniform(0.3, 1.0), rng.uniform(0.3, 1.0))
        if r - R <= 3.0 * mass:
            continue
        if any(math.dist(c, o.center) < R + o.radius for o in out):
            continue
        out.append(Sphere(c, R, alb))
    return tuple(out)


def batch_cameras(seed: int = 0, n: int = 64, sizes=(256, 512, 1024, 2048),
                  r_range=(15.0, 100.0), incl_range=(0.0, 89.0)) -> tuple:
    """Orbit sequence of n cameras: square resolution drawn from sizes,
    r_obs log-uniform in r_range, inclination uniform in incl_range, azimuth
    stepping once around the hole."""
    rng = SplitMix64(seed ^ 0x5EED0005)
    cams = []
    for k in range(n):
        size = sizes[rng.next_u64() % len(sizes)]
        r = math.exp(rng.uniform(math.log(r_range[0]), math.log(r_range[1])))
        inc = rng.uniform(*incl_range)
        cams.append(Camera(r_obs=r, incl_deg=inc, w=size, h=size,
                           azim_deg=360.0 * k / n))
    return tuple(cams)


def config1(size: int = 64) -> Workload:
    """64x64 pinhole, M = 1, r_obs = 30M, 60 deg FOV, no disk, sky seed 0,
    FP64 Dormand-Prince rtol = atol = 1e-10.  The inclination is not fixed by
    the workload text; 90 deg (observer in the equatorial plane) is used."""
    return Workload("c1_fp64_64", Scene(mass=1.0, sky_seed=0),
                    (Camera(30.0, 90.0, size, size),), "fp64", 1e-10, 1e-10)


def config2(size: int = 1024, mode: str = "fp64") -> Workload:
    """1024^2, r_obs = 40M, inclination 80 deg, disk [6M, 20M], sky seed 0."""
    rtol, atol = (1e-10, 1e-10) if mode == "fp64" else (1e-5, 1e-7)
    return Workload(f"c2_{mode}_{size}", Scene(mass=1.0, disk=(6.0, 20.0), sky_seed=0),
                    (Camera(40.0, 80.0, size, size),), mode, rtol, atol)


def config3(size: int = 4096, mode: str = "mixed") -> Workload:
    """4096^2, r_obs = 50M, inclination 75 deg, disk [6M, 30M], 8 spheres
    (seed 0), FP32 stepping with FP64 in the band |b - 3 sqrt(3) M| < 0.05M."""
    rtol, atol = (1e-10, 1e-10) if mode == "fp64" else (1e-5, 1e-7)
    sc = Scene(mass=1.0, disk=(6.0, 30.0), spheres=seeded_spheres(0), sky_seed=0)
    return Workload(f"c3_{mode}_{size}", sc, (Camera(50.0, 75.0, size, size),), mode,
                    rtol, atol, band=0.05)


def config4(size: int = 4096, spheres: bool = True) -> Workload:
    """The config-3 scene rendered through the MLP surrogate with fallback."""
    w = config3(size, "surrogate")
    if not spheres:
        w = replace(w, scene=replace(w.scene, spheres=()), name=w.name + "_nosph")
    return w


def config5(n_cams: int = 64, scale: int = 1) -> Workload:
    """64 cameras of uneven resolution in one launch; disk [6M, 20M], sky seed 0.
    scale > 1 divides every resolution (for fast tests)."""
    cams = batch_cameras(0, n_cams)
    if scale > 1:
        cams = tuple(replace(c, w=max(8, c.w // scale), h=max(8, c.h // scale)) for c in cams)
    return Workload(f"c5_batch{n_cams}", Scene(mass=1.0, disk=(6.0, 20.0), sky_seed=0),
                    cams, "fp32", 1e-5, 1e-7)


def surrogate_samples(n: int, seed: int = 0, b_lo: float = 3.0 * math.sqrt(3.0) + 1e-4,
                      b_hi: float = 1e3, r_range=(15.0, 100.0)):
    """Training inputs for the surrogate: b log-uniform in [b_lo, b_hi],
    r_obs uniform in r_range, psi0 uniform in (0, pi]; returned as three
    Python lists (use numpy in callers for large n)."""
    import numpy as np
    rng = np.random.Generator(np.random.Philox(key=seed))
    lb = rng.uniform(math.log(b_lo), math.log(b_hi), n)
    r = rng.uniform(r_range[0], r_range[1], n)
    psi = math.pi - rng.uniform(0.0, math.pi, n)     # (0, pi]
    return np.exp(lb), r, psi


def reachable_surrogate_samples(n: int, seed: int = 0, b_lo: float = 3.0 * math.sqrt(3.0) + 1e-4,
                                b_hi: float = 1e3, r_range=(15.0, 100.0)):
    """n training inputs drawn as surrogate_samples draws them, keeping only
    pairs (b, r_obs) a static observer at r_obs can receive: b below
    r_obs / sqrt(1 - 2/r_obs) (the ray through the image edge at 90 degrees;
    units of M).  The kept pairs follow the same density restricted to that
    domain, and all n of them are valid integrator samples."""
    import numpy as np
    bs, rs, ps = [], [], []
    have, k = 0, 0
    while have < n:
        b, r, psi = surrogate_samples(max(2 * (n - have), 1024), seed * 1009 + k, b_lo, b_hi, r_range)
        keep = b < (1.0 - 1e-6) * r / np.sqrt(1.0 - 2.0 / r)
        bs.append(b[keep])
        rs.append(r[keep])
        ps.append(psi[keep])
        have += int(keep.sum())
        k += 1
    return (np.concatenate(bs)[:n], np.concatenate(rs)[:n], np.concatenate(ps)[:n])


def sky_texture(seed: int = 0, w: int = 512, h: int = 256):
    """A synthetic equirectangular RGBA8 sky image (h x w, uint32), standing
    in for the paper's background photographs: a smooth seeded colour field
    (a few random low-order waves in theta and phi) with a sprinkling of
    bright one-texel stars."""
    import numpy as np
    rng = np.random.Generator(np.random.Philox(key=seed))
    th = (np.arange(h) + 0.5) / h * math.pi
    ph = (np.arange(w) + 0.5) / w * 2 * math.pi
    T, P = np.meshgrid(th, ph, indexing="ij")
    img = np.zeros((h, w, 3))
    for c in range(3):
        acc = np.full((h, w), 0.35)
        for _ in range(4):
            k, m = rng.integers(1, 6), rng.integers(1, 6)
            acc += rng.uniform(0.05, 0.15) * np.sin(k * T + rng.uniform(0, 6.3)) * \
                np.cos(m * P + rng.uniform(0, 6.3))
        img[..., c] = acc
    stars = rng.random((h, w)) < 0.004
    img[stars] = 1.0
    q = np.clip(np.floor(img * 255 + 0.5), 0, 255).astype(np.uint32)
    return q[..., 0] | (q[..., 1] << 8) | (q[..., 2] << 16) | (np.uint32(255) << 24)
