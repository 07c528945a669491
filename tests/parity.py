"""Comparison of renderer outputs with the CPU oracle.

Bars (every form, every pixel, no exclusions):
  - flags bit-exact outside the oracle's ambiguity mask;
  - exit-direction great-circle error at the 99.9th percentile over pixels
    the oracle gives a direction for (not captured, not ambiguous):
    FP64 1e-9 rad, FP32 / MIXED 1e-4 rad, SURROGATE 1e-3 rad;
  - at most 0.1% of all RGBA8 pixels, ambiguous ones included, off by more
    than 1 in a channel.  Only where 0.1% of the image is less than one
    pixel (under 1000 pixels) does the budget become "no pixel outside the
    ambiguity mask";
  - the ambiguity mask itself covers at most AMBIG_FRAC_MAX of the pixels.

The ambiguity mask holds the pixels whose outcome a correct renderer of the
form may decide either way because a boundary lies within the form's own
error of them.  Its widths follow from each form's bounds:
  - eps_ang (sky-cell edges): twice the form's direction bound, since the
    bound holds at the 99.9th percentile and the tail reaches about twice it
    (FP32 2e-4, surrogate 2e-3 rad); FP64 keeps the oracle's 1e-9 rad;
  - eps_r (disk edges, sphere grazes): the hit radius moves by r times the
    relative error of the hit position, at most r_out = 30 M times the
    direction bound for the integrator forms (3e-3 M) and r_out times the
    calibrated 2e-3 relative crossing-radius bound for the surrogate
    (6e-2 M); FP64 keeps 1e-7 M;
  - eps_b (the capture boundary |b - b_c|): 1e-6 M, the workload's band,
    for FP64, MIXED and SURROGATE (their near-critical rays are set up and
    integrated in FP64).  The pure FP32 form computes b itself in FP32: the
    camera ray, plane reduction and b take about ten roundings of relative
    size 6e-8 each, so b carries an error of a few 1e-6 M at b_c = 5.2 M and
    the form cannot place the boundary closer than that; its band is
    1e-5 M.
"""
from __future__ import annotations

import numpy as np

import oracle

OUTCOME = 0xFF8F   # ESC | CAPT | DISK | SPHERE | STEP_LIMIT bits and sphere index

DIR_TOL = {"fp64": 1e-9, "fp32": 1e-4, "mixed": 1e-4, "surrogate": 1e-3}

# ambiguity thresholds per mode: (eps_r [M], eps_ang [rad], eps_b [M])
AMBIG = {"fp64": (1e-7, 1e-9, 1e-6),
         "mixed": (3e-3, 2e-4, 1e-6),
         "fp32": (3e-3, 2e-4, 1e-5),
         "surrogate": (6e-2, 2e-3, 1e-6)}

# Largest share of the pixels the mask may cover, for images of at least
# 1000 pixels (measured at 4096^2: FP64 none, FP32 and MIXED 0.3%, surrogate
# 3.4%; a camera on the pole axis, where the sky cells' phi edges meet, 0.5%
# in FP64).  A pixel rendered with n rays (anti-aliasing) is ambiguous when
# any of its rays is, so its share scales with n.
AMBIG_FRAC_MAX = {"fp64": 1e-2, "fp32": 1e-2, "mixed": 1e-2, "surrogate": 6e-2}

B_CRIT = 3.0 * np.sqrt(3.0)


def oracle_opts(mode: str):
    er, ea, eb = AMBIG[mode]
    return oracle.opts(rtol=1e-10, atol=1e-10, eps_r=er, eps_ang=ea, eps_b=eb)


def unit(theta, phi):
    theta = np.asarray(theta, np.float64)
    phi = np.asarray(phi, np.float64)
    return np.stack([np.sin(theta) * np.cos(phi), np.sin(theta) * np.sin(phi), np.cos(theta)], -1)


def great_circle(t1, p1, t2, p2):
    a, b = unit(t1, p1), unit(t2, p2)
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def weighted_quantile(x: np.ndarray, w: np.ndarray, q: float) -> float:
    """The q-quantile of values x drawn with weights w (the smallest x whose
    cumulative weight reaches q of the total)."""
    if len(x) == 0:
        return 0.0
    o = np.argsort(x)
    cw = np.cumsum(w[o])
    return float(x[o][min(len(x) - 1, int(np.searchsorted(cw, q * cw[-1])))])


def compare(got: dict, ref: dict, mode: str, weight=None) -> dict:
    """Metrics of a render (numpy arrays theta, phi, flags, rgba) against the
    oracle's render of the same pixels.  `weight` (one per pixel) makes the
    quantile and the RGBA fraction those of the image a stratified sample
    was drawn from: each sampled pixel stands for `weight` pixels of it.
    Flags and NaNs are checked on every sampled pixel regardless."""
    flags = np.asarray(got["flags"]).astype(np.uint16)
    rflags = ref["flags"].astype(np.uint16)
    amb = ref["ambig"] != 0
    clean = ~amb
    n = len(rflags)
    flag_bad = int(np.sum((flags[clean] & OUTCOME) != (rflags[clean] & OUTCOME)))
    # directions: pixels the oracle gives a direction for, agreeing outcome
    same = clean & ((flags & OUTCOME) == (rflags & OUTCOME))
    has_dir = same & ~np.isnan(ref["theta"])
    ang = great_circle(np.asarray(got["theta"])[has_dir], np.asarray(got["phi"])[has_dir],
                       ref["theta"][has_dir], ref["phi"][has_dir])
    wt = np.ones(n) if weight is None else np.asarray(weight, np.float64)
    nan_bad = int(np.sum(np.isnan(np.asarray(got["theta"], np.float64)[has_dir])))
    # directions must be NaN exactly where the oracle's are (captured)
    nan_mismatch = int(np.sum(np.isnan(np.asarray(got["theta"], np.float64)[same])
                              != np.isnan(ref["theta"][same])))
    g = np.asarray(got["rgba"]).astype(np.uint32)
    r = ref["rgba"].astype(np.uint32)
    diff = np.zeros(n, np.int32)
    for c in range(4):
        diff = np.maximum(diff, np.abs(((g >> (8 * c)) & 255).astype(np.int32)
                                       - ((r >> (8 * c)) & 255).astype(np.int32)))
    rgba_off = diff > 1
    return {
        "rgba_off_clean": int(np.sum(rgba_off & clean)),
        "rgba_off_ambig": int(np.sum(rgba_off & amb)),
        "n": n,
        "n_ambig": int(amb.sum()),
        "ambig_frac": float(np.sum(wt * amb) / np.sum(wt)) if n else 0.0,
        "flag_mismatch": flag_bad,
        "dir_p999": weighted_quantile(ang, wt[has_dir], 0.999),
        "dir_max": float(ang.max()) if len(ang) else 0.0,
        "dir_nan_bad": nan_bad + nan_mismatch,
        "rgba_off_frac": float(np.sum(wt * rgba_off) / np.sum(wt)) if n else 0.0,
        "n_dir": int(len(ang)),
    }


def assert_parity(m: dict, mode: str, rays_per_pixel: int = 1) -> None:
    assert m["flag_mismatch"] == 0, m
    assert m["dir_nan_bad"] == 0, m
    assert m["dir_p999"] <= DIR_TOL[mode], m
    if m["n"] >= 1000:
        # 0.1% of the pixels, ambiguous ones counted, may be off by more than 1
        assert m["rgba_off_frac"] <= 1e-3, m
        assert m["ambig_frac"] <= AMBIG_FRAC_MAX[mode] * rays_per_pixel, m
    else:
        # a budget under one pixel: no pixel outside the ambiguity mask (a
        # share of the mask means nothing in images this small: a column
        # through the image centre can lie on a sky-cell edge entirely)
        assert m["rgba_off_clean"] == 0, m


def band_pixels(cam, lo: float, hi: float, mass: float = 1.0, ic: int = 0) -> np.ndarray:
    """Pixel indices (row-major) of a camera looking at the hole whose impact
    parameter satisfies lo <= |b - b_c| < hi, from the pixel centre's image-
    plane radius rho = tan(alpha): b = r sin(alpha) / sqrt(1 - 2M/r) (static
    observer) or r sin(alpha) / sqrt(1 - 2M sin^2(alpha) / r) (Euclidean)."""
    s = np.tan(np.radians(cam.fov_deg) / 2.0)
    sy_half = s * cam.h / cam.w
    x = (np.arange(cam.w) + 0.5) * (2.0 * s / cam.w) - s
    y = sy_half - (np.arange(cam.h) + 0.5) * (2.0 * sy_half / cam.h)
    rho2 = x[None, :] ** 2 + y[:, None] ** 2
    s2 = rho2 / (1.0 + rho2)
    r = cam.r_obs
    if ic == 0:
        b = r * np.sqrt(s2) / np.sqrt(1.0 - 2.0 * mass / r)
    else:
        b = r * np.sqrt(s2) / np.sqrt(1.0 - 2.0 * mass * s2 / r)
    d = np.abs(b - 3.0 * np.sqrt(3.0) * mass).ravel()
    return np.flatnonzero((d >= lo) & (d < hi))
