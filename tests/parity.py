"""Comparison of renderer outputs with the CPU oracle.

Tolerances (exit-direction great-circle error at the 99.9th percentile over
non-captured, non-ambiguous pixels; flags bit-exact outside the oracle's
ambiguity mask; at most 0.1% of all RGBA8 pixels, ambiguous ones included,
off by more than 1):
    FP64 1e-9 rad, FP32 / MIXED 1e-4 rad, SURROGATE 1e-3 rad.
The ambiguity thresholds scale with each mode's precision: a correct
renderer may decide a disk edge, sphere graze, sky-cell edge or the capture
boundary either way when it lies within the mode's error of it.
"""
from __future__ import annotations

import numpy as np

import oracle

OUTCOME = 0xFF8F   # ESC | CAPT | DISK | SPHERE | STEP_LIMIT bits and sphere index

DIR_TOL = {"fp64": 1e-9, "fp32": 1e-4, "mixed": 1e-4, "surrogate": 1e-3}

# ambiguity thresholds per mode: (eps_r [M], eps_ang [rad], eps_b [M])
AMBIG = {"fp64": (1e-7, 1e-9, 1e-6),
         "mixed": (2e-3, 2e-4, 1e-6),
         "fp32": (2e-3, 2e-4, 1e-6),
         "surrogate": (6e-2, 2e-3, 1e-6)}

# Pure FP32 has no FP64 band: its bar applies outside |b - b_c| < 0.05 M (the
# band the MIXED mode integrates in FP64); inside it the error is reported.
FP32_EXCLUDED_BAND = 0.05
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


def compare(got: dict, ref: dict, mode: str, exclude=None) -> dict:
    """Metrics of a render (numpy arrays theta, phi, flags, rgba) against the
    oracle's render of the same pixels; `exclude` removes pixels entirely
    (pure FP32 mode: the photon-sphere band, by default)."""
    if exclude is None and mode == "fp32":
        exclude = np.abs(ref["b"] - B_CRIT) < FP32_EXCLUDED_BAND
    if exclude is not None:
        keep = ~np.asarray(exclude, bool)
        got = {k: np.asarray(v)[keep] for k, v in got.items()}
        ref = {k: np.asarray(v)[keep] for k, v in ref.items()}
    flags = np.asarray(got["flags"]).astype(np.uint16)
    rflags = ref["flags"].astype(np.uint16)
    amb = ref["ambig"] != 0
    clean = ~amb
    n = len(rflags)
    flag_bad = int(np.sum((flags[clean] & OUTCOME) != (rflags[clean] & OUTCOME)))
    # directions: pixels the oracle gives a direction for, agreeing outcome
    same = clean & ((flags & OUTCOME) == (rflags & OUTCOME))
    has_dir = same & ~np.isnan(ref["theta"])
    ang = great_circle(got["theta"][has_dir], got["phi"][has_dir],
                       ref["theta"][has_dir], ref["phi"][has_dir])
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
        "flag_mismatch": flag_bad,
        "dir_p999": float(np.quantile(ang, 0.999)) if len(ang) else 0.0,
        "dir_max": float(ang.max()) if len(ang) else 0.0,
        "dir_nan_bad": nan_bad + nan_mismatch,
        "rgba_off_frac": float(rgba_off.mean()),
        "n_dir": int(len(ang)),
    }


def assert_parity(m: dict, mode: str) -> None:
    assert m["flag_mismatch"] == 0, m
    assert m["dir_nan_bad"] == 0, m
    assert m["dir_p999"] <= DIR_TOL[mode], m
    # at most 0.1% of the pixels may differ by more than 1 in a channel;
    # in images too small for that budget to hold one pixel, only pixels the
    # oracle marks ambiguous (hits on an edge, sky-cell borders) may differ
    assert m["rgba_off_frac"] <= 1e-3 or m["rgba_off_clean"] == 0, m
