"""Polynomial inverse trigonometric functions of the FP32 kernels
(Abramowitz & Stegun 4.4.49 for arctan, 4.4.46 for arccos): the
coefficients are read from the CUDA source and evaluated here in FP64 over
a dense grid, so a mistyped coefficient shows as an error above the
published bound (2e-8) without a GPU."""
import os
import re

import numpy as np

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2507_16165_gb300", "csrc", "tracer.cuh")


def _body(name: str) -> str:
    text = open(SRC).read()
    i = text.index(name)
    return text[i:text.index("\n}\n", i)]


def _floats(body: str) -> list[float]:
    return [float(x) for x in re.findall(r"(-?\d+\.\d+)f", body)]


def test_arctan_polynomial_within_published_bound():
    c = _floats(_body("float atan_unit(float t)"))
    # Horner coefficients from t^16 down to t^2, applied to t^2
    assert len(c) == 8
    t = np.linspace(-1.0, 1.0, 2_000_001)
    t2 = t * t
    p = np.full_like(t, c[0])
    for k in c[1:]:
        p = p * t2 + k
    approx = t + t * t2 * p
    assert np.max(np.abs(approx - np.arctan(t))) < 2e-8


def test_arccos_polynomial_within_published_bound():
    c = _floats(_body("float m_acos(float x)"))
    # first float is the clamp 1.0f, then Horner coefficients a7 .. a0, then pi
    coeffs = [x for x in c if abs(x) < 1.6 and x != 1.0][:8]
    assert len(coeffs) == 8
    a = np.linspace(0.0, 1.0, 2_000_001)
    p = np.full_like(a, coeffs[0])
    for k in coeffs[1:]:
        p = p * a + k
    assert np.max(np.abs(np.sqrt(1.0 - a) * p - np.arccos(a))) < 2.5e-8


def test_periastron_bound_behind_the_sphere_cull():
    """The kernels drop sphere k from a ray's mask when b exceeds
    (|c_k| + R_k)(1 + 1e-5) + 2.25M, relying on r_p >= b - 2.2M for every
    unbound orbit: with b = r_p sqrt(r_p / (r_p - 2M)) from the first
    integral at the turning point, b - r_p is largest (3 sqrt(3) - 3 =
    2.196) at the photon orbit r_p = 3M and falls toward M at large r_p.
    Checked on a dense grid of r_p, and against the cubic's middle root for
    sampled b (the periastron the oracle solves for)."""
    rp = np.concatenate([np.linspace(3.0, 4.0, 200001), np.geomspace(4.0, 1e8, 200001)])
    excess = rp * np.sqrt(rp / (rp - 2.0)) - rp
    assert excess.max() <= 3.0 * np.sqrt(3.0) - 3.0 + 1e-12 < 2.2
    assert excess.min() > 1.0 - 1e-6
    for b in np.geomspace(3.0 * np.sqrt(3.0) * (1 + 1e-9), 1e5, 400):
        roots = np.sort(np.roots([2.0, -1.0, 0.0, 1.0 / b**2]).real)
        r_p = 1.0 / roots[1]
        assert r_p >= b - 2.2
    src = open(os.path.join(os.path.dirname(SRC), "bh_types.cuh")).read()
    assert "* (1.0 + 1e-5) + 2.25 * s.M" in src
