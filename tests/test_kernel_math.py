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
