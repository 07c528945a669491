"""Closed forms of Schwarzschild photon orbits, independent of the oracle.

Everything here follows from the first integral of Eq. 1 (sign reconciled):
    (du/dphi)^2 = P(u) = 1/b^2 - u^2 + 2 M u^3 = 2M (u - u1)(u - u2)(u - u3)
with real roots u1 < 0 < u2 <= u3 when b >= 3 sqrt(3) M.  The angle swept
between two values of u on one leg of the orbit is an elliptic integral of
the first kind, evaluated with Carlson's R_F through the cubic-case reduction
(DLMF 19.29.4-19.29.5):
    int_y^x prod_i (a_i + b_i t)^(-1/2) dt = 2 R_F(U12^2, U13^2, U23^2),
    U_ij = (X_i X_j Y_k + Y_i Y_j X_k) / (x - y),  X_i = sqrt(a_i + b_i x),
    Y_i = sqrt(a_i + b_i y).
R_F comes from scipy.special.elliprf; a second, quadrature-based route is
kept to cross-check the reduction itself.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize
from scipy.special import elliprf

B_CRIT = 3.0 * math.sqrt(3.0)


def cubic_roots(M: float, b: float):
    """Real roots u1 < u2 <= u3 of 2M u^3 - u^2 + 1/b^2 (b > b_c)."""
    r = np.roots([2.0 * M, -1.0, 0.0, 1.0 / (b * b)])
    r = np.sort(r.real[np.abs(r.imag) < 1e-9 * np.abs(r).max()])
    if len(r) != 3:
        raise ValueError("b below the critical impact parameter: one real root")
    # polish with Newton in float64
    out = []
    for x in r:
        for _ in range(3):
            f = 2 * M * x ** 3 - x * x + 1 / (b * b)
            df = 6 * M * x * x - 2 * x
            if df != 0:
                x = x - f / df
        out.append(x)
    return tuple(sorted(out))


def leg_angle(M: float, b: float, y: float, x: float) -> float:
    """int_y^x du / sqrt(P(u)) for u1 <= y < x <= u2 (Carlson R_F)."""
    u1, u2, u3 = cubic_roots(M, b)
    # factors (t - u1), (u2 - t), (u3 - t)
    if not x > y:
        return 0.0
    X = (math.sqrt(x - u1), math.sqrt(max(0.0, u2 - x)), math.sqrt(u3 - x))
    Y = (math.sqrt(y - u1), math.sqrt(u2 - y), math.sqrt(u3 - y))
    d = x - y
    U12 = (X[0] * X[1] * Y[2] + Y[0] * Y[1] * X[2]) / d
    U13 = (X[0] * X[2] * Y[1] + Y[0] * Y[2] * X[1]) / d
    U23 = (X[1] * X[2] * Y[0] + Y[1] * Y[2] * X[0]) / d
    return 2.0 * float(elliprf(U12 * U12, U13 * U13, U23 * U23)) / math.sqrt(2.0 * M)


def leg_angle_quad(M: float, b: float, y: float, x: float) -> float:
    """Same integral by adaptive quadrature after u = u2 - s^2 (removes the
    inverse square-root singularity at the turning point)."""
    u1, u2, u3 = cubic_roots(M, b)

    def f(s):
        u = u2 - s * s
        return 2.0 / math.sqrt(2.0 * M * (u - u1) * (u3 - u))

    s_lo, s_hi = math.sqrt(max(0.0, u2 - x)), math.sqrt(u2 - y)
    val, _ = integrate.quad(f, s_lo, s_hi, epsabs=1e-15, epsrel=1e-14, limit=200)
    return val


def phi_inf(M: float, b: float, u0: float) -> float:
    """Total azimuth swept by an ingoing ray from u0 to escape (u = 0)."""
    if M == 0.0:
        return math.pi - math.asin(min(1.0, b * u0))
    u2 = cubic_roots(M, b)[1]
    return leg_angle(M, b, u0, u2) + leg_angle(M, b, 0.0, u2)


def phi_at_u(M: float, b: float, u0: float, u: float, outgoing: bool) -> float:
    """Azimuth where an ingoing ray from u0 reaches u, before (outgoing=False)
    or after (outgoing=True) its periastron."""
    u2 = cubic_roots(M, b)[1]
    if not outgoing:
        return leg_angle(M, b, u0, u)
    return leg_angle(M, b, u0, u2) + leg_angle(M, b, u, u2)


def weak_field_deflection(M: float, b: float) -> float:
    """First two terms of the infinity-to-infinity deflection series
    4M/b + 15 pi M^2 / (4 b^2); the next term is 128 M^3 / (3 b^3)."""
    return 4.0 * M / b + 15.0 * math.pi * M * M / (4.0 * b * b)


def static_b(M: float, r: float, sin_alpha: float) -> float:
    """Impact parameter of a ray leaving a static observer at radius r at
    angle alpha from the outward radial direction."""
    return r * sin_alpha / math.sqrt(1.0 - 2.0 * M / r)


def shadow_angle(M: float, r: float) -> float:
    """Angular radius of the captured region seen by a static observer."""
    return math.asin(B_CRIT * M * math.sqrt(1.0 - 2.0 * M / r) / r)


def einstein_ring_angle(M: float, r: float) -> float:
    """Off-axis angle psi (static observer) whose ray leaves exactly behind
    the hole: phi_inf = pi, with alpha = pi - psi."""
    u0 = 1.0 / r

    def g(psi):
        b = static_b(M, r, math.sin(psi))
        return phi_inf(M, b, u0) - math.pi

    lo = shadow_angle(M, r) * (1 + 1e-9) + 1e-9
    return optimize.brentq(g, lo, 1.2, xtol=1e-15, rtol=1e-15, maxiter=500)
