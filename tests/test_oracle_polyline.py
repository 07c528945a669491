"""Pins of the oracle's second method: the paper's fixed-step polyline
(Sec. 2.1-2.2; classical Runge-Kutta at a fixed step eps, straight segments,
segment intersection).  Each check is fixed by the mathematics, not by the
method's own output:
  - at M = 0 the exact orbit is a straight line, the Runge-Kutta points lie
    on it to O(eps^4) and so do the segments: escape directions equal the
    camera directions, disk hits the ray-plane intersection;
  - with M > 0 a segment crosses the disk plane on the line of nodes, so a
    disk hit's direction is the exact node direction, the same as the
    adaptive method's to rounding;
  - the escape angle comes from the linear interpolant of u through the
    last two points, where u'' = 3Mu^2 - u vanishes with u, so its error
    falls at third order in eps (a first- or second-order stepper, or an
    interpolation at the wrong end, would not);
  - flags agree with the adaptive method outside the ambiguity mask."""
import numpy as np
import pytest

import oracle
import oracle_pins as P
from paper_2507_16165_gb300 import workloads as W


@pytest.mark.parametrize("pin", P.POLYLINE, ids=[p.__name__ for p in P.POLYLINE])
def test_polyline_pin(pin):
    ok, detail = pin(oracle.load())
    assert ok, detail


def test_flags_agree_with_the_adaptive_method():
    w = W.config3(40, "fp64")
    amb = oracle.opts(eps_r=1e-3, eps_ang=1e-5, eps_b=1e-3)
    ref = oracle.render(w.scene, w.cameras, amb, nthreads=4)
    o = oracle.opts(eps=0.01, eps_r=1e-3, eps_ang=1e-5, eps_b=1e-3, method=oracle.METHOD_POLYLINE)
    got = oracle.render(w.scene, w.cameras, o, nthreads=4)
    clean = (ref["ambig"] == 0) & (got["ambig"] == 0)
    assert clean.sum() > 0.9 * len(clean)
    assert np.array_equal(got["flags"][clean] & 0x8F, ref["flags"][clean] & 0x8F)
