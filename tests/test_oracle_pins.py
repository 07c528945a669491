"""The CPU oracle against facts the physics fixes (see oracle_pins.py)."""
import pytest

import oracle
import oracle_pins as P


@pytest.fixture(scope="module")
def lib():
    return oracle.load()


@pytest.mark.parametrize("check", P.ALL, ids=[f.__name__ for f in P.ALL])
def test_pin(lib, check):
    ok, detail = check(lib)
    assert ok, detail


def test_carlson_reduction_matches_quadrature():
    """The R_F reduction used by the closed forms agrees with adaptive
    quadrature of the same integral (guards the pin itself)."""
    import closed_forms as cf
    for b in (5.2, 5.3, 6.0, 10.0, 50.0, 1000.0):
        u2 = cf.cubic_roots(1.0, b)[1]
        for y in (0.0, 1 / 30):
            if y < u2:
                assert abs(cf.leg_angle(1.0, b, y, u2) - cf.leg_angle_quad(1.0, b, y, u2)) < 1e-12


def test_periastron_root_at_critical():
    """b = 3 sqrt(3) M puts the double root of the cubic at u = 1/(3M)."""
    import numpy as np
    import closed_forms as cf
    r = np.roots([2.0, -1.0, 0.0, 1.0 / cf.B_CRIT ** 2])
    assert np.min(np.abs(r - 1.0 / 3.0)) < 1e-7


def test_render_pixels_matches_render(lib):
    """The pixel-list entry point returns exactly what the full render does."""
    import numpy as np
    from paper_2507_16165_gb300 import workloads as W
    w = W.config3(48)
    full = oracle.render(w.scene, w.cameras, lib=lib)
    rng = np.random.default_rng(0)
    idx = rng.choice(48 * 48, 200, replace=False)
    sub = oracle.render_pixels(w.scene, w.cameras, np.zeros(200, np.int32), idx % 48, idx // 48,
                               lib=lib)
    for k in ("flags", "rgba", "steps"):
        assert np.array_equal(sub[k], full[k][idx])
    assert np.array_equal(sub["theta"], full["theta"][idx], equal_nan=True)


def test_openmp_matches_serial(lib):
    """Threaded rendering (dynamic scanline schedule) gives identical bits."""
    import numpy as np
    from paper_2507_16165_gb300 import workloads as W
    w = W.config2(40)
    a = oracle.render(w.scene, w.cameras, nthreads=1, lib=lib)
    b = oracle.render(w.scene, w.cameras, nthreads=4, lib=lib)
    for k in ("flags", "rgba", "steps"):
        assert np.array_equal(a[k], b[k])
