"""The oracle still reproduces its own committed regression fixtures."""
import os

import numpy as np
import pytest

import oracle
from golden.make_golden import FIXTURES

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("name", sorted(FIXTURES))
def test_golden(name):
    rows = np.loadtxt(os.path.join(HERE, name), comments="#")
    scene, cams = FIXTURES[name]()
    out = oracle.render(scene, cams, oracle.opts())
    assert len(rows) == len(out["flags"])
    assert np.array_equal(rows[:, 1].astype(np.uint16), out["flags"])
    clean = rows[:, 3] == 0
    assert np.array_equal(rows[clean, 2].astype(np.uint32), out["rgba"][clean])
    for col, key in ((4, "theta"), (5, "phi")):
        a, b = rows[:, col], out[key]
        both = ~np.isnan(a)
        assert np.array_equal(np.isnan(a), np.isnan(b))
        d = np.abs(a[both] - b[both])
        d = np.minimum(d, 2 * np.pi - d)
        assert d.max(initial=0.0) < 1e-11
