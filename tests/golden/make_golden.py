"""Writes the oracle regression fixtures in this directory.

The paper prints no worked example (no pixel values, trajectories or
tables), so the fixtures here are written by this script from the CPU oracle
alone.  They are regression guards for the oracle, not independent pins; the
independent pins live in tests/oracle_pins.py.

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2507_16165_gb300 import workloads as W  # noqa: E402


def c1_small(size=16):
    """Config-1 scene and camera (M = 1, r_obs = 30M, 60 deg, no disk,
    sky seed 0, rtol = atol = 1e-10) at 16 x 16 pixels."""
    w = W.config1(size)
    return w.scene, w.cameras


def c3_small(size=16):
    """Config-3 scene (disk [6M, 30M], 8 seeded spheres, r_obs = 50M, 75 deg)
    at 16 x 16 pixels, FP64 tolerance 1e-10."""
    w = W.config3(size, "fp64")
    return w.scene, w.cameras


FIXTURES = {"oracle_c1_16.txt": c1_small, "oracle_c3_16.txt": c3_small}


def write(name, maker):
    scene, cams = maker()
    out = oracle.render(scene, cams, oracle.opts())
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# {maker.__doc__.strip().splitlines()[0]}\n")
        f.write("# written by tests/golden/make_golden.py from the CPU oracle\n")
        f.write("# index flags rgba ambig theta phi\n")
        for i in range(len(out["flags"])):
            f.write(f"{i} {int(out['flags'][i])} {int(out['rgba'][i])} {int(out['ambig'][i])} "
                    f"{out['theta'][i]:.15e} {out['phi'][i]:.15e}\n")


if __name__ == "__main__":
    for n, m in FIXTURES.items():
        write(n, m)
