"""Full-size renders (config 2 at 1024^2, config 3 at 4096^2 in every form,
config 4 through the surrogate) in the launch configuration bench.py times
-- bh_render on a side stream with the workload's tolerances and the
default launch shape -- checked against the oracle on seeded pixel samples
plus the full middle row, which crosses the shadow edge and the photon-
sphere band."""
import os

import numpy as np
import pytest

import oracle
import parity
import paper_2507_16165_gb300 as bh
from gpu_util import to_numpy
from paper_2507_16165_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WEIGHTS = os.path.join(os.path.dirname(bh.__file__), "data", "surrogate_m1.bin")

FULL = {
    "c2_fp64_1024": (W.config2(1024, "fp64"), "fp64"),
    "c2_fp32_1024": (W.config2(1024, "fp32"), "fp32"),
    "c3_fp64_4096": (W.config3(4096, "fp64"), "fp64"),
    "c3_fp32_4096": (W.config3(4096, "fp32"), "fp32"),
    "c3_mixed_4096": (W.config3(4096, "mixed"), "mixed"),
    "c4_surrogate_4096": (W.config4(4096), "surrogate"),
}


@pytest.mark.parametrize("name", sorted(FULL))
def test_full_size_sampled_parity(name):
    import torch
    w, mode = FULL[name]
    cam = w.cameras[0]
    n = w.n_rays
    sc = bh.Scene(w.scene)
    try:
        if mode == "surrogate":
            bh.bh_surrogate_load(sc.handle, WEIGHTS)
        stream = torch.cuda.Stream()
        opts = bh.render_opts(mode, stream, rtol=w.rtol, atol=w.atol, band=w.band)
        f64 = mode == "fp64"
        dirs = torch.empty(2 * n, dtype=torch.float64 if f64 else torch.float32, device="cuda")
        flags = torch.empty(n, dtype=torch.int16, device="cuda")
        rgba = torch.empty(n, dtype=torch.int32, device="cuda")
        cams = sc.cameras(w.cameras)
        bh.bh_render(sc.handle, cams, [cam.w], [cam.h], dirs, flags, rgba, opts)
        stream.synchronize()
        st = sc.stats()
        assert st["status"] == 0 and st["rays"] == n
        rng = np.random.default_rng(2024)
        idx = np.unique(np.concatenate([rng.choice(n, 20000, replace=False),
                                        (cam.h // 2) * cam.w + np.arange(cam.w)]))
        full = to_numpy({"theta": dirs[:n], "phi": dirs[n:], "flags": flags, "rgba": rgba})
        got = {k: v[idx] for k, v in full.items()}
        ref = oracle.render_pixels(w.scene, w.cameras, np.zeros(len(idx), np.int32),
                                   idx % cam.w, idx // cam.w, parity.oracle_opts(mode),
                                   nthreads=8)
        m = parity.compare(got, ref, mode)
        parity.assert_parity(m, mode)
        if mode == "mixed":
            assert st["n_band"] > 0 and np.any(got["flags"] & bh.BH_FLAG_BAND)
        if mode == "surrogate":
            assert st["n_surrogate"] > 0.3 * n
    finally:
        sc.close()
