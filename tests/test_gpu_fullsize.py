"""Full-size renders (config 2 at 1024^2, config 3 at 4096^2 in every form,
config 4 through the surrogate) in the launch configuration bench.py times
-- bh_render on a side stream with the workload's tolerances and the
default launch shape -- checked against the oracle on a stratified pixel
sample: seeded random pixels of the whole frame, its full middle row (which
crosses the shadow edge and the photon-sphere band), every pixel within
2e-3 M of the critical impact parameter and a sample of the rest of the
|b - b_c| < 2M ring, where the exit directions are most sensitive.  Each
stratum's pixels are weighted by the share of the frame they stand for, so
the 99.9th-percentile and RGBA bars are those of the whole frame, with no
pixel left out; flags are bit-exact on every sampled pixel outside the
oracle's ambiguity mask."""
import os
from dataclasses import replace

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
    "c2_fp64_1024": (W.config2(1024, "fp64"), "fp64", {}),
    "c2_fp32_1024": (W.config2(1024, "fp32"), "fp32", {}),
    "c3_fp64_4096": (W.config3(4096, "fp64"), "fp64", {}),
    "c3_fp32_4096": (W.config3(4096, "fp32"), "fp32", {}),
    "c3_mixed_4096": (W.config3(4096, "mixed"), "mixed", {}),
    # the mixed form with the FP64 turning-point solve for every ray
    "c3_mixed_literal_4096": (W.config3(4096, "mixed"), "mixed", {"periastron_reset": 2}),
    # twice the FP64 band: more band rays than two band warps per SM take at
    # about 1.7 a lane, so the band pass keeps more of its warps
    "c3_mixed_wide_band_4096": (replace(W.config3(4096, "mixed"), band=0.1), "mixed", {}),
    "c4_surrogate_4096": (W.config4(4096), "surrogate", {}),
}

# strata: (lo, hi) of |b - b_c| in M and the largest sample drawn from each
STRATA = [((0.0, 2e-3), 4000), ((2e-3, 0.05), 1500), ((0.05, 2.0), 1500)]


def stratified_sample(cam, n_random, seed=2024):
    """(pixel indices, weights): a uniform sample of the frame plus its middle
    row (weight: frame pixels per sampled pixel) and the near-critical strata
    (weight: stratum pixels per sampled pixel), uniform pixels falling in a
    stratum counted with that stratum."""
    n = cam.w * cam.h
    rng = np.random.default_rng(seed)
    strata = []
    taken = np.zeros(n, bool)
    for (lo, hi), k in STRATA:
        pix = parity.band_pixels(cam, lo, hi)
        pick = pix if len(pix) <= k else rng.choice(pix, k, replace=False)
        strata.append((pix, pick))
        taken[pix] = True
    rest = np.flatnonzero(~taken)
    uni = np.unique(np.concatenate([rng.choice(rest, n_random, replace=False),
                                    (cam.h // 2) * cam.w + np.arange(cam.w)]))
    uni = uni[~taken[uni]]
    idx = [uni]
    wts = [np.full(len(uni), len(rest) / len(uni))]
    for pix, pick in strata:
        if len(pick):
            idx.append(pick)
            wts.append(np.full(len(pick), len(pix) / len(pick)))
    return np.concatenate(idx), np.concatenate(wts)


@pytest.mark.parametrize("name", sorted(FULL))
def test_full_size_sampled_parity(name):
    import torch
    w, mode, extra = FULL[name]
    cam = w.cameras[0]
    n = w.n_rays
    sc = bh.Scene(w.scene)
    try:
        if mode == "surrogate":
            bh.bh_surrogate_load(sc.handle, WEIGHTS)
        stream = torch.cuda.Stream()
        opts = bh.render_opts(mode, stream, rtol=w.rtol, atol=w.atol, band=w.band, **extra)
        f64 = mode == "fp64"
        dirs = torch.empty(2 * n, dtype=torch.float64 if f64 else torch.float32, device="cuda")
        flags = torch.empty(n, dtype=torch.int16, device="cuda")
        rgba = torch.empty(n, dtype=torch.int32, device="cuda")
        cams = sc.cameras(w.cameras)
        bh.bh_render(sc.handle, cams, [cam.w], [cam.h], dirs, flags, rgba, opts)
        stream.synchronize()
        st = sc.stats()
        assert st["status"] == 0 and st["rays"] == n
        idx, wt = stratified_sample(cam, 8000 if f64 else 20000)
        full = to_numpy({"theta": dirs[:n], "phi": dirs[n:], "flags": flags, "rgba": rgba})
        got = {k: v[idx] for k, v in full.items()}
        ref = oracle.render_pixels(w.scene, w.cameras, np.zeros(len(idx), np.int32),
                                   idx % cam.w, idx // cam.w, parity.oracle_opts(mode),
                                   nthreads=16)
        m = parity.compare(got, ref, mode, weight=wt)
        parity.assert_parity(m, mode)
        if mode == "mixed":
            assert st["n_band"] > 0 and np.any(got["flags"] & bh.BH_FLAG_BAND)
        if name == "c3_mixed_wide_band_4096":
            sms = torch.cuda.get_device_properties(0).multi_processor_count
            assert st["n_band"] > 2 * sms * 32 * 1.7, st["n_band"]
        if mode == "surrogate":
            assert st["n_surrogate"] > 0.3 * n
    finally:
        sc.close()
