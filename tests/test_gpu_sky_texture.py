"""Image sky (equirectangular RGBA8, bilinear) on the GPU against the
oracle's lookup of the same image, plus the upload entry point."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import parity
import paper_2507_16165_gb300 as bh
from gpu_util import render
from paper_2507_16165_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TEX = W.sky_texture(seed=5, w=512, h=256)


@pytest.mark.parametrize("mode", ["fp64", "fp32", "mixed"])
def test_sky_texture_matches_oracle(mode):
    w = W.config2(96, mode if mode != "mixed" else "fp32")
    w = replace(w, scene=replace(w.scene, sky_texture=TEX))
    er, ea, eb = parity.AMBIG[mode]
    ref = oracle.render(w.scene, w.cameras, oracle.opts(eps_r=er, eps_ang=ea, eps_b=eb), nthreads=8)
    rtol, atol = (1e-10, 1e-10) if mode == "fp64" else (1e-5, 1e-7)
    got, st = render(w.scene, w.cameras, mode, rtol=rtol, atol=atol)
    m = parity.compare(got, ref, mode)
    parity.assert_parity(m, mode)
    esc = (ref["flags"] & 0xFF) == oracle.ESC
    checker = oracle.render(replace(w.scene, sky_texture=None), w.cameras, oracle.opts(), nthreads=8)
    assert np.mean(checker["rgba"][esc] != ref["rgba"][esc]) > 0.9   # the image is what shows


def test_sky_texture_upload_and_reset():
    import torch
    w = W.config1(16)
    sc = bh.Scene(w.scene)
    try:
        a = sc.render(w.cameras, "fp32")["rgba"].clone()
        bh.bh_scene_sky_texture(sc.handle, TEX)
        b = sc.render(w.cameras, "fp32")["rgba"].clone()
        bh.bh_scene_sky_texture(sc.handle, None)
        c = sc.render(w.cameras, "fp32")["rgba"].clone()
        torch.cuda.synchronize()
        assert not torch.equal(a, b) and torch.equal(a, c)
        with pytest.raises(bh.BHError):
            bh.bh_scene_sky_texture(sc.handle, np.zeros((0, 4), np.uint32))
    finally:
        sc.close()
