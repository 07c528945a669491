"""Anti-aliased renders (n x n stratified samples per pixel, box filter)
on the GPU against the oracle's same pixels: colours within the RGBA bar,
the centre ray's direction and flags as for one sample, and the expected
ray count."""
import numpy as np
import pytest

import oracle
import parity
import paper_2507_16165_gb300 as bh
from gpu_util import render
from paper_2507_16165_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", ["fp32", "fp64"])
@pytest.mark.parametrize("spp", [4, 9])
def test_spp_matches_oracle(mode, spp):
    n = int(round(spp ** 0.5))
    w = W.config3(48, mode) if mode == "fp64" else W.config2(96, "fp32")
    er, ea, eb = parity.AMBIG[mode]
    o = oracle.opts(eps_r=er, eps_ang=ea, eps_b=eb, spp_n=n)
    ref = oracle.render(w.scene, w.cameras, o, nthreads=8)
    rtol, atol = (1e-10, 1e-10) if mode == "fp64" else (1e-5, 1e-7)
    got, st = render(w.scene, w.cameras, mode, rtol=rtol, atol=atol, spp=spp)
    assert st["status"] == 0
    assert st["rays"] == w.n_rays * (spp + 1)
    m = parity.compare(got, ref, mode)
    # a pixel is ambiguous when any of its spp + 1 rays is
    parity.assert_parity(m, mode, rays_per_pixel=spp + 1)


def test_spp_rejected_where_unsupported():
    w = W.config2(8, "fp32")
    sc = bh.Scene(w.scene)
    try:
        with pytest.raises(bh.BHError) as e:
            sc.render(w.cameras, "mixed", spp=4)
        assert e.value.code == -7
        with pytest.raises(bh.BHError) as e:
            sc.render(w.cameras, "fp32", spp=5)
        assert e.value.code == -1
    finally:
        sc.close()
