"""Keplerian disk shading (Doppler and gravitational shift) on the GPU
against the oracle, which computes the shift by another route (local static
frame and special-relativistic Doppler factor; see oracle_pins.DOPPLER)."""
from dataclasses import replace

import numpy as np
import pytest

import oracle
import parity
import paper_2507_16165_gb300 as bh
from gpu_util import render
from paper_2507_16165_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [("fp64", W.config2(96, "fp64")), ("fp32", W.config2(128, "fp32")),
         ("mixed", W.config3(128, "mixed")),
         ("fp32", replace(W.config2(96, "fp32"),
                          cameras=(replace(W.config2(96).cameras[0], incl_deg=89.0),)))]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_doppler_matches_oracle(case):
    mode, w = CASES[case]
    er, ea, eb = parity.AMBIG[mode]
    ref = oracle.render(w.scene, w.cameras, oracle.opts(eps_r=er, eps_ang=ea, eps_b=eb, doppler=1),
                        nthreads=8)
    rtol, atol = (1e-10, 1e-10) if mode == "fp64" else (1e-5, 1e-7)
    got, st = render(w.scene, w.cameras, mode, rtol=rtol, atol=atol, band=w.band, doppler=1)
    m = parity.compare(got, ref, mode)
    parity.assert_parity(m, mode)
    # the shading changed where the disk is seen
    plain = oracle.render(w.scene, w.cameras, oracle.opts(), nthreads=8)
    disk = (ref["flags"] & 0xFF) == oracle.DISK
    assert disk.sum() > 100
    assert np.mean(plain["rgba"][disk] != ref["rgba"][disk]) > 0.5


def test_doppler_refused_outside_integrator_modes():
    w = W.config2(8, "fp32")
    sc = bh.Scene(w.scene)
    try:
        with pytest.raises(bh.BHError) as e:
            sc.render(w.cameras, "paper", doppler=1)
        assert e.value.code == -7
    finally:
        sc.close()
