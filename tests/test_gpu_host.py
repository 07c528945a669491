"""bh_render_host: the frame rendered in strips of whole tile rows, each
strip's outputs copied to host buffers while the next strip renders.  Every
ray is computed as in one whole render, so the host outputs must equal
bh_render's device outputs bit for bit: one camera and a batch of cameras
of uneven size, every integrator form, strip counts that do not divide the
tile rows evenly, and a strip count of one."""
import numpy as np
import pytest

import paper_2507_16165_gb300 as bh
from paper_2507_16165_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WEIGHTS = __import__("os").path.join(__import__("os").path.dirname(bh.__file__), "data",
                                     "surrogate_m1.bin")


def _both(w, mode, strips, **kw):
    import torch
    n = w.n_rays
    f64 = mode in ("fp64", "paper")
    sc = bh.Scene(w.scene)
    try:
        if mode == "surrogate":
            bh.bh_surrogate_load(sc.handle, WEIGHTS)
        cams = sc.cameras(w.cameras)
        wv = [c.w for c in w.cameras]
        hv = [c.h for c in w.cameras]
        o = dict(rtol=w.rtol, atol=w.atol, band=w.band, **kw)
        dt = torch.float64 if f64 else torch.float32
        dd = torch.empty(2 * n, dtype=dt, device="cuda")
        df = torch.empty(n, dtype=torch.int16, device="cuda")
        dr = torch.empty(n, dtype=torch.int32, device="cuda")
        bh.bh_render(sc.handle, cams, wv, hv, dd, df, dr, bh.render_opts(mode, **o))
        torch.cuda.synchronize()
        ref_rays = sc.stats()["rays"]
        hd = torch.full((2 * n,), -7.0, dtype=dt).pin_memory()
        hf = torch.full((n,), -7, dtype=torch.int16).pin_memory()
        hr = torch.full((n,), -7, dtype=torch.int32).pin_memory()
        bh.bh_render_host(sc.handle, cams, wv, hv, hd, hf, hr,
                          bh.render_opts(mode, host_strips=strips, **o))
        st = sc.stats()
        return (dd.cpu().numpy(), df.cpu().numpy(), dr.cpu().numpy()), \
               (hd.numpy(), hf.numpy(), hr.numpy()), ref_rays, st
    finally:
        sc.close()


def _same(dev, host):
    for a, b in zip(dev, host):
        ia = a.view(np.uint64 if a.dtype == np.float64 else np.uint32) if a.dtype.kind == "f" else a
        ib = b.view(np.uint64 if b.dtype == np.float64 else np.uint32) if b.dtype.kind == "f" else b
        assert np.array_equal(ia, ib)


@pytest.mark.parametrize("mode,strips", [("fp32", 5), ("fp32", 1), ("mixed", 3), ("mixed", 0),
                                         ("fp64", 2), ("paper_fp32", 4), ("surrogate", 3)])
def test_host_render_equals_device_render(mode, strips):
    w = W.config3(300, "fp64" if mode == "fp64" else "mixed")
    dev, host, rays, st = _both(w, mode, strips)
    _same(dev, host)
    assert st["rays"] == rays == w.n_rays
    assert st["status"] == 0


def test_host_render_of_a_camera_batch_in_strips():
    # 16 cameras of uneven size (scaled-down orbit sequence): strips cut inside
    # cameras and across camera boundaries
    w = W.config5(16, scale=8)
    dev, host, rays, st = _both(w, "fp32", 7)
    _same(dev, host)
    assert st["rays"] == rays == w.n_rays


def test_host_strip_count_is_checked():
    w = W.config3(64, "mixed")
    sc = bh.Scene(w.scene)
    try:
        cams = sc.cameras(w.cameras)
        n = w.n_rays
        import torch
        with pytest.raises(bh.BHError):
            bh.bh_render_host(sc.handle, cams, [64], [64], torch.empty(2 * n), None, None,
                              bh.render_opts("fp32", host_strips=bh.BH_MAX_HOST_STRIPS + 1))
    finally:
        sc.close()
