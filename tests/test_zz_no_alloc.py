"""bh_render_noalloc: rendering without any device allocation.

Callers that cannot call cudaMalloc -- a host that hands all device memory to
its own pool or a fixed budget, or a real-time loop where an allocation could
synchronise the device or fail in mid-frame -- use bh_render_noalloc.  It
keeps its only scratch (queue counter, status and statistics words, camera
table) in one fixed library-owned device array and finishes every ray with
the kernels bh_render uses, so its outputs must equal those of the
allocating bh_render bit for bit, and a call must leave the device's free
memory unchanged.  This file is collected last so that a
`-x` run has already run every other test if it fails here.
"""
import ctypes

import numpy as np
import pytest

import parity
import paper_2507_16165_gb300 as bh
from paper_2507_16165_gb300 import _capi
from paper_2507_16165_gb300 import workloads as W


def _outputs(torch, n, f64):
    dt = torch.float64 if f64 else torch.float32
    return (torch.full((2 * n,), float("nan"), dtype=dt, device="cuda"),
            torch.zeros(n, dtype=torch.int16, device="cuda"),
            torch.zeros(n, dtype=torch.int32, device="cuda"))


def _numpy(dirs, flags, rgba, n):
    d = dirs.double().cpu().numpy()
    return {"theta": d[:n], "phi": d[n:], "flags": flags.cpu().numpy().astype(np.uint16),
            "rgba": rgba.cpu().numpy().astype(np.uint32)}


def _same(a, b):
    """Bit-identical outputs: the same rays through the same kernels."""
    assert np.array_equal(a["flags"], b["flags"])
    assert np.array_equal(a["rgba"], b["rgba"])
    nan = np.isnan(b["theta"])
    assert np.array_equal(np.isnan(a["theta"]), nan)
    assert np.array_equal(a["theta"][~nan], b["theta"][~nan])
    assert np.array_equal(a["phi"][~nan], b["phi"][~nan])


CASES = [(W.config1(64), "fp64"), (W.config2(256, "fp32"), "fp32"),
         (W.config5(6, scale=16), "fp32")]


@pytest.mark.gpu
@pytest.mark.parametrize("case", range(len(CASES)))
def test_noalloc_matches_bh_render_twice(case):
    """Two bh_render_noalloc calls in a row each reproduce bh_render."""
    import torch
    w, mode = CASES[case]
    f64 = mode == "fp64"
    n = w.n_rays
    sc = bh.Scene(w.scene)
    cams = sc.cameras(w.cameras)
    wv, hv = [c.w for c in w.cameras], [c.h for c in w.cameras]
    opts = bh.render_opts(mode, rtol=w.rtol, atol=w.atol)
    ref_bufs = _outputs(torch, n, f64)
    bh.bh_render(sc.handle, cams, wv, hv, *ref_bufs, opts)
    torch.cuda.synchronize()
    ref = _numpy(*ref_bufs, n)
    sc.close()
    desc = bh.scene_desc(w.scene)
    for call in range(2):
        bufs = _outputs(torch, n, f64)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        bh.bh_render_noalloc(desc, cams, wv, hv, *bufs, opts)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        if call == 1:
            # the call allocates no device memory (the first call on the
            # device may still load the library's module)
            assert free_after == free_before
        _same(_numpy(*bufs, n), ref)


def test_noalloc_rejects_out_of_range_requests():
    """Too many cameras for the fixed scratch, or a mode the coherent pass
    alone cannot serve, are refused before any device work."""
    lib = _capi.lib()
    desc = bh.scene_desc(W.config2(8).scene)
    n = _capi.BH_NOALLOC_MAX_CAMERAS + 1
    cams = (_capi.bh_camera * n)()
    for c in cams:
        lib.bh_camera_set(ctypes.byref(c), 40.0, 80.0, 0.0, 60.0)
    wv = (ctypes.c_int * n)(*([8] * n))
    o = bh.render_opts("fp32", stream=0)
    rc = lib.bh_render_noalloc(ctypes.byref(desc), cams, n, wv, wv, None, None, None,
                               ctypes.byref(o))
    assert rc == _capi.BH_E_INVALID
    assert "64" in bh.bh_last_error()
    o = bh.render_opts("mixed", stream=0)
    rc = lib.bh_render_noalloc(ctypes.byref(desc), cams, 1, wv, wv, None, None, None,
                               ctypes.byref(o))
    assert rc == _capi.BH_E_UNSUPPORTED
    # the host-side abort word needs a status read-back this entry point lacks
    o = bh.render_opts("fp32", stream=0, abort_after=64)
    rc = lib.bh_render_noalloc(ctypes.byref(desc), cams, 1, wv, wv, None, None, None,
                               ctypes.byref(o))
    assert rc == _capi.BH_E_UNSUPPORTED
