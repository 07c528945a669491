"""Batched multi-camera rendering: CUDA-graph replay (integrator modes and the
surrogate), launch shapes (tile, queue chunk, block) and the autotuner."""
import os

import numpy as np
import pytest

import oracle
import parity
import paper_2507_16165_gb300 as bh
from gpu_util import to_numpy
from paper_2507_16165_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _buffers(torch, n, f64=False):
    return (torch.empty(2 * n, dtype=torch.float64 if f64 else torch.float32, device="cuda"),
            torch.empty(n, dtype=torch.int16, device="cuda"),
            torch.empty(n, dtype=torch.int32, device="cuda"))


def _np(bufs, n):
    d, f, r = bufs
    return to_numpy({"theta": d[:n], "phi": d[n:], "flags": f, "rgba": r})


WEIGHTS = os.path.join(os.path.dirname(bh.__file__), "data", "surrogate_m1.bin")


def _same(a, b):
    assert np.array_equal(a["flags"], b["flags"])
    assert np.array_equal(a["rgba"], b["rgba"])
    assert np.array_equal(a["theta"], b["theta"], equal_nan=True)
    assert np.array_equal(a["phi"], b["phi"], equal_nan=True)


@pytest.mark.parametrize("mode", ["fp32", "mixed", "surrogate"])
def test_graph_replay_equals_render(mode):
    import torch
    w = W.config5(8, scale=8)
    n = w.n_rays
    sc = bh.Scene(w.scene)
    try:
        if mode == "surrogate":
            bh.bh_surrogate_load(sc.handle, WEIGHTS)
        cams = sc.cameras(w.cameras)
        wv, hv = [c.w for c in w.cameras], [c.h for c in w.cameras]
        opts = bh.render_opts(mode, rtol=w.rtol, atol=w.atol)
        ref = _buffers(torch, n)
        bh.bh_render(sc.handle, cams, wv, hv, *ref, opts)
        torch.cuda.synchronize()
        ref_np = _np(ref, n)
        out = _buffers(torch, n)
        g = bh.bh_graph_create(sc.handle, cams, wv, hv, *out, opts)
        try:
            for _ in range(3):
                out[1].zero_()
                bh.bh_graph_launch(g)
                torch.cuda.synchronize()
                got = _np(out, n)
                assert np.array_equal(got["flags"], ref_np["flags"])
                assert np.array_equal(got["rgba"], ref_np["rgba"])
                assert np.array_equal(got["theta"], ref_np["theta"], equal_nan=True)
            st = sc.stats()
            assert st["rays"] == n and st["status"] == 0
            if mode == "surrogate":
                assert st["n_surrogate"] > 0 and st["kernel_ms"][3] > 0
        finally:
            bh.bh_graph_destroy(g)
    finally:
        sc.close()


@pytest.mark.parametrize("mode", ["fp32", "mixed", "fp64", "surrogate"])
def test_launch_shape_changes_schedule_not_result(mode):
    """Every tile shape, queue chunk and block size gives the same rays
    bit for bit: a ray's arithmetic does not depend on its neighbours."""
    import torch
    w = W.config5(6, scale=16)
    n = w.n_rays
    f64 = mode == "fp64"
    sc = bh.Scene(w.scene)
    try:
        if mode == "surrogate":
            bh.bh_surrogate_load(sc.handle, WEIGHTS)
        cams = sc.cameras(w.cameras)
        wv, hv = [c.w for c in w.cameras], [c.h for c in w.cameras]
        tol = dict(rtol=1e-10, atol=1e-10) if f64 else dict(rtol=w.rtol, atol=w.atol)
        ref = _buffers(torch, n, f64)
        bh.bh_render(sc.handle, cams, wv, hv, *ref, bh.render_opts(mode, **tol))
        torch.cuda.synchronize()
        ref_np = _np(ref, n)
        for tw, th, chunk, block, budget in [(4, 8, 64, 128, 0), (8, 8, 1024, 512, 0),
                                             (16, 16, 256, 256, 24), (32, 2, 32, 512, 0),
                                             (1, 32, 96, 64, 0)]:
            out = _buffers(torch, n, f64)
            o = bh.render_opts(mode, tile_w=tw, tile_h=th, queue_chunk=chunk, block_size=block,
                               budget=budget, **tol)
            bh.bh_render(sc.handle, cams, wv, hv, *out, o)
            torch.cuda.synchronize()
            st = sc.stats()
            assert st["rays"] == n and st["status"] == 0
            _same(_np(out, n), ref_np)
    finally:
        sc.close()


def test_launch_shape_rejects_bad_values():
    import ctypes

    from paper_2507_16165_gb300 import _capi
    w = W.config2(8)
    sc = bh.Scene(w.scene)
    try:
        cams = sc.cameras(w.cameras)
        for kw in [dict(tile_w=8, tile_h=2), dict(tile_w=3, tile_h=32), dict(tile_w=32, tile_h=16),
                   dict(queue_chunk=48), dict(queue_chunk=2048), dict(block_size=1024)]:
            o = bh.render_opts("fp32", **kw)
            W1 = (ctypes.c_int * 1)(8)
            rc = _capi.lib().bh_render(sc.handle, bh._cams_array(cams), 1, W1, W1, None, None,
                                       None, ctypes.byref(o))
            assert rc == _capi.BH_E_INVALID, kw
        # a camera that does not look at the hole is refused, not rendered
        bad = (_capi.bh_camera * 1)()
        ctypes.memmove(ctypes.byref(bad[0]), ctypes.byref(cams[0]), ctypes.sizeof(_capi.bh_camera))
        bad[0].fwd[0] += 1e-3
        o = bh.render_opts("fp32")
        W1 = (ctypes.c_int * 1)(8)
        rc = _capi.lib().bh_render(sc.handle, bad, 1, W1, W1, None, None, None, ctypes.byref(o))
        assert rc == _capi.BH_E_INVALID and "look at the hole" in bh.bh_last_error()
    finally:
        sc.close()


def test_autotune_picks_a_shape_used_by_later_renders():
    import torch
    w = W.config3(512, "fp32")
    n = w.n_rays
    sc = bh.Scene(w.scene)
    try:
        cams = sc.cameras(w.cameras)
        opts = bh.render_opts("fp32", rtol=w.rtol, atol=w.atol)
        bufs = _buffers(torch, n)
        bh.bh_render(sc.handle, cams, [512], [512], *bufs, opts)
        torch.cuda.synchronize()
        before = _np(bufs, n)
        res = bh.bh_autotune(sc.handle, cams, [512], [512], *bufs, opts)
        assert res["trials"] > 10
        assert res["ms_best"] <= res["ms_default"]
        assert (res["tile_w"], res["tile_h"]) in ((8, 4), (4, 8), (8, 8), (16, 16))
        assert res["block_size"] in (128, 256, 512)
        assert res["queue_chunk"] in (32, 64, 128, 256, 512, 1024)
        bh.bh_render(sc.handle, cams, [512], [512], *bufs, opts)
        torch.cuda.synchronize()
        after = _np(bufs, n)
        # a launch shape changes the schedule, never the result
        assert np.array_equal(before["flags"], after["flags"])
        assert np.array_equal(before["rgba"], after["rgba"])
        assert np.array_equal(before["theta"], after["theta"], equal_nan=True)
    finally:
        bh.bh_autotune_reset()
        sc.close()


def _batch_sample(w, n, k, seed):
    rng = np.random.default_rng(seed)
    sizes = np.array([c.w * c.h for c in w.cameras])
    offs = np.concatenate([[0], np.cumsum(sizes)])
    idx = np.sort(rng.choice(n, k, replace=False))
    cam = np.searchsorted(offs, idx, side="right") - 1
    loc = idx - offs[cam]
    px = loc % np.array([w.cameras[c].w for c in cam])
    py = loc // np.array([w.cameras[c].w for c in cam])
    return idx, cam, px, py


@pytest.mark.parametrize("mode", ["fp32", "surrogate"])
def test_batch64_full_size_sampled_parity(mode):
    """The 64-camera orbit sequence at full resolution (about 9e7 rays) in
    one graph replay -- the FP32 integrator, or the surrogate with its FP32
    integrator fallback and FP64 photon-sphere band, each with the launch
    shape the autotuner picked on this workload -- checked against the
    oracle on 20000 sampled pixels."""
    import torch
    w = W.config5(64)
    n = w.n_rays
    sc = bh.Scene(w.scene)
    try:
        if mode == "surrogate":
            bh.bh_surrogate_load(sc.handle, WEIGHTS)
        cams = sc.cameras(w.cameras)
        wv, hv = [c.w for c in w.cameras], [c.h for c in w.cameras]
        opts = bh.render_opts(mode, rtol=w.rtol, atol=w.atol)
        out = _buffers(torch, n)
        res = bh.bh_autotune(sc.handle, cams, wv, hv, *out, opts)
        assert res["ms_best"] <= res["ms_default"]
        g = bh.bh_graph_create(sc.handle, cams, wv, hv, *out, opts)
        out[1].zero_()
        bh.bh_graph_launch(g)
        torch.cuda.synchronize()
        bh.bh_graph_destroy(g)
        st = sc.stats()
        assert st["rays"] == n and st["status"] == 0
        if mode == "surrogate":
            assert st["n_surrogate"] > 0.3 * n
        idx, cam, px, py = _batch_sample(w, n, 20000, 5)
        ref = oracle.render_pixels(w.scene, w.cameras, cam, px, py, parity.oracle_opts(mode),
                                   nthreads=16)
        full = _np(out, n)
        got = {k: v[idx] for k, v in full.items()}
        m = parity.compare(got, ref, mode)
        parity.assert_parity(m, mode)
    finally:
        bh.bh_autotune_reset()
        sc.close()
