"""The C-ABI library on the host: it loads, exports what include/bh.h
declares, matches the header's struct layout, and rejects bad arguments
before touching a device (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2507_16165_gb300 as bh
from paper_2507_16165_gb300 import _build, _capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bh.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_capi.LIB_PATH):
        _build.build()
    return _capi.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bh_[a-z0-9_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "bh_render" in names and "bh_scene_create" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in bh.h but not exported"
    out = subprocess.run(["nm", "-D", "--defined-only", _capi.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(bh_[a-z0-9_]+)", out))
    assert set(names) <= exported
    assert {n for n, _, _ in _capi.SIGNATURES} <= exported


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "bh.h"\nint main(void){'
                   'printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(bh_sphere), sizeof(bh_scene_desc),'
                   'sizeof(bh_camera), sizeof(bh_render_opts), sizeof(bh_stats),'
                   'offsetof(bh_render_opts, abort_after), offsetof(bh_stats, kernel_ms),'
                   'sizeof(bh_tune_result), offsetof(bh_render_opts, h_max_far),'
                   'offsetof(bh_render_opts, paper_eps), offsetof(bh_render_opts, spp),'
                   'offsetof(bh_render_opts, doppler), offsetof(bh_render_opts, rtol_far),'
                   'offsetof(bh_render_opts, host_strips), offsetof(bh_render_opts, rtol_near),'
                   'offsetof(bh_render_opts, queue_chunk), offsetof(bh_tune_result, queue_chunk));'
                   'return 0;}')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(_capi.bh_sphere), ctypes.sizeof(_capi.bh_scene_desc),
            ctypes.sizeof(_capi.bh_camera), ctypes.sizeof(_capi.bh_render_opts),
            ctypes.sizeof(_capi.bh_stats), _capi.bh_render_opts.abort_after.offset,
            _capi.bh_stats.kernel_ms.offset, ctypes.sizeof(_capi.bh_tune_result),
            _capi.bh_render_opts.h_max_far.offset, _capi.bh_render_opts.paper_eps.offset,
            _capi.bh_render_opts.spp.offset, _capi.bh_render_opts.doppler.offset,
            _capi.bh_render_opts.rtol_far.offset, _capi.bh_render_opts.host_strips.offset,
            _capi.bh_render_opts.rtol_near.offset, _capi.bh_render_opts.queue_chunk.offset,
            _capi.bh_tune_result.queue_chunk.offset]
    assert got == want


def test_version(lib):
    assert bh.bh_version() == 2


def test_camera_basis(lib):
    import numpy as np
    for inc, az in [(90.0, 0.0), (75.0, 30.0), (0.0, 0.0), (180.0, 12.0), (45.0, -100.0)]:
        c = bh.bh_camera_set(50.0, inc, az, 60.0)
        f, r, u, p = (np.array(x[:]) for x in (c.fwd, c.right, c.up, c.pos))
        assert np.allclose(p, -50.0 * f)
        for a, b in [(f, r), (f, u), (r, u)]:
            assert abs(np.dot(a, b)) < 1e-14
        for a in (f, r, u):
            assert abs(np.linalg.norm(a) - 1) < 1e-14
        assert np.allclose(np.cross(r, f), u)
        assert abs(c.tan_half - np.tan(np.radians(30.0))) < 1e-15


@pytest.mark.parametrize("args", [(-1.0, 10.0, 0.0, 60.0), (10.0, 10.0, 0.0, 0.0),
                                  (10.0, 10.0, 0.0, 180.0), (float("nan"), 0.0, 0.0, 60.0)])
def test_camera_rejects(lib, args):
    with pytest.raises(bh.BHError) as e:
        bh.bh_camera_set(*args)
    assert e.value.code == _capi.BH_E_INVALID


def _desc(**kw):
    from paper_2507_16165_gb300 import workloads as W
    d = bh.scene_desc(W.config3(8).scene)
    for k, v in kw.items():
        setattr(d, k, v)
    return d


@pytest.mark.parametrize("kw", [dict(mass=-1.0), dict(disk_r_in=1.5), dict(disk_r_out=5.0),
                                dict(n_spheres=9), dict(n_spheres=-1), dict(ic=2)])
def test_scene_rejects_before_device(lib, kw):
    h = ctypes.c_void_p()
    rc = lib.bh_scene_create(ctypes.byref(_desc(**kw)), ctypes.byref(h))
    assert rc == _capi.BH_E_INVALID
    assert h.value is None
    assert bh.bh_last_error()


def test_scene_rejects_sphere_inside_horizon(lib):
    d = _desc()
    d.spheres[0].center[:] = [1.0, 0.0, 0.0]
    h = ctypes.c_void_p()
    assert lib.bh_scene_create(ctypes.byref(d), ctypes.byref(h)) == _capi.BH_E_INVALID


def test_null_arguments(lib):
    assert lib.bh_scene_create(None, None) == _capi.BH_E_INVALID
    o = bh.render_opts("fp32", stream=0)
    cams = (_capi.bh_camera * 1)()
    W = (ctypes.c_int * 1)(4)
    assert lib.bh_render(None, cams, 1, W, W, None, None, None, ctypes.byref(o)) == _capi.BH_E_INVALID
    assert lib.bh_render_stats(None, None) == _capi.BH_E_INVALID
    assert lib.bh_scene_sync(None) == _capi.BH_E_INVALID
    lib.bh_scene_destroy(None)


def test_binding_fails_loudly_without_library(tmp_path):
    """No silent fallback: a missing library is an error, not a CPU path."""
    saved = _capi._lib
    try:
        _capi._lib = None
        with pytest.raises(RuntimeError, match="build the CUDA extension"):
            _capi.lib(str(tmp_path / "missing.so"))
    finally:
        _capi._lib = saved
