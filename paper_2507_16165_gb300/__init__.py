"""GB300 Schwarzschild light-ray renderer: thin Python binding of libbh.so.

The functions named bh_* mirror the C-ABI in include/bh.h one to one and only
marshal arguments (torch tensors -> device pointers, Python numbers -> C
structs).  All rendering runs in the CUDA kernels of libbh.so; importing this
package does not load the library, the first bh_* call does, and it raises if
the library has not been built.

    import torch, paper_2507_16165_gb300 as bh
    from paper_2507_16165_gb300 import workloads as W
    w = W.config2(256, "fp32")
    out = bh.render_workload(w)            # dict of torch CUDA tensors
"""
from __future__ import annotations

import ctypes

from . import _capi
from ._capi import (BH_FLAG_BAND, BH_FLAG_CAPT, BH_FLAG_DISK, BH_FLAG_ESC,  # noqa: F401
                    BH_FLAG_FP64, BH_FLAG_SPHERE, BH_FLAG_STEP_LIMIT, BH_FLAG_SURR,
                    BH_MODE_FP32, BH_MODE_FP64, BH_MODE_MIXED, BH_MODE_PAPER_EPS,
                    BH_MAX_HOST_STRIPS, BH_MODE_PAPER_EPS_FP32, BH_MODE_SURROGATE, MODES,
                    BHError, check)

__all__ = ["bh_version", "bh_last_error", "bh_scene_create", "bh_scene_destroy",
           "bh_scene_sky_texture",
           "bh_camera_set", "bh_render", "bh_render_host", "bh_scene_sync",
           "bh_render_stats", "bh_render_noalloc", "bh_graph_create", "bh_graph_launch",
           "bh_graph_destroy", "bh_autotune", "bh_autotune_reset", "bh_surrogate_labels",
           "bh_surrogate_train", "bh_surrogate_calibrate", "bh_surrogate_get", "bh_surrogate_save", "bh_surrogate_load",
           "bh_mlp_grad", "bh_mlp_infer", "bh_selftest_wait_timeout", "Scene", "render_opts",
           "render_workload"]


def bh_version() -> int:
    return int(_capi.lib().bh_version())


def bh_last_error() -> str:
    return _capi.lib().bh_last_error().decode(errors="replace")


def scene_desc(scene) -> _capi.bh_scene_desc:
    """C scene description from a workloads.Scene-like object."""
    d = _capi.bh_scene_desc()
    d.mass = float(scene.mass)
    disk = getattr(scene, "disk", None)
    d.disk_enabled = 1 if disk is not None else 0
    if disk is not None:
        d.disk_r_in, d.disk_r_out = float(disk[0]), float(disk[1])
    sph = list(getattr(scene, "spheres", ()))
    if len(sph) > _capi.BH_MAX_SPHERES:
        raise ValueError("at most 8 spheres")
    d.n_spheres = len(sph)
    for k, s in enumerate(sph):
        d.spheres[k].center[:] = [float(x) for x in s.center]
        d.spheres[k].radius = float(s.radius)
        d.spheres[k].albedo[:] = [float(x) for x in s.albedo]
    d.sky_seed = int(scene.sky_seed)
    d.ic = int(getattr(scene, "ic", 0))
    return d


def bh_scene_sky_texture(scene: int, texels) -> None:
    """Use an equirectangular RGBA8 image (h x w uint32 host array) as the
    sky; None restores the procedural checker."""
    import numpy as np
    if texels is None:
        check(_capi.lib().bh_scene_sky_texture(scene, None, 0, 0), "bh_scene_sky_texture")
        return
    t = np.ascontiguousarray(texels, np.uint32)
    if t.ndim != 2:
        raise ValueError("texels must be an h x w array")
    check(_capi.lib().bh_scene_sky_texture(scene, t.ctypes.data, t.shape[1], t.shape[0]),
          "bh_scene_sky_texture")


def bh_scene_create(desc: _capi.bh_scene_desc) -> int:
    h = ctypes.c_void_p()
    check(_capi.lib().bh_scene_create(ctypes.byref(desc), ctypes.byref(h)), "bh_scene_create")
    return h.value


def bh_scene_destroy(handle: int) -> None:
    if handle:
        _capi.lib().bh_scene_destroy(handle)


def bh_camera_set(r_obs: float, incl_deg: float, azim_deg: float = 0.0,
                  fov_deg: float = 60.0) -> _capi.bh_camera:
    cam = _capi.bh_camera()
    check(_capi.lib().bh_camera_set(ctypes.byref(cam), r_obs, incl_deg, azim_deg, fov_deg),
          "bh_camera_set")
    return cam


def render_opts(mode="mixed", stream=None, **kw) -> _capi.bh_render_opts:
    """bh_render_opts from keyword arguments (unset fields: tuned defaults)."""
    o = _capi.bh_render_opts()
    o.mode = MODES[mode] if isinstance(mode, str) else int(mode)
    o.stream = _stream_ptr(stream)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown render option {k}")
        setattr(o, k, v)
    return o


def _stream_ptr(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream or None
        except Exception:
            return None
        return None
    return int(getattr(stream, "cuda_stream", stream)) or None


def _cams_array(cams):
    arr = (_capi.bh_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = c
    return arr


def _ptr(t) -> int | None:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr() or None
    if hasattr(t, "ctypes"):
        return t.ctypes.data
    return int(t)


def bh_render(scene: int, cams, w, h, out_dirs, out_flags, out_rgba8, opts) -> None:
    """Asynchronous render into device tensors (see include/bh.h)."""
    n = len(cams)
    W = (ctypes.c_int * n)(*[int(x) for x in w])
    H = (ctypes.c_int * n)(*[int(x) for x in h])
    check(_capi.lib().bh_render(scene, _cams_array(cams), n, W, H, _ptr(out_dirs),
                                _ptr(out_flags), _ptr(out_rgba8), ctypes.byref(opts)),
          "bh_render")


def bh_render_host(scene: int, cams, w, h, host_dirs, host_flags, host_rgba8, opts) -> None:
    """Render into host buffers (numpy arrays or CPU tensors); synchronous."""
    n = len(cams)
    W = (ctypes.c_int * n)(*[int(x) for x in w])
    H = (ctypes.c_int * n)(*[int(x) for x in h])
    check(_capi.lib().bh_render_host(scene, _cams_array(cams), n, W, H, _ptr(host_dirs),
                                     _ptr(host_flags), _ptr(host_rgba8), ctypes.byref(opts)),
          "bh_render_host")


def bh_render_noalloc(desc: _capi.bh_scene_desc, cams, w, h, out_dirs, out_flags, out_rgba8,
                      opts) -> None:
    """bh_render_noalloc of the C-ABI: FP32 / FP64 render into caller device
    buffers using only the library's fixed scratch array (no allocation)."""
    n = len(cams)
    W = (ctypes.c_int * n)(*[int(x) for x in w])
    H = (ctypes.c_int * n)(*[int(x) for x in h])
    check(_capi.lib().bh_render_noalloc(ctypes.byref(desc), _cams_array(cams), n, W, H,
                                        _ptr(out_dirs), _ptr(out_flags), _ptr(out_rgba8),
                                        ctypes.byref(opts)), "bh_render_noalloc")


def bh_graph_create(scene: int, cams, w, h, out_dirs, out_flags, out_rgba8, opts) -> int:
    """Capture one render into a CUDA graph; returns the bh_graph handle."""
    n = len(cams)
    W = (ctypes.c_int * n)(*[int(x) for x in w])
    H = (ctypes.c_int * n)(*[int(x) for x in h])
    g = ctypes.c_void_p()
    check(_capi.lib().bh_graph_create(scene, _cams_array(cams), n, W, H, _ptr(out_dirs),
                                      _ptr(out_flags), _ptr(out_rgba8), ctypes.byref(opts),
                                      ctypes.byref(g)), "bh_graph_create")
    return g.value


def bh_graph_launch(graph: int, stream=None) -> None:
    check(_capi.lib().bh_graph_launch(graph, _stream_ptr(stream)), "bh_graph_launch")


def bh_graph_destroy(graph: int) -> None:
    if graph:
        _capi.lib().bh_graph_destroy(graph)


def bh_autotune(scene: int, cams, w, h, out_dirs, out_flags, out_rgba8, opts) -> dict:
    """Time launch shapes on this workload; the fastest becomes the default."""
    n = len(cams)
    W = (ctypes.c_int * n)(*[int(x) for x in w])
    H = (ctypes.c_int * n)(*[int(x) for x in h])
    res = _capi.bh_tune_result()
    check(_capi.lib().bh_autotune(scene, _cams_array(cams), n, W, H, _ptr(out_dirs),
                                  _ptr(out_flags), _ptr(out_rgba8), ctypes.byref(opts),
                                  ctypes.byref(res)), "bh_autotune")
    return {name: getattr(res, name) for name, _ in _capi.bh_tune_result._fields_}


def bh_autotune_reset() -> None:
    check(_capi.lib().bh_autotune_reset(), "bh_autotune_reset")


def bh_surrogate_labels(mass: float, b, r_obs, psi0, phi_inf, u_a, u_b, status, stream=None):
    """FP64 integrator labels of bare orbits into device tensors."""
    check(_capi.lib().bh_surrogate_labels(float(mass), int(b.numel()), _ptr(b), _ptr(r_obs),
                                          _ptr(psi0), _ptr(phi_inf), _ptr(u_a), _ptr(u_b),
                                          _ptr(status), _stream_ptr(stream)),
          "bh_surrogate_labels")


def bh_surrogate_train(scene: int, b, r_obs, psi0, stream=None, **kw) -> dict:
    """Train and calibrate the scene's surrogate on host float64 arrays."""
    import numpy as np
    b = np.ascontiguousarray(b, np.float64)
    r_obs = np.ascontiguousarray(r_obs, np.float64)
    psi0 = np.ascontiguousarray(psi0, np.float64)
    o = _capi.bh_train_opts()
    o.stream = _stream_ptr(stream)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown training option {k}")
        setattr(o, k, v)
    rep = _capi.bh_train_report()
    check(_capi.lib().bh_surrogate_train(scene, len(b), _ptr(b), _ptr(r_obs), _ptr(psi0),
                                         ctypes.byref(o), ctypes.byref(rep)), "bh_surrogate_train")
    out = {n: getattr(rep, n) for n, _ in _capi.bh_train_report._fields_}
    out["val_rmse"] = list(rep.val_rmse)
    return out


def bh_surrogate_calibrate(scene: int, b, r_obs, psi0, nb_lb=32, nb_r=8, stream=None,
                           **kw) -> dict:
    """Recalibrate the scene's surrogate on held-out host float64 samples.

    Returns per-bin arrays of shape (nb_lb, nb_r): p999_delta (rad),
    p999_r (M), counts, served (bool), and served_fraction."""
    import numpy as np
    b = np.ascontiguousarray(b, np.float64)
    r_obs = np.ascontiguousarray(r_obs, np.float64)
    psi0 = np.ascontiguousarray(psi0, np.float64)
    o = _capi.bh_calib_opts()
    o.nb_lb, o.nb_r = int(nb_lb), int(nb_r)
    o.stream = _stream_ptr(stream)
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown calibration option {k}")
        setattr(o, k, v)
    nbin = o.nb_lb * o.nb_r
    pd = np.empty(nbin, np.float32)
    pr = np.empty(nbin, np.float32)
    cnt = np.empty(nbin, np.int32)
    served = ctypes.c_float()
    check(_capi.lib().bh_surrogate_calibrate(scene, len(b), _ptr(b), _ptr(r_obs), _ptr(psi0),
                                             ctypes.byref(o), _ptr(pd), _ptr(pr), _ptr(cnt),
                                             ctypes.byref(served)), "bh_surrogate_calibrate")
    _, table = bh_surrogate_get(scene)
    shape = (o.nb_lb, o.nb_r)
    return {"p999_delta": pd.reshape(shape), "p999_r": pr.reshape(shape),
            "counts": cnt.reshape(shape), "served": table.astype(bool),
            "served_fraction": served.value}


def bh_surrogate_get(scene: int):
    """(FP32 parameters, calibration table as an (nb_lb, nb_r) array)."""
    import numpy as np
    p = np.empty(_capi.BH_MLP_NPARAM, np.float32)
    nb_lb, nb_r = ctypes.c_int(), ctypes.c_int()
    check(_capi.lib().bh_surrogate_get(scene, None, None, ctypes.byref(nb_lb), ctypes.byref(nb_r)),
          "bh_surrogate_get")
    t = np.empty(nb_lb.value * nb_r.value, np.uint8)
    check(_capi.lib().bh_surrogate_get(scene, _ptr(p), _ptr(t), None, None), "bh_surrogate_get")
    return p, t.reshape(nb_lb.value, nb_r.value)


def bh_surrogate_save(scene: int, path: str) -> None:
    check(_capi.lib().bh_surrogate_save(scene, path.encode()), "bh_surrogate_save")


def bh_surrogate_load(scene: int, path: str) -> None:
    check(_capi.lib().bh_surrogate_load(scene, path.encode()), "bh_surrogate_load")


def bh_mlp_grad(params, x, t, stream=None):
    """(outputs, gradient, loss) of one forward/backward pass (host arrays)."""
    import numpy as np
    params = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    if x.ndim != 2 or x.shape[1] != 16:
        raise ValueError("x must be n x 16 feature rows")
    n = len(x)
    y = np.empty((n, 3), np.float32)
    g = np.empty(_capi.BH_MLP_NPARAM, np.float32)
    loss = ctypes.c_float()
    check(_capi.lib().bh_mlp_grad(_ptr(params), n, _ptr(x), _ptr(t), _ptr(y), _ptr(g),
                                  ctypes.byref(loss), _stream_ptr(stream)), "bh_mlp_grad")
    return y, g, loss.value


def bh_selftest_wait_timeout(tries: int = 20, wait_ns: int = 100000) -> dict:
    """Run out the tensor-core kernels' bounded wait on purpose (nothing
    arrives on its barrier): {"timed_out": bool, "waited_ms": float}."""
    t = ctypes.c_int()
    ms = ctypes.c_double()
    check(_capi.lib().bh_selftest_wait_timeout(int(tries), int(wait_ns), ctypes.byref(t),
                                               ctypes.byref(ms)), "bh_selftest_wait_timeout")
    return {"timed_out": bool(t.value), "waited_ms": ms.value}


def bh_mlp_infer(params, x, stream=None):
    """Outputs of the render's inference MLP (host arrays)."""
    import numpy as np
    params = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    if x.ndim != 2 or x.shape[1] != 16:
        raise ValueError("x must be n x 16 feature rows")
    y = np.empty((len(x), 3), np.float32)
    check(_capi.lib().bh_mlp_infer(_ptr(params), len(x), _ptr(x), _ptr(y), _stream_ptr(stream)),
          "bh_mlp_infer")
    return y


def bh_scene_sync(scene: int) -> None:
    check(_capi.lib().bh_scene_sync(scene), "bh_scene_sync")


def bh_render_stats(scene: int) -> dict:
    st = _capi.bh_stats()
    check(_capi.lib().bh_render_stats(scene, ctypes.byref(st)), "bh_render_stats")
    out = {name: int(getattr(st, name)) for name, _ in _capi.bh_stats._fields_
           if name != "kernel_ms"}
    out["kernel_ms"] = [float(x) for x in st.kernel_ms]
    return out


class Scene:
    """Owns a bh_scene handle for a workloads.Scene-like description."""

    def __init__(self, scene):
        self.spec = scene
        self.handle = bh_scene_create(scene_desc(scene))
        tex = getattr(scene, "sky_texture", None)
        if tex is not None:
            bh_scene_sky_texture(self.handle, tex)

    def close(self):
        if self.handle:
            bh_scene_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def cameras(self, cams):
        return [bh_camera_set(c.r_obs, c.incl_deg, c.azim_deg, c.fov_deg) for c in cams]

    def render(self, cams, mode="mixed", dirs=None, flags=None, rgba=None, stream=None, **kw):
        """Render workloads.Camera-like cameras into (new or given) CUDA tensors."""
        import torch
        n = sum(int(c.w) * int(c.h) for c in cams)
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        dt = torch.float64 if m in (BH_MODE_FP64, BH_MODE_PAPER_EPS) else torch.float32
        dev = torch.device("cuda", torch.cuda.current_device())
        if dirs is None:
            dirs = torch.empty(2 * n, dtype=dt, device=dev)
        if flags is None:
            flags = torch.empty(n, dtype=torch.int16, device=dev)
        if rgba is None:
            rgba = torch.empty(n, dtype=torch.int32, device=dev)
        opts = render_opts(m, stream, **kw)
        bh_render(self.handle, self.cameras(cams), [c.w for c in cams], [c.h for c in cams],
                  dirs, flags, rgba, opts)
        return {"theta": dirs[:n], "phi": dirs[n:], "flags": flags, "rgba": rgba}

    def stats(self) -> dict:
        return bh_render_stats(self.handle)


def render_workload(w, mode=None, **kw) -> dict:
    """Render a workloads.Workload with its own mode and tolerances."""
    sc = Scene(w.scene)
    out = sc.render(w.cameras, mode or w.mode, rtol=w.rtol, atol=w.atol, band=w.band, **kw)
    out["stats"] = sc.stats()
    sc.close()
    return out
