"""Helpers for GPU tests: render through the C-ABI and pull results to numpy."""
from __future__ import annotations

import numpy as np

import paper_2507_16165_gb300 as bh


def to_numpy(out: dict) -> dict:
    return {"theta": out["theta"].double().cpu().numpy(),
            "phi": out["phi"].double().cpu().numpy(),
            "flags": out["flags"].cpu().numpy().astype(np.uint16),
            "rgba": out["rgba"].cpu().numpy().astype(np.uint32)}


def render(scene, cams, mode, **kw):
    """(numpy outputs, stats) of one render of workloads.Camera-like cams."""
    import torch
    sc = bh.Scene(scene)
    try:
        out = sc.render(cams, mode, **kw)
        torch.cuda.synchronize()
        bh.bh_scene_sync(sc.handle)
        st = sc.stats()
        return to_numpy(out), st
    finally:
        sc.close()
