"""The MLP surrogate on the GPU: integrator labels, tensor-core gradients
and inference against the FP64 reference MLP, training, calibrated
rendering against the oracle, persistence."""
import math
import os

import numpy as np
import pytest

import oracle
import parity
import paper_2507_16165_gb300 as bh
from gpu_util import render
from oracle import mlp
from paper_2507_16165_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_labels_match_oracle():
    import torch
    b, r, psi = W.surrogate_samples(4096, seed=11)
    keep = b < 0.95 * r
    b, r, psi = b[keep][:512], r[keep][:512], psi[keep][:512]
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    out = [torch.empty(len(b), dtype=torch.float64, device="cuda") for _ in range(3)]
    st = torch.empty(len(b), dtype=torch.int32, device="cuda")
    bh.bh_surrogate_labels(1.0, dev(b), dev(r), dev(psi), *out, st)
    torch.cuda.synchronize()
    phi, ua, ub = (o.cpu().numpy() for o in out)
    st = st.cpu().numpy()
    assert np.all(st == 0)
    for i in range(0, len(b), 8):
        u0 = 1.0 / r[i]
        v0 = math.sqrt(1.0 / b[i] ** 2 - u0 * u0 + 2 * u0 ** 3)
        f, pe, _ = oracle.orbit_exit(1.0, u0, v0)
        assert f == oracle.ESC
        assert abs(pe - phi[i]) < 1e-8 * max(1.0, 1.0 / (b[i] - 3 * math.sqrt(3)))
        us, _ = oracle.orbit_sample(1.0, u0, v0, np.array([psi[i], psi[i] + math.pi]))
        assert abs(us[0] - ua[i]) < 1e-9 and abs(us[1] - ub[i]) < 1e-9


def _rand_params(seed):
    rng = np.random.default_rng(seed)
    d = mlp.unpack(rng.normal(0.0, 0.25, mlp.NPARAM))
    d["W1"][mlp.NFEAT:, :] = 0.0
    d["W4"][:, 3:] = 0.0
    d["b4"][3:] = 0.0
    return mlp.pack(d).astype(np.float32)


# Element-wise allowances.  Both sides round the same values to BF16 (weights;
# back-propagated gradients; activations as BF16 high + low pairs); they
# differ by the kernels' SiLU, evaluated from the hardware tanh (relative
# error about 2^-11), and by FP32 accumulation.  A value that the two sides
# compute a hair apart may round to neighbouring BF16 numbers: one BF16
# spacing, at most 2^-7 of the value.  Each gradient element is a sum of
# products, so it is held to a multiple of the same sum taken over absolute
# values (the products' magnitudes, back-propagated through |W| and
# |SiLU'|): GRAD_ALLOW covers one BF16 spacing in each product plus the
# tanh error compounded over the three hidden layers.  Forward outputs carry
# no rounding of their own beyond the weights' (training: activations enter
# as BF16 pairs exact to 2^-16; inference: the same BF16 weight values held
# in FP16, activations as FP16 pairs exact to about 2^-22), only the tanh error:
# INFER_ALLOW of the absolute-value sum.
GRAD_ALLOW = 3 * 2.0 ** -7
INFER_ALLOW = 8 * 2.0 ** -11


def _abs_bounds(p, x, t):
    """Absolute-value sums of the forward products (per output) and of the
    backward products (per parameter) of the reference network."""
    _, c = mlp.forward(p.astype(np.float64), x.astype(np.float64), use_bf16=True)
    W = [np.abs(w) for w in c["W"]]
    P = mlp.unpack(p.astype(np.float64))
    n = len(x)
    # forward: |X||W1| + |b1| ... through |SiLU| (|SiLU(z)| <= |z|)
    A = np.abs(c["X"]) @ W[0] + np.abs(P["b1"])
    for k in (1, 2, 3):
        A = A @ W[k] + np.abs(P["b%d" % (k + 1)])
    fwd = A[:, :mlp.NOUT]
    # backward: |dZ| propagated through |W|^T and |SiLU'|
    y, _ = mlp.forward(p.astype(np.float64), x.astype(np.float64), use_bf16=True)
    dZ = np.zeros((n, mlp.NO))
    dZ[:, :mlp.NOUT] = np.abs(2.0 * (y - t) / (n * mlp.NOUT))
    g = {"W4": np.abs(c["H3"]).T @ dZ, "b4": dZ.sum(0)}
    for k, (H, Z) in zip((3, 2, 1), (("H2", "Z3"), ("H1", "Z2"), ("X", "Z1"))):
        dZ = (dZ @ W[k].T) * np.abs(mlp.silu_grad(c[Z]))
        g["W%d" % k] = np.abs(c[H]).T @ dZ
        g["b%d" % k] = dZ.sum(0)
    return fwd, mlp.pack(g)


def test_training_gradients_match_fp64_reference():
    """bh_mlp_grad element by element against the FP64 reference on the
    same BF16-rounded values (GRAD_ALLOW of each element's absolute-value
    sum), outputs likewise (INFER_ALLOW); and close to the exact FP64
    gradient in norm."""
    rng = np.random.default_rng(5)
    p = _rand_params(6)
    x = np.zeros((256, 16), np.float32)
    x[:, :mlp.NFEAT] = rng.uniform(-1, 1, (256, mlp.NFEAT))
    t = rng.normal(0, 1, (256, 3)).astype(np.float32)
    y, g, loss = bh.bh_mlp_grad(p, x, t)
    loss_r, g_r, y_r = mlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t, use_bf16=True)
    fwd, gabs = _abs_bounds(p, x, t)
    assert np.all(np.abs(y - y_r) <= INFER_ALLOW * fwd + 1e-6)
    assert abs(loss - loss_r) <= 1e-2 * loss_r
    err = np.abs(g - g_r)
    bound = GRAD_ALLOW * gabs + 1e-9
    bad = err > bound
    assert not bad.any(), (int(bad.sum()), float((err / bound).max()))
    # the BF16 path stays close to the exact FP64 gradient too
    _, g_exact, _ = mlp.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t)
    assert np.linalg.norm(g - g_exact) <= 5e-2 * np.linalg.norm(g_exact)


def test_inference_path_matches_fp64_reference():
    """The render's inference path (tcgen05 tensor-core MLP, FP16 W^T tiles)
    element by element against the FP64 reference on the BF16-rounded
    weights (INFER_ALLOW of each output's absolute-value sum)."""
    rng = np.random.default_rng(7)
    p = _rand_params(8)
    x = np.zeros((1000, 16), np.float32)
    x[:, :mlp.NFEAT] = rng.uniform(-1, 1, (1000, mlp.NFEAT))
    y = bh.bh_mlp_infer(p, x)
    y_r, _ = mlp.forward(p.astype(np.float64), x.astype(np.float64), use_bf16=True)
    fwd, _ = _abs_bounds(p, x, np.zeros((1000, 3)))
    err = np.abs(y - y_r)
    assert np.all(err <= INFER_ALLOW * fwd + 1e-6), float((err / (INFER_ALLOW * fwd + 1e-6)).max())


WEIGHTS = os.path.join(os.path.dirname(bh.__file__), "data", "surrogate_m1.bin")


@pytest.fixture(scope="module")
def trained():
    """The surrogate the project trained (paper_2507_16165_gb300/
    train_surrogate.py: 2^22 samples, 900 epochs), loaded into a scene."""
    w = W.config4(256, spheres=False)
    sc = bh.Scene(w.scene)
    bh.bh_surrogate_load(sc.handle, WEIGHTS)
    yield w, sc
    sc.close()


def test_training_converges():
    """A short training run from scratch: the integrator labels most
    in-domain samples and the loss falls two orders of magnitude below its
    starting value (about 0.5 for these targets)."""
    w = W.config4(16, spheres=False)
    sc = bh.Scene(w.scene)
    try:
        b, r, psi = W.surrogate_samples(1 << 18, seed=3)
        rep = bh.bh_surrogate_train(sc.handle, b, r, psi, epochs=40, batch=8192, seed=4)
    finally:
        sc.close()
    assert rep["n_valid"] > 0.25 * rep["n_samples"]
    assert rep["steps"] == 40 * (rep["n_train"] // 8192)
    assert rep["final_loss"] < 5e-3
    assert max(rep["val_rmse"]) < 0.15   # the untrained network starts near 0.7


BC = 3.0 * math.sqrt(3.0)


def _features(b, r, psi):
    """The network's 12 input features (restated from their definition:
    normalised ln(b - b_c), r and psi0; b_c/b, sin and |cos| of the flat
    exit angle alpha, cos and sin psi0, sin and cos of (alpha - psi0),
    10/r, (b_c/b)^2), zero padded to 16 columns."""
    s = b * np.sqrt(1 - 2 / r) / r
    c = np.sqrt(1 - np.minimum(s * s, 1))
    x = np.zeros((len(b), 16))
    x[:, 0] = (np.log(b - BC) + 1.155) / 8.06
    x[:, 1] = (r - 57.5) / 42.5
    x[:, 2] = (psi - math.pi / 2) / (math.pi / 2)
    x[:, 3] = BC / b
    x[:, 4] = s
    x[:, 5] = c
    x[:, 6] = np.cos(psi)
    x[:, 7] = np.sin(psi)
    x[:, 8] = s * np.cos(psi) + c * np.sin(psi)
    x[:, 9] = s * np.sin(psi) - c * np.cos(psi)
    x[:, 10] = 10 / r
    x[:, 11] = (BC / b) ** 2
    return x


def test_calibration_table_matches_its_definition(trained):
    """bh_surrogate_calibrate on fresh samples: per bin, the 99.9th
    percentiles recomputed here from integrator labels and the inference
    kernel agree with the library's, and a bin is served exactly when it
    has >= 50 samples and both percentiles are within the thresholds.
    The errors are differences of FP32 outputs near 1, so features rounded
    one ulp apart move them by a few ulps: 1% agreement is asked, and the
    served decision is checked where the percentiles are not within 1% of
    a threshold."""
    import torch
    w, sc = trained
    b, r, psi = W.surrogate_samples(1 << 16, seed=77)
    nb_lb, nb_r = 8, 4
    cal = bh.bh_surrogate_calibrate(sc.handle, b, r, psi, nb_lb=nb_lb, nb_r=nb_r)
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    lab = [torch.empty(len(b), dtype=torch.float64, device="cuda") for _ in range(3)]
    st = torch.empty(len(b), dtype=torch.int32, device="cuda")
    bh.bh_surrogate_labels(1.0, dev(b), dev(r), dev(psi), *lab, st)
    torch.cuda.synchronize()
    phi, ua, ub = (t.cpu().numpy() for t in lab)
    ok = (st.cpu().numpy() == 0) & (b > BC + 1e-5) & np.isfinite(ua) & np.isfinite(ub)
    b, r, psi, phi, ua, ub = b[ok], r[ok], psi[ok], phi[ok], ua[ok], ub[ok]
    params, _ = bh.bh_surrogate_get(sc.handle)
    x = _features(b, r, psi).astype(np.float32)
    y = bh.bh_mlp_infer(params, x).astype(np.float64)
    alpha = math.pi - np.arcsin(np.minimum(1.0, b * np.sqrt(1 - 2 / r) / r))
    t0 = ((phi - alpha) * b / 4 - 3) / 3
    err_d = np.abs((y[:, 0] - t0.astype(np.float32)) * 12 / b)
    ib = np.clip(((x[:, 0] + 1) * 0.5 * nb_lb).astype(int), 0, nb_lb - 1)
    ir = np.clip(((r - 15) / 85 * nb_r).astype(int), 0, nb_r - 1)
    for i in range(nb_lb):
        for j in range(nb_r):
            m = (ib == i) & (ir == j)
            assert cal["counts"][i, j] == m.sum()
            if m.sum() == 0:
                continue
            v = np.sort(err_d[m])
            q = v[min(len(v) - 1, math.ceil(0.999 * (len(v) - 1)))]
            assert abs(cal["p999_delta"][i, j] - q) <= 1e-2 * q + 1e-8
            rel = []
            for u, yk in ((ua[m], y[m, 1]), (ub[m], y[m, 2])):
                ut = (u * b[m]).astype(np.float32) / b[m]
                keep = (ut > 1 / 60) & (ut < 1 / 2.5)
                up = yk[keep] / b[m][keep]
                rel.append(np.where(up > 0, np.abs(ut[keep] / np.where(up > 0, up, 1) - 1), 1e9))
            rel = np.sort(np.concatenate(rel))
            qr = rel[min(len(rel) - 1, math.ceil(0.999 * (len(rel) - 1)))] if len(rel) else 0.0
            assert abs(cal["p999_r"][i, j] - qr) <= 1e-2 * qr + 1e-8
            if abs(q - 1e-3) > 1e-5 and abs(qr - 2e-3) > 2e-5:
                served = m.sum() >= 50 and q <= 1e-3 and qr <= 2e-3
                assert cal["served"][i, j] == served
    bh.bh_surrogate_load(sc.handle, WEIGHTS)   # restore the shipped table


def _timed_render(sc, cams, mode, reps=5, **kw):
    """Median device time (CUDA events) of renders of one frame, and stats."""
    import torch
    cam = cams[0]
    n = cam.w * cam.h
    f64 = mode == "fp64"
    dirs = torch.empty(2 * n, dtype=torch.float64 if f64 else torch.float32, device="cuda")
    flags = torch.empty(n, dtype=torch.int16, device="cuda")
    rgba = torch.empty(n, dtype=torch.int32, device="cuda")
    c = sc.cameras(cams)
    stream = torch.cuda.Stream()
    opts = bh.render_opts(mode, stream, **kw)
    ms = []
    for i in range(reps + 1):
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        bh.bh_render(sc.handle, c, [cam.w], [cam.h], dirs, flags, rgba, opts)
        e.record(stream)
        stream.synchronize()
        if i:
            ms.append(a.elapsed_time(e))
    bh.bh_scene_sync(sc.handle)
    return float(np.median(ms)), sc.stats(), flags


def test_network_gain_in_steps_and_time(trained):
    """What the network gains, on the config-4 frame at 2048^2 (spheres
    included): every ray it serves is finished without integration, so the
    surrogate render takes fewer integrator steps than the mixed-precision
    render of the same frame, by about the steps those rays would have
    cost; in time it renders the frame far faster than the FP64 integrator
    -- the paper's method in its own precision -- at its 1e-3 rad bound.
    Against the FP32 / mixed integrator the network costs more time per
    ray than the integration it saves (its 192 SiLU activations alone take
    about 12 SM cycles a ray on the special-function unit, against about 12
    for the whole FP32 integration); the measured ratio is printed, not
    asserted."""
    w = W.config4(2048)
    sc = bh.Scene(w.scene)
    try:
        bh.bh_surrogate_load(sc.handle, WEIGHTS)
        t64, s64, _ = _timed_render(sc, w.cameras, "fp64", reps=2, rtol=1e-10, atol=1e-10)
        tmx, smx, _ = _timed_render(sc, w.cameras, "mixed", rtol=1e-5, atol=1e-7)
        tsu, ssu, flags = _timed_render(sc, w.cameras, "surrogate", rtol=1e-5, atol=1e-7)
    finally:
        sc.close()
    n = w.n_rays
    served = ssu["n_surrogate"] / n
    assert served > 0.3
    assert int(((flags & bh.BH_FLAG_SURR) != 0).sum()) == ssu["n_surrogate"]
    total = smx["steps"]
    saved = total - ssu["steps"]
    # served rays are the cheaper ones (far from the photon sphere), so the
    # saving is a positive share of the steps but below the served share
    assert saved > 0.2 * served * total
    assert tsu < t64 / 5.0
    print(f"\nnetwork gain at 2048^2: served {served:.3f}, steps {total} -> {ssu['steps']}; "
          f"FP64 {t64:.3f} ms, mixed {tmx:.3f} ms, surrogate {tsu:.3f} ms "
          f"(x{t64 / tsu:.1f} over FP64, x{tmx / tsu:.2f} of mixed)")


@pytest.mark.parametrize("size,spheres", [(256, False), (256, True), (70, False)])
def test_surrogate_render_parity(trained, size, spheres):
    """The surrogate render against the oracle.  The surrogate pass takes 128
    queue slots a CTA; 70 x 70 leaves its queue (162 tiles of 8 x 4, 5184
    slots) half a group short and its edge tiles part outside the image."""
    import torch
    w0, sc0 = trained
    w = W.config4(size, spheres=spheres)
    sc = bh.Scene(w.scene)
    bh.bh_surrogate_load(sc.handle, WEIGHTS)
    out = sc.render(w.cameras, "surrogate", rtol=1e-5, atol=1e-7, tile_w=8, tile_h=4)
    torch.cuda.synchronize()
    bh.bh_scene_sync(sc.handle)
    st = sc.stats()
    got = {"theta": out["theta"].double().cpu().numpy(), "phi": out["phi"].double().cpu().numpy(),
           "flags": out["flags"].cpu().numpy().astype(np.uint16),
           "rgba": out["rgba"].cpu().numpy().astype(np.uint32)}
    sc.close()
    ref = oracle.render(w.scene, w.cameras, parity.oracle_opts("surrogate"), nthreads=8)
    m = parity.compare(got, ref, "surrogate")
    assert st["rays"] == w.n_rays
    assert st["n_surrogate"] > (0.3 if spheres else 0.6) * w.n_rays
    assert np.sum((got["flags"] & bh.BH_FLAG_SURR) != 0) == st["n_surrogate"]
    # served rays never include the photon-sphere band or sphere planes
    assert not np.any((got["flags"] & bh.BH_FLAG_SURR) & (got["flags"] & bh.BH_FLAG_BAND))
    parity.assert_parity(m, "surrogate")


def test_save_load_roundtrip(trained, tmp_path):
    import torch
    w, sc = trained
    path = str(tmp_path / "surr.bin")
    bh.bh_surrogate_save(sc.handle, path)
    p0, t0 = bh.bh_surrogate_get(sc.handle)
    sc2 = bh.Scene(w.scene)
    try:
        bh.bh_surrogate_load(sc2.handle, path)
        p1, t1 = bh.bh_surrogate_get(sc2.handle)
        assert np.array_equal(p0, p1) and np.array_equal(t0, t1)
        a = sc.render(w.cameras, "surrogate")
        b = sc2.render(w.cameras, "surrogate")
        torch.cuda.synchronize()
        assert torch.equal(a["flags"], b["flags"]) and torch.equal(a["rgba"], b["rgba"])
        # a corrupted file is refused, not loaded
        raw = bytearray(open(path, "rb").read())
        raw[100] ^= 0xFF
        bad = str(tmp_path / "bad.bin")
        open(bad, "wb").write(bytes(raw))
        with pytest.raises(bh.BHError) as e:
            bh.bh_surrogate_load(sc2.handle, bad)
        assert e.value.code == -6
    finally:
        sc2.close()


def test_surrogate_without_training_is_refused():
    import torch
    w = W.config4(16, spheres=False)
    sc = bh.Scene(w.scene)
    try:
        with pytest.raises(bh.BHError) as e:
            sc.render(w.cameras, "surrogate")
        assert e.value.code == -5
    finally:
        sc.close()
    torch.cuda.synchronize()


def test_tensor_core_wait_gives_up_and_device_stays_usable():
    """The tensor-core kernels' bounded wait, run out on purpose: one CTA
    holds tensor memory and waits on a barrier that nothing arrives on.  The
    wait gives up and reports, the tensor memory is released (a second run
    allocates again), and the inference kernel, which allocates tensor
    memory too, still runs and matches the FP64 network."""
    for _ in range(2):
        r = bh.bh_selftest_wait_timeout(tries=20, wait_ns=100000)
        assert r["timed_out"]
        assert 0.0 < r["waited_ms"] < 1000.0
    rng = np.random.default_rng(3)
    p = _rand_params(4)
    x = np.zeros((256, 16), np.float32)
    x[:, :mlp.NFEAT] = rng.uniform(-1, 1, (256, mlp.NFEAT))
    y = bh.bh_mlp_infer(p, x)
    y_r, _ = mlp.forward(p.astype(np.float64), x.astype(np.float64), use_bf16=True)
    fwd, _ = _abs_bounds(p, x, np.zeros((256, 3)))
    assert np.all(np.abs(y - y_r) <= INFER_ALLOW * fwd + 1e-6)


@pytest.mark.parametrize("r_obs", [10.0, 150.0])
def test_surrogate_outside_training_domain_falls_back(trained, r_obs):
    """Observers outside the network's training domain (r_obs in [15, 100] M):
    the network serves no ray, every ray goes to the integrator's fallback
    passes, and the render matches the oracle at the surrogate form's bars."""
    import torch
    sc0 = W.config4(16, spheres=False).scene
    cam = W.Camera(r_obs, 75.0, 64, 48, azim_deg=15.0, fov_deg=60.0 if r_obs < 50 else 12.0)
    sc = bh.Scene(sc0)
    bh.bh_surrogate_load(sc.handle, WEIGHTS)
    out = sc.render([cam], "surrogate", rtol=1e-5, atol=1e-7)
    torch.cuda.synchronize()
    bh.bh_scene_sync(sc.handle)
    st = sc.stats()
    got = {"theta": out["theta"].double().cpu().numpy(), "phi": out["phi"].double().cpu().numpy(),
           "flags": out["flags"].cpu().numpy().astype(np.uint16),
           "rgba": out["rgba"].cpu().numpy().astype(np.uint32)}
    sc.close()
    assert st["n_surrogate"] == 0
    assert st["n_fallback"] + st["n_band"] <= st["rays"] == cam.w * cam.h
    ref = oracle.render(sc0, [cam], parity.oracle_opts("surrogate"), nthreads=8)
    parity.assert_parity(parity.compare(got, ref, "surrogate"), "surrogate")
