"""The FP64 reference MLP against central finite differences and the BF16
rounding rule (test infrastructure for the tensor-core kernels)."""
import numpy as np

from oracle import mlp
from paper_2507_16165_gb300 import _capi


def _params(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, mlp.NPARAM)
    d = mlp.unpack(p)
    d["W1"][mlp.NFEAT:, :] = 0.0  # padded inputs
    d["W4"][:, 3:] = 0.0          # padded outputs
    d["b4"][3:] = 0.0
    return mlp.pack(d)


def test_parameter_count_matches_the_c_abi():
    assert mlp.NPARAM == _capi.BH_MLP_NPARAM == 10448


def test_bf16_rounding_rule():
    v = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.0e38, 1e-40])
    r = mlp.bf16(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                 # halfway: ties to even
    assert r[2] == 1.0 + 2 ** -7       # above halfway: rounds up
    assert r[3] == -2.5
    assert np.isfinite(r[4])
    assert abs(r[5]) < 1e-39


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(2)
    x = rng.uniform(-1, 1, (24, mlp.NFEAT))
    t = rng.normal(0, 1, (24, 3))
    _, g, _ = mlp.loss_and_grad(p, x, t)
    idx = rng.choice(np.flatnonzero(np.abs(g) > 1e-6), 60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_only(pp, x, t) - mlp.loss_only(pm, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_padding_gets_no_gradient():
    rng = np.random.default_rng(3)
    p = _params(4)
    x = rng.uniform(-1, 1, (16, mlp.NFEAT))
    t = rng.normal(0, 1, (16, 3))
    _, g, _ = mlp.loss_and_grad(p, x, t)
    d = mlp.unpack(g)
    assert np.all(d["W1"][mlp.NFEAT:, :] == 0.0)
    assert np.all(d["W4"][:, 3:] == 0.0)
    assert np.all(d["b4"][3:] == 0.0)
