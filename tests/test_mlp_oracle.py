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


def test_forward_routes_one_feature_through_distinct_units():
    """A network whose weights route feature 2 to hidden unit 5, then unit 9,
    then unit 13, then output 1 (scales 1.5, -0.7, 2.0, 3.0; a bias on each
    unit on the route and on every output) reduces to a composition of SiLU,
    z * logistic(z), with SciPy's logistic function.  A transposed weight
    matrix, a bias on the wrong layer or unit, another activation or an
    output read from the wrong column fails it."""
    from scipy.special import expit

    def silu(z):
        return z * expit(z)

    d = mlp.unpack(np.zeros(mlp.NPARAM))
    d["W1"][2, 5] = 1.5
    d["b1"][5] = 0.1
    d["W2"][5, 9] = -0.7
    d["b2"][9] = -0.2
    d["W3"][9, 13] = 2.0
    d["b3"][13] = 0.3
    d["W4"][13, 1] = 3.0
    d["b4"][:3] = [0.25, -0.5, 0.75]
    p = mlp.pack(d)
    x = np.zeros((5, mlp.NFEAT))
    x[:, 2] = [-3.0, -0.4, 0.0, 0.9, 4.0]
    x[:, 0] = 7.0  # a feature that no weight routes: no effect
    y, _ = mlp.forward(p, x)
    h1 = silu(1.5 * x[:, 2] + 0.1)
    h2 = silu(-0.7 * h1 - 0.2)
    h3 = silu(2.0 * h2 + 0.3)
    np.testing.assert_allclose(y[:, 1], 3.0 * h3 - 0.5, rtol=1e-14, atol=1e-15)
    np.testing.assert_array_equal(y[:, 0], np.full(5, 0.25))
    np.testing.assert_array_equal(y[:, 2], np.full(5, 0.75))
    # every unit off the route holds SiLU(0) = 0: the hidden biases elsewhere are zero
    _, cache = mlp.forward(p, x)
    assert np.all(np.delete(cache["H1"], 5, axis=1) == 0.0)
    assert np.all(np.delete(cache["H2"], 9, axis=1) == 0.0)


def test_forward_pin_catches_planted_mistakes(monkeypatch):
    """Mistakes planted in a copy of the reference's source, on the CPU: each
    makes the routing pin above fail."""
    import inspect
    import sys
    import types

    import pytest

    src = inspect.getsource(mlp)
    planted = [
        ("Z2 = r2(H1) @ W[1] + b[1]", "Z2 = r2(H1) @ W[1].T + b[1]"),       # transposed operand
        ("Z3 = r2(H2) @ W[2] + b[2]", "Z3 = r2(H2) @ W[2] + b[1]"),         # bias of another layer
        ("return z / (1.0 + np.exp(-z))", "return np.tanh(z)"),              # another activation
        ("return Z4[:, :NOUT], cache", "return Z4[:, 1:NOUT + 1], cache"),  # outputs shifted
        ("Z1 = r2(X) @ W[0] + b[0]", "Z1 = r2(X) @ W[0]"),                  # dropped bias
    ]
    this = sys.modules[__name__]
    for old, new in planted:
        assert src.count(old) == 1, old
        mutant = types.ModuleType("mlp_mutant")
        exec(compile(src.replace(old, new), "mlp_mutant", "exec"), mutant.__dict__)
        monkeypatch.setattr(this, "mlp", mutant)
        with pytest.raises(AssertionError):
            test_forward_routes_one_feature_through_distinct_units()
    monkeypatch.setattr(this, "mlp", mlp)
