"""Plain FP64 reference of the surrogate MLP (numpy).

TEST INFRASTRUCTURE ONLY, like the rest of this package: it checks the
tensor-core training and inference kernels and is itself checked against
central finite differences.

Network: x (12 features, zero padded to 16) -> W1 (16x64) + b1 -> SiLU ->
W2 (64x64) + b2 -> SiLU -> W3 (64x64) + b3 -> SiLU -> W4 (64x16) + b4, of
which the first 3 outputs are used.  Loss: mean squared error over the 3
used outputs and the samples.  The parameter vector stores, in order, W1,
b1, W2, b2, W3, b3, W4, b4, each W row-major as W[in][out].

With use_bf16=True the values the tensor-core kernels round are rounded the
same way: weights, output-layer and back-propagated gradients to BF16;
inputs and hidden activations, which the kernels feed as BF16 high + low
pairs, to hi + lo in the forward pass and to BF16 in the weight gradients;
everything else stays FP64.
"""
from __future__ import annotations

import numpy as np

K0, HID, NO, NOUT, NFEAT = 16, 64, 16, 3, 12
SHAPES = [("W1", (K0, HID)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
          ("W3", (HID, HID)), ("b3", (HID,)), ("W4", (HID, NO)), ("b4", (NO,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def bf16(a) -> np.ndarray:
    """Round float values to the nearest BF16 (ties to even), returned as
    float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_split(a) -> np.ndarray:
    """a as the sum of its BF16 rounding and the BF16 rounding of the rest."""
    hi = bf16(a)
    return hi + bf16(np.asarray(a, np.float64) - hi)


def unpack(p) -> dict:
    p = np.asarray(p, np.float64)
    out, o = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[n], np.float64).ravel() for n, _ in SHAPES])


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(p, x, use_bf16=False):
    """Outputs (n x 3) and the cached activations."""
    P = unpack(p)
    ident = (lambda a: np.asarray(a, np.float64))
    r = bf16 if use_bf16 else ident
    r2 = bf16_split if use_bf16 else ident
    n = len(x)
    x = np.asarray(x, np.float64)
    X = np.zeros((n, K0))
    X[:, :x.shape[1]] = x
    W = [r(P["W1"]), r(P["W2"]), r(P["W3"]), r(P["W4"])]
    b = [P["b1"], P["b2"], P["b3"], P["b4"]]
    Z1 = r2(X) @ W[0] + b[0]
    H1 = silu(Z1)
    Z2 = r2(H1) @ W[1] + b[1]
    H2 = silu(Z2)
    Z3 = r2(H2) @ W[2] + b[2]
    H3 = silu(Z3)
    Z4 = r2(H3) @ W[3] + b[3]
    cache = dict(X=X, Z1=Z1, H1=H1, Z2=Z2, H2=H2, Z3=Z3, H3=H3, Z4=Z4, W=W)
    return Z4[:, :NOUT], cache


def loss_and_grad(p, x, t, use_bf16=False):
    """(loss, gradient vector, outputs) of the mean squared error."""
    y, c = forward(p, x, use_bf16)
    r = bf16 if use_bf16 else (lambda a: np.asarray(a, np.float64))
    n = len(x)
    t = np.asarray(t, np.float64)
    e = y - t
    loss = float(np.sum(e * e) / (n * NOUT))
    dZ4 = np.zeros((n, NO))
    dZ4[:, :NOUT] = 2.0 * e / (n * NOUT)
    dZ4 = r(dZ4)
    W = c["W"]
    g = {}
    g["W4"] = r(c["H3"]).T @ dZ4
    g["b4"] = dZ4.sum(0)
    dZ3 = r((dZ4 @ W[3].T) * silu_grad(c["Z3"]))
    g["W3"] = r(c["H2"]).T @ dZ3
    g["b3"] = dZ3.sum(0)
    dZ2 = r((dZ3 @ W[2].T) * silu_grad(c["Z2"]))
    g["W2"] = r(c["H1"]).T @ dZ2
    g["b2"] = dZ2.sum(0)
    dZ1 = r((dZ2 @ W[1].T) * silu_grad(c["Z1"]))
    g["W1"] = r(c["X"]).T @ dZ1
    g["b1"] = dZ1.sum(0)
    return loss, pack(g), y


def loss_only(p, x, t):
    y, _ = forward(p, x)
    e = y - np.asarray(t, np.float64)
    return float(np.sum(e * e) / (len(x) * NOUT))
