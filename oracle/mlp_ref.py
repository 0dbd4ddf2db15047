"""Plain FP64 reference of the initial-guess network (numpy).

TEST INFRASTRUCTURE ONLY: imported by the tests, never by the product package.

The network maps 33 features of an interface cell (the volume fractions of
its 3x3x3 lattice neighbourhood and 6 scale-free shape numbers) through two
hidden layers of 64 ReLU units to 4 outputs (a unit normal and the plane's
offset s = (d - d_min) / (d_max - d_min) in the cell's projection range),
trained by the mean squared error.  Storage and arithmetic points follow the
GPU form: inputs, weights and the hidden activations rounded to BF16 before
each product, products summed exactly here (FP32 on the GPU), biases and
outputs unrounded; the backward pass rounds each upstream gradient to BF16
before its products, as the GPU does.  Parameters are one flat float array:
W1 [33 x 64] (input-major), b1 [64], W2 [64 x 64], b2 [64], W3 [64 x 4], b3 [4].
"""
from __future__ import annotations

import numpy as np

N_IN, N_HID, N_OUT = 33, 64, 4
SHAPES = [(N_IN, N_HID), (N_HID,), (N_HID, N_HID), (N_HID,), (N_HID, N_OUT), (N_OUT,)]
N_PARAM = sum(int(np.prod(s)) for s in SHAPES)


def bf16(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isnan(f), np.nan, out)


def unpack(p):
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(np.asarray(p[o:o + n], np.float64).reshape(s))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(a, np.float64).reshape(-1) for a in parts])


def forward(p, X, quant: bool = True):
    """Returns (Y, cache) for features X [n x 33]; quant=False skips the BF16
    rounding (the plain real-valued network, for finite-difference checks)."""
    q = bf16 if quant else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X0 = q(X)
    Z1 = X0 @ q(W1) + b1
    H1 = q(np.maximum(Z1, 0.0))
    Z2 = H1 @ q(W2) + b2
    H2 = q(np.maximum(Z2, 0.0))
    Y = H2 @ q(W3) + b3
    return Y, (X0, Z1, H1, Z2, H2)


def loss(p, X, T, quant: bool = True):
    Y, _ = forward(p, X, quant)
    return float(((Y - T) ** 2).sum() / X.shape[0])


def backward(p, X, T, quant: bool = True):
    """(loss, gradient as a flat array) of the mean squared error."""
    q = bf16 if quant else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p)
    Y, (X0, Z1, H1, Z2, H2) = forward(p, X, quant)
    n = X.shape[0]
    dY = 2.0 * (Y - T) / n
    dYb = q(dY)
    gW3 = H2.T @ dYb
    gb3 = dY.sum(0)
    dZ2 = (dYb @ q(W3).T) * (Z2 > 0)
    dZ2b = q(dZ2)
    gW2 = H1.T @ dZ2b
    gb2 = dZ2.sum(0)
    dZ1 = (dZ2b @ q(W2).T) * (Z1 > 0)
    dZ1b = q(dZ1)
    gW1 = X0.T @ dZ1b
    gb1 = dZ1.sum(0)
    return float(((Y - T) ** 2).sum() / n), pack([gW1, gb1, gW2, gb2, gW3, gb3])

