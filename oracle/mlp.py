"""Pair-correction network of the learned coarse level -- oracle side.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The learned coarse level maps the geometry of a close body pair to a 6x6
rigid-body pair-mobility correction with a small multilayer perceptron
6 -> 128 -> 128 -> 128 -> 36 (tanh on the hidden layers, linear output).  The
network is trained on two-body mobility solves with the squared-error loss and
the Adam update (Kingma & Ba, "Adam: a method for stochastic optimization",
ICLR 2015, Algorithm 1).  The paper has no network; this follows the learned
preconditioner of the hot-path specification.

Numerics mirrored from the GPU kernels: weights and every matrix-product
operand are rounded to bfloat16 (round to nearest even) before the product;
products are summed exactly here (float64), in FP32 on the GPU.  Biases,
activations, the loss and the optimizer state are float64 here, FP32 there.

Parameter vector layout (float, 38564 entries): for l = 1..4, W_l [n_l][n_{l-1}]
row-major then b_l [n_l], with widths n = (6, 128, 128, 128, 36).

* ``bf16``       round a float array to the nearest bfloat16 (ties to even)
* ``unpack``     split the parameter vector into (W_l, b_l)
* ``forward``    network output and the hidden activations
* ``loss_grad``  loss (1 / (B 36)) sum (y - t)^2 and its gradient by back-propagation
* ``adam``       one Adam step

Parity: pinned by central finite differences of the loss (with rounding off,
float64), which checks the back-propagation; by the Adam first step, which
moves every parameter by lr g / (|g| + eps) exactly; and by a network whose
layers reduce to a known affine map.
"""
from __future__ import annotations

import numpy as np

WIDTHS = (6, 128, 128, 128, 36)


def n_params(widths=WIDTHS) -> int:
    return sum(widths[i + 1] * widths[i] + widths[i + 1] for i in range(len(widths) - 1))


def bf16(a: np.ndarray) -> np.ndarray:
    """Nearest bfloat16 value (ties to even) of each element, returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def unpack(theta: np.ndarray, widths=WIDTHS):
    layers, o = [], 0
    for i in range(len(widths) - 1):
        n_in, n_out = widths[i], widths[i + 1]
        W = np.asarray(theta[o:o + n_out * n_in], dtype=np.float64).reshape(n_out, n_in)
        o += n_out * n_in
        b = np.asarray(theta[o:o + n_out], dtype=np.float64)
        o += n_out
        layers.append((W, b))
    return layers


def _r(a, rounding):
    return bf16(a) if rounding else np.asarray(a, dtype=np.float64)


def forward(theta: np.ndarray, X: np.ndarray, rounding: bool = True):
    """Output [B, 36] and the list of layer inputs (X, h1, h2, h3)."""
    layers = unpack(theta)
    acts = [np.asarray(X, dtype=np.float64)]
    h = acts[0]
    for l, (W, b) in enumerate(layers):
        z = _r(h, rounding) @ _r(W, rounding).T + b
        if l < len(layers) - 1:
            h = np.tanh(z)
            acts.append(h)
        else:
            h = z
    return h, acts


def loss_grad(theta: np.ndarray, X: np.ndarray, T: np.ndarray, rounding: bool = True):
    """(loss, gradient) of the mean squared error over batch and outputs."""
    layers = unpack(theta)
    Y, acts = forward(theta, X, rounding)
    B, n_out = Y.shape
    loss = float(np.sum((Y - T) ** 2) / (B * n_out))
    dz = 2.0 * (Y - T) / (B * n_out)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        a = acts[l]
        gW = _r(dz, rounding).T @ _r(a, rounding)
        gb = dz.sum(axis=0)
        grads[l] = (gW, gb)
        if l > 0:
            dh = _r(dz, rounding) @ _r(W, rounding)
            dz = dh * (1.0 - a * a)  # tanh'(z) = 1 - tanh(z)^2
    g = np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])
    return loss, g


def adam(theta, m, v, g, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
