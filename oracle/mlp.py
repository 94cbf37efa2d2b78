"""CPU FP64 oracle of the warm-start network — test infrastructure only.

The network maps n_in features -> H -> H -> n_out with ReLU after the two
hidden layers:  H1 = relu(X W1^T + b1),  H2 = relu(H1 W2^T + b2),
Y = H2 W3^T + b3.  Its training loss is the weighted mean squared error
L = sum_{b,o} w_o (Y - T)^2 / (2 batch), and its gradients follow by the chain
rule (back-propagation):

    dY = w (Y - T) / batch
    dW3 = dY^T H2,   db3 = sum_b dY,   dZ2 = (dY W3) * [H2 > 0]
    dW2 = dZ2^T H1,  db2 = sum_b dZ2,  dZ1 = (dZ2 W2) * [H1 > 0]
    dW1 = dZ1^T X,   db1 = sum_b dZ1

The GPU kernels round every GEMM operand to bf16 (nearest, ties to even)
and accumulate in fp32; with ``bf16=True`` this oracle rounds the same
operands at the same points (from the float32 values the kernels hold) and
accumulates in float64, so the two differ only by the fp32 accumulation.
With ``bf16=False`` it is the plain FP64 network (used for the finite-
difference pin).  Parameters are packed as W1 (H x n_in), b1, W2 (H x H), b2,
W3 (n_out x H), b3, all row-major.

Only tests/ may import this module; it shares no code with the library.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """float32 values rounded to the nearest bf16 (ties to even), returned as
    float64.  A bf16 keeps the top 16 bits of the float32 pattern."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p, n_in: int, H: int, n_out: int):
    p = np.asarray(p, dtype=np.float64)
    sizes = [H * n_in, H, H * H, H, n_out * H, n_out]
    parts, o = [], 0
    for sz in sizes:
        parts.append(p[o:o + sz])
        o += sz
    assert o == p.size, (o, p.size)
    W1, b1, W2, b2, W3, b3 = parts
    return W1.reshape(H, n_in), b1, W2.reshape(H, H), b2, W3.reshape(n_out, H), b3


def _op(a, bf16: bool):
    return bf16_round(a) if bf16 else np.asarray(a, dtype=np.float64)


def forward(p, X, n_in: int, H: int, n_out: int, bf16: bool = True):
    """Y and the hidden activations (H1, H2) of a batch X (batch x n_in)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, H, n_out)
    st = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if bf16 else (lambda a: a)
    H1 = st(np.maximum(_op(X, bf16) @ _op(W1, bf16).T + b1, 0.0))
    H2 = st(np.maximum(_op(H1, bf16) @ _op(W2, bf16).T + b2, 0.0))
    Y = st(_op(H2, bf16) @ _op(W3, bf16).T + b3)
    return Y, H1, H2


def loss_and_grad(p, X, T, n_in: int, H: int, n_out: int, out_weights=None, bf16: bool = True):
    """(loss, gradient packed like p) of the weighted mean squared error."""
    W1, b1, W2, b2, W3, b3 = unpack(p, n_in, H, n_out)
    batch = X.shape[0]
    w = np.ones(n_out) if out_weights is None else np.asarray(out_weights, dtype=np.float64)
    Y, H1, H2 = forward(p, X, n_in, H, n_out, bf16)
    D = Y - np.asarray(T, dtype=np.float64)
    loss = float(np.sum(w * D * D) / (2.0 * batch))
    st = (lambda a: np.asarray(a, np.float32).astype(np.float64)) if bf16 else (lambda a: a)
    dY = st(w * D / batch)
    gW3 = _op(dY, bf16).T @ _op(H2, bf16)
    gb3 = dY.sum(axis=0)
    dZ2 = st((_op(dY, bf16) @ _op(W3, bf16)) * (H2 > 0))
    gW2 = _op(dZ2, bf16).T @ _op(H1, bf16)
    gb2 = dZ2.sum(axis=0)
    dZ1 = st((_op(dZ2, bf16) @ _op(W2, bf16)) * (H1 > 0))
    gW1 = _op(dZ1, bf16).T @ _op(X, bf16)
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam(p, m, v, g, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One bias-corrected Adam step (Kingma and Ba 2015); returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1**step)
    vh = v / (1 - beta2**step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
