"""FP64 reference of the warm-start network's forward pass, loss and gradients (test
infrastructure; the network is an extension of the method, not a part of the paper).

Network: x (4) -> tanh(W1 x + b1) (H) -> tanh(W2 h1 + b2) (H) -> W3 h2 + b3 (1).
Loss: mean over rows of (y - t)^2.  Parameter vector order: W1 (H x 4, row-major), b1 (H),
W2 (H x H), b2 (H), W3 (1 x H), b3 (1).
"""
from __future__ import annotations

import numpy as np


def unpack(theta: np.ndarray, H: int, F: int = 4):
    o = 0
    W1 = theta[o:o + H * F].reshape(H, F); o += H * F
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + H].reshape(1, H); o += H
    b3 = theta[o:o + 1]; o += 1
    assert o == theta.size
    return W1, b1, W2, b2, W3, b3


def n_params(H: int, F: int = 4) -> int:
    return H * F + H + H * H + H + H + 1


def forward(theta: np.ndarray, X: np.ndarray, H: int):
    W1, b1, W2, b2, W3, b3 = unpack(theta, H, X.shape[1])
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    y = (h2 @ W3.T + b3)[:, 0]
    return y, (h1, h2)


def loss_and_grad(theta: np.ndarray, X: np.ndarray, t: np.ndarray, H: int):
    """Mean squared error and its gradient by the chain rule, layer by layer."""
    W1, b1, W2, b2, W3, b3 = unpack(theta, H, X.shape[1])
    y, (h1, h2) = forward(theta, X, H)
    n = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n                       # d loss / d y
    gW3 = dy @ h2                          # (H,)
    gb3 = np.array([dy.sum()])
    dh2 = np.outer(dy, W3[0]) * (1.0 - h2 * h2)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (1.0 - h1 * h1)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def adam_step(theta, m, v, g, it, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015) with bias correction; it counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** it)
    vh = v / (1 - b2 ** it)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to bfloat16 (round to nearest, ties to even) and back to FP32."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)
