"""FP64 CPU reference of the learned ranker's MLP (in -> H -> H -> H -> 1,
ReLU, mean squared error): forward pass and gradients by plain backprop.

TEST INFRASTRUCTURE ONLY: used by the tests to check the tensor-core forward
and backward kernels. It imports nothing from the product package.
"""
import numpy as np


def bf16(x):
    """Round float values to bfloat16 (round to nearest even), returned as float64."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(params, x):
    w1, b1, w2, b2, w3, b3, w4, b4 = [np.asarray(p, dtype=np.float64) for p in params]
    z1 = x @ w1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ w2.T + b2
    h2 = np.maximum(z2, 0.0)
    z3 = h2 @ w3.T + b3
    h3 = np.maximum(z3, 0.0)
    y = h3 @ w4 + b4[0]
    return y, (h1, h2, h3)


def forward_bf16(params, x):
    """forward() with every hidden activation rounded to bfloat16 after its
    ReLU, as the tensor-core path stores them between layers (the products
    and sums themselves stay exact in FP64)."""
    w1, b1, w2, b2, w3, b3, w4, b4 = [np.asarray(p, dtype=np.float64) for p in params]
    h1 = bf16(np.maximum(x @ w1.T + b1, 0.0))
    h2 = bf16(np.maximum(h1 @ w2.T + b2, 0.0))
    h3 = bf16(np.maximum(h2 @ w3.T + b3, 0.0))
    return h3 @ w4 + b4[0], (h1, h2, h3)


def grads(params, x, t):
    """Gradients of mean((y - t)^2) with respect to every parameter."""
    w1, b1, w2, b2, w3, b3, w4, b4 = [np.asarray(p, dtype=np.float64) for p in params]
    y, (h1, h2, h3) = forward(params, x)
    M = x.shape[0]
    dy = 2.0 * (y - t) / M
    gw4 = h3.T @ dy
    gb4 = np.array([dy.sum()])
    dz3 = np.outer(dy, w4) * (h3 > 0)
    gw3 = dz3.T @ h2
    gb3 = dz3.sum(0)
    dz2 = (dz3 @ w3) * (h2 > 0)
    gw2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ w2) * (h1 > 0)
    gw1 = dz1.T @ x
    gb1 = dz1.sum(0)
    loss = float(np.mean((y - t) ** 2))
    return [gw1, gb1, gw2, gb2, gw3, gb3, gw4, gb4], loss
