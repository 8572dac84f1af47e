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


# ---------------------------------------------------------------------------
# Gradients at the rounding points of the tensor-core training pass, with a
# bound per entry. The training pass keeps BF16 copies of the three GEMM
# weight matrices, rounds every hidden activation to BF16 after its ReLU,
# rounds the head's dz = dy * w4 and each dh = dz W to BF16 before the ReLU
# mask, and accumulates every sum in FP32. The reference below takes the same
# rounding points in FP64 arithmetic. Its bound follows each value as an
# interval: an FP32 sum of K terms is off by at most 2 K 2^-24 times the sum
# of their magnitudes, upstream errors propagate through the magnitudes, and
# since round-to-nearest and ReLU are monotonic, a BF16 rounding of a value
# known to within e lies between the roundings of the interval's ends -- it is
# exactly the reference's unless the interval straddles a rounding boundary.
# ---------------------------------------------------------------------------
U32 = 2.0 ** -24


def _round_interval(z, ez, relu=False):
    f = (lambda v: np.maximum(v, 0.0)) if relu else (lambda v: v)  # noqa: E731
    r = bf16(f(z))
    lo, hi = bf16(f(z - ez)), bf16(f(z + ez))
    return r, np.maximum(hi - r, r - lo)


def _mask(v, ev, h, eh):
    """v masked by h > 0 (ReLU backward), where h is known to within eh."""
    on = h - eh > 0                      # surely positive on both sides
    off = (h == 0) & (eh == 0)           # surely zero
    unsure = ~on & ~off
    out = np.where(on, v, 0.0)
    err = np.where(on, ev, 0.0)
    out = np.where(unsure & (h > 0), v, out)
    err = np.where(unsure, np.abs(v) + ev, err)
    return out, err


def grads_bf16(params, x, t, acts=None):
    """Gradients of mean((y - t)^2) at the training pass's rounding points (BF16 weights, BF16
    activations and BF16 dz / dh; x taken as given), and an absolute bound per entry on how far an
    FP32-accumulating pass with those rounding points can be from them. `acts` (optional): the
    three BF16 hidden activations of the pass being checked, taken as exact -- then the bound
    covers the backward pass alone, with that pass's own ReLU masks. Returns (grads, bounds, loss)
    with grads and bounds in the parameter order w1, b1, w2, b2, w3, b3, w4, b4."""
    w1, b1, w2, b2, w3, b3, w4, b4 = [np.asarray(p, dtype=np.float64) for p in params]
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    W = [bf16(w1), bf16(w2), bf16(w3)]
    Bs = [b1, b2, b3]
    M = x.shape[0]
    a, ea = x, np.zeros_like(x)
    hs, ehs = [], []
    for l in range(3):
        if acts is not None:
            a, ea = np.asarray(acts[l], dtype=np.float64), np.zeros(acts[l].shape)
            assert np.array_equal(bf16(a), a), "activations must be BF16 values"
        else:
            K = a.shape[1]
            z = a @ W[l].T + Bs[l]
            ez = 2 * K * U32 * (np.abs(a) @ np.abs(W[l]).T + np.abs(Bs[l])) + ea @ np.abs(W[l]).T
            a, ea = _round_interval(z, ez, relu=True)
        hs.append(a)
        ehs.append(ea)
    h3, eh3 = hs[2], ehs[2]
    H = h3.shape[1]
    y = h3 @ w4 + b4[0]
    ey = 2 * H * U32 * (np.abs(h3) @ np.abs(w4) + abs(b4[0])) + eh3 @ np.abs(w4)
    dy = 2.0 * (y - t) / M
    edy = 2.0 * ey / M + 4 * U32 * np.abs(dy)
    loss = float(np.mean((y - t) ** 2))
    gw4 = h3.T @ dy
    egw4 = np.abs(h3).T @ edy + eh3.T @ np.abs(dy) + 2 * M * U32 * (np.abs(h3).T @ np.abs(dy))
    gb4 = np.array([dy.sum()])
    egb4 = np.array([edy.sum() + 2 * M * U32 * np.abs(dy).sum()])
    pre = np.outer(dy, w4)
    dz, edz = _round_interval(pre, np.outer(edy, np.abs(w4)) + U32 * np.abs(pre))
    dz, edz = _mask(dz, edz, h3, eh3)
    acts, eacts = [x, hs[0], hs[1]], [np.zeros_like(x), ehs[0], ehs[1]]
    gw, egw, gb, egb = [None] * 3, [None] * 3, [None] * 3, [None] * 3
    for l in (2, 1, 0):
        a, ea = acts[l], eacts[l]
        gw[l] = dz.T @ a
        egw[l] = np.abs(dz).T @ ea + edz.T @ np.abs(a) + 2 * M * U32 * (np.abs(dz).T @ np.abs(a))
        gb[l] = dz.sum(0)
        egb[l] = edz.sum(0) + 2 * M * U32 * np.abs(dz).sum(0)
        if l > 0:
            pre = dz @ W[l]
            epre = edz @ np.abs(W[l]) + 2 * H * U32 * (np.abs(dz) @ np.abs(W[l]))
            d, ed = _round_interval(pre, epre)
            dz, edz = _mask(d, ed, hs[l - 1], ehs[l - 1])
    grads = [gw[0], gb[0], gw[1], gb[1], gw[2], gb[2], gw4, gb4]
    bounds = [egw[0], egb[0], egw[1], egb[1], egw[2], egb[2], egw4, egb4]
    return grads, bounds, loss
