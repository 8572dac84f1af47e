"""Inputs for the MLP gradient checks (no arithmetic of the method): a dyadic case in which
every FP32 sum of the training pass is exact, a random case, and an FP32 stand-in of the
training pass's arithmetic on the CPU (the rounding points of the tensor-core kernels, FP32
sums) used to pin the FP64 reference's bounds without a GPU."""
import numpy as np

from oracle import mlp_oracle as R


def dyadic_case(I=64, H=256, M=512, seed=0):
    """Weights, inputs and targets on small dyadic grids: x in {-1, 0, 1}; rows of W1 and W2 with
    three and of W3 with two nonzero entries +-1; biases in {-1/2, 0, 1/2} (layer 1) and
    {-1/4, 0, 1/4} (layers 2, 3); w4 in {-1/8, 0, 1/8}; b4 = 1/16; t = y - e with e in
    {-1/2, ..., 1/2} and M a power of two. Every hidden activation is then a BF16 value, every
    product and partial sum of the pass a multiple of a quantum q with sum |terms| < 2^24 q, so
    FP32 accumulation in any order is exact and the pass equals its FP64 restatement bit for bit."""
    assert M & (M - 1) == 0
    rng = np.random.default_rng(seed)

    def sparse(rows, cols, nnz):
        w = np.zeros((rows, cols))
        for j in range(rows):
            k = rng.choice(cols, nnz, replace=False)
            w[j, k] = rng.choice([-1.0, 1.0], nnz)
        return w

    w1, w2, w3 = sparse(H, I, 3), sparse(H, H, 3), sparse(H, H, 2)
    b1 = rng.choice([-0.5, 0.0, 0.5], H)
    b2 = rng.choice([-0.25, 0.0, 0.25], H)
    b3 = rng.choice([-0.25, 0.0, 0.25], H)
    w4 = rng.choice([-0.125, 0.0, 0.125], H)
    b4 = np.array([0.0625])
    params = [w1, b1, w2, b2, w3, b3, w4, b4]
    x = rng.choice([-1.0, 0.0, 1.0], (M, I))
    y, _ = R.forward_bf16(params, x)
    e = rng.choice([-0.5, -0.25, 0.0, 0.25, 0.5], M)
    t = y - e
    assert np.array_equal(t.astype(np.float32).astype(np.float64), t)
    return params, x, t


def random_case(I=64, H=256, M=512, seed=1):
    """He-uniform weights with nonzero biases, BF16 inputs, standard normal targets (FP32 values)."""
    rng = np.random.default_rng(seed)
    l1, l = np.sqrt(6 / I), np.sqrt(6 / H)
    params = [rng.uniform(-l1, l1, (H, I)), 0.1 * rng.standard_normal(H), rng.uniform(-l, l, (H, H)),
              0.1 * rng.standard_normal(H), rng.uniform(-l, l, (H, H)), 0.1 * rng.standard_normal(H),
              rng.uniform(-l, l, H), np.array([0.3])]
    params = [p.astype(np.float32).astype(np.float64) for p in params]
    x = R.bf16(rng.standard_normal((M, I)))
    t = rng.standard_normal(M).astype(np.float32).astype(np.float64)
    return params, x, t


def _bf32(v):
    return R.bf16(v).astype(np.float32)


def fp32_pass(params, x, t):
    """The training pass's arithmetic on the CPU: BF16 copies of W1..W3, hidden activations rounded
    to BF16 after the ReLU, FP32 sums, dy = 2 (y - t) / M, dz = BF16(dy w4) and dh = BF16(dz W)
    masked by the ReLU. Returns (activations, gradients) in the parameter order."""
    w1, b1, w2, b2, w3, b3, w4, b4 = [np.asarray(p, np.float32) for p in params]
    W = [_bf32(w1), _bf32(w2), _bf32(w3)]
    Bs = [b1, b2, b3]
    M = x.shape[0]
    a = np.asarray(x, np.float32)
    hs = []
    for l in range(3):
        a = _bf32(np.maximum(a @ W[l].T + Bs[l], np.float32(0)))
        hs.append(a)
    y = hs[2] @ w4 + b4[0]
    dy = (np.float32(2) * (y - np.asarray(t, np.float32)) / np.float32(M)).astype(np.float32)
    gw4 = hs[2].T @ dy
    gb4 = np.array([dy.sum(dtype=np.float32)], np.float32)
    dz = _bf32(np.outer(dy, w4)) * (hs[2] > 0)
    acts = [np.asarray(x, np.float32), hs[0], hs[1]]
    gw, gb = [None] * 3, [None] * 3
    for l in (2, 1, 0):
        gw[l] = dz.T @ acts[l]
        gb[l] = dz.sum(0, dtype=np.float32)
        if l > 0:
            dz = _bf32(dz @ W[l]) * (hs[l - 1] > 0)
    return hs, [gw[0], gb[0], gw[1], gb[1], gw[2], gb[2], gw4, gb4]
