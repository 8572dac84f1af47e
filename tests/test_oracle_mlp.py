"""Pins of the FP64 MLP reference used to check the tensor-core kernels:
bfloat16 rounding on known values, a hand-computed network, gradients against
central finite differences, and the BF16-hidden forward against the plain one."""
import numpy as np
import pytest

from oracle import mlp_oracle as R


def test_bf16_rounding_known_values():
    # bfloat16 keeps 8 significand bits (7 stored): spacing 2^-7 just above 1
    assert R.bf16(1.0) == 1.0
    assert R.bf16(1.0 + 2.0 ** -7) == 1.0 + 2.0 ** -7
    assert R.bf16(1.0 + 2.0 ** -8) == 1.0                     # tie -> even significand
    assert R.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2 * 2.0 ** -7  # tie -> even (rounds up)
    assert R.bf16(1.0 + 2.0 ** -8 + 2.0 ** -12) == 1.0 + 2.0 ** -7
    assert R.bf16(-3.14159265) == -3.140625
    assert R.bf16(0.0) == 0.0 and R.bf16(-0.0) == 0.0
    assert R.bf16(65504.0) == 65536.0
    x = np.random.default_rng(0).standard_normal(1000)
    r = R.bf16(x)
    assert np.all(np.abs(r - x) <= np.abs(x) * 2.0 ** -8 * (1 + 1e-12))   # half an ulp
    assert np.array_equal(R.bf16(r), r)                                  # idempotent


def _params(rng, I, H, scale=1.0):
    return [scale * rng.standard_normal((H, I)), 0.1 * rng.standard_normal(H),
            scale * rng.standard_normal((H, H)) / np.sqrt(H), 0.1 * rng.standard_normal(H),
            scale * rng.standard_normal((H, H)) / np.sqrt(H), 0.1 * rng.standard_normal(H),
            rng.standard_normal(H), np.array([0.2])]


def test_forward_hand_computed():
    # H = 1, I = 2: y = w4 * relu(w3 * relu(w2 * relu(w1 . x + b1) + b2) + b3) + b4
    p = [np.array([[2.0, -1.0]]), np.array([0.5]), np.array([[3.0]]), np.array([-1.0]), np.array([[-2.0]]),
         np.array([10.0]), np.array([0.25]), np.array([1.0])]
    x = np.array([[1.0, 1.0], [0.0, 3.0]])
    # row 0: z1 = 1.5 -> 1.5; z2 = 3.5; z3 = 3 -> y = 1.75 ; row 1: z1 = -2.5 -> 0; z2 = -1 -> 0; z3 = 10 -> y = 3.5
    y, (h1, h2, h3) = R.forward(p, x)
    assert np.allclose(y, [1.75, 3.5], rtol=0, atol=1e-15)
    assert np.allclose(h1[:, 0], [1.5, 0.0]) and np.allclose(h2[:, 0], [3.5, 0.0]) and np.allclose(h3[:, 0], [3.0, 10.0])


def test_grads_match_central_differences():
    rng = np.random.default_rng(5)
    I, H, M = 3, 4, 6
    p = _params(rng, I, H)
    x = rng.standard_normal((M, I))
    t = rng.standard_normal(M)
    g, loss = R.grads(p, x, t)
    assert loss == pytest.approx(np.mean((R.forward(p, x)[0] - t) ** 2), rel=1e-14)
    h = 1e-6
    for k in range(len(p)):
        num = np.zeros_like(p[k], dtype=np.float64)
        for idx in np.ndindex(p[k].shape):
            pp = [q.copy() for q in p]
            pm = [q.copy() for q in p]
            pp[k][idx] += h
            pm[k][idx] -= h
            num[idx] = (np.mean((R.forward(pp, x)[0] - t) ** 2) - np.mean((R.forward(pm, x)[0] - t) ** 2)) / (2 * h)
        assert np.allclose(g[k], num, rtol=1e-5, atol=1e-8), k


def test_forward_bf16_rounds_only_the_hidden_layers():
    # small integers and halves are exact in bfloat16: rounding the hidden values changes nothing
    rng = np.random.default_rng(7)
    I, H, M = 4, 8, 10
    p = [rng.integers(-2, 3, (H, I)).astype(float), rng.integers(-2, 3, H) / 2.0,
         rng.integers(-1, 2, (H, H)).astype(float), rng.integers(-2, 3, H) / 2.0,
         rng.integers(-1, 2, (H, H)).astype(float), rng.integers(-2, 3, H) / 2.0,
         rng.integers(-3, 4, H).astype(float), np.array([1.5])]
    x = rng.integers(-3, 4, (M, I)).astype(float)
    y, hs = R.forward(p, x)
    yb, hb = R.forward_bf16(p, x)
    assert np.all(np.abs(np.concatenate([h.ravel() for h in hs])) < 256)   # all exactly representable
    assert np.array_equal(y, yb)
    # generic values: the hidden layers are the rounded ones, the output is not rounded
    p2 = _params(rng, I, H)
    x2 = rng.standard_normal((M, I))
    y2, _ = R.forward(p2, x2)
    yb2, (h1, h2, h3) = R.forward_bf16(p2, x2)
    assert all(np.array_equal(R.bf16(h), h) for h in (h1, h2, h3))
    assert not np.array_equal(y2, yb2) and np.allclose(y2, yb2, rtol=0.05, atol=0.05)
    assert np.array_equal(h1, R.bf16(np.maximum(x2 @ p2[0].T + p2[1], 0)))


def test_dyadic_case_is_exact():
    """On the dyadic case every rounding point of the training pass is exact: the BF16-point
    reference equals the plain FP64 backprop (pinned above by central differences) and an FP32
    pass in numpy's summation order, bit for bit -- so the GPU's gradients must too."""
    import mlp_cases as MC

    for M in (512, 4096):
        p, x, t = MC.dyadic_case(M=M)
        g, _, loss = R.grads_bf16(p, x, t)
        plain = [R.bf16(p[0]), p[1], R.bf16(p[2]), p[3], R.bf16(p[4]), p[5], p[6], p[7]]
        gp, lp = R.grads(plain, x, t)
        hs, g32 = MC.fp32_pass(p, x, t)
        assert loss == lp
        for k in range(8):
            assert np.array_equal(g[k], gp[k]), k
            assert np.array_equal(g32[k].astype(np.float64), g[k]), k
            assert np.count_nonzero(g[k]) >= 0.4 * g[k].size, k   # not a trivially zero gradient
        _, hr = R.forward_bf16(p, x)
        assert all(np.array_equal(a.astype(np.float64), b) for a, b in zip(hs, hr))


def test_bf16_bound_covers_an_fp32_pass():
    """The per-entry bound of grads_bf16, given the activations of the pass it checks, covers an
    FP32 pass with the training kernels' rounding points on random values, and is tight for the
    layers next to the head (below 1 % of the entry for most of them)."""
    import mlp_cases as MC

    p, x, t = MC.random_case()
    hs, g32 = MC.fp32_pass(p, x, t)
    g, E, _ = R.grads_bf16(p, x, t, acts=hs)
    for k in range(8):
        assert np.all(np.abs(g32[k] - g[k]) <= E[k]), k
    for k in (4, 5, 6, 7):
        nz = g[k] != 0
        assert np.median(E[k][nz] / np.abs(g[k][nz])) < 1e-2, k


def test_bf16_bound_catches_planted_mistakes():
    """Mistakes planted in the reference's gradients on the CPU -- a row of dW3 with the wrong sign,
    three entries of db3 5 % off, one unit's db2 zeroed, dW2 scaled by 2 -- fall outside the bound
    against a correct FP32 pass."""
    import mlp_cases as MC

    p, x, t = MC.random_case()
    hs, g32 = MC.fp32_pass(p, x, t)
    g, E, _ = R.grads_bf16(p, x, t, acts=hs)

    def outside(k, gm):
        return np.abs(g32[k] - gm) > E[k]

    row = int(np.argmax(np.abs(g[4]).sum(1)))
    gm = g[4].copy(); gm[row] *= -1
    assert outside(4, gm)[row].mean() > 0.9
    gm = g[5].copy(); j = np.argsort(-np.abs(g[5]))[:3]; gm[j] *= 1.05
    assert outside(5, gm)[j].all()
    gm = g[3].copy(); u = int(np.argmax(np.abs(g[3]))); gm[u] = 0.0
    assert outside(3, gm)[u]
    assert outside(2, 2 * g[2]).mean() > 0.5
