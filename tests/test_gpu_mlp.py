"""Tensor-core GEMM and MLP kernels against plain FP64 references."""
import numpy as np
import pytest

from oracle import mlp_oracle as R

pytestmark = pytest.mark.gpu


def _bf16_tensor(a):
    import torch
    return torch.tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (128, 256, 64), (300, 200, 100), (257, 64, 256), (1000, 256, 256),
                                   (256, 48, 8), (130, 256, 40)])
def test_gemm_matches_fp64(M, N, K):
    from paper_1909_10286_gb300 import mlp
    import torch

    rng = np.random.default_rng(M * 7 + N * 3 + K)
    a = R.bf16(rng.standard_normal((M, K)))
    b = R.bf16(rng.standard_normal((N, K)))
    bias = rng.standard_normal(N).astype(np.float32)
    c = mlp.gemm_bf16(_bf16_tensor(a), _bf16_tensor(b), torch.tensor(bias).cuda(), relu=False).cpu().numpy()
    want = a @ b.T + bias
    # exact products of BF16 values, FP32 accumulation: error ~ K * 2^-24 * |terms|
    tol = 1e-5 * np.sqrt(K) * (np.abs(a) @ np.abs(b).T + np.abs(bias)) + 1e-6
    assert np.all(np.abs(c - want) <= tol), float(np.max(np.abs(c - want) / tol))
    r = mlp.gemm_bf16(_bf16_tensor(a), _bf16_tensor(b), torch.tensor(bias).cuda(), relu=True).cpu().numpy()
    assert np.all(np.abs(r - np.maximum(want, 0)) <= tol)


def _gpu_grads(params, x, t):
    """The library's gradients (bl_mlp_grads) and loss for parameters `params` on (x, t)."""
    from paper_1909_10286_gb300 import mlp
    import torch

    M, I = x.shape
    H = params[1].shape[0]
    net = mlp.MLP(I, H, max_batch=M, seed=3)
    net.set([np.asarray(q, np.float32) for q in params])
    loss = net.grads(_bf16_tensor(x), torch.tensor(t, dtype=torch.float32).cuda())
    g = [a.astype(np.float64) for a in net.get(grads=True)]
    y = net.forward(_bf16_tensor(x)).cpu().numpy()
    net.close()
    return g, loss, y


@pytest.mark.parametrize("M", [512, 4096])
def test_mlp_gradients_exact_on_a_dyadic_grid(M):
    """Every rounding point of the training pass is exact on the dyadic case (tests/mlp_cases.py):
    the forward, the loss and every entry of every gradient equal the plain FP64 backprop bit for
    bit. M = 4096 splits the weight-gradient products over 16 slices of the batch."""
    import mlp_cases as MC

    p, x, t = MC.dyadic_case(M=M)
    g_ref, loss_ref = R.grads([R.bf16(p[0]), p[1], R.bf16(p[2]), p[3], R.bf16(p[4]), p[5], p[6], p[7]], x, t)
    y_ref, _ = R.forward_bf16(p, x)
    g, loss, y = _gpu_grads(p, x, t)
    assert np.array_equal(y.astype(np.float64), y_ref)
    assert loss == loss_ref
    for k, (a, b) in enumerate(zip(g, g_ref)):
        assert np.array_equal(a, b), (k, int(np.sum(a != b)), float(np.max(np.abs(a - b))))


def test_mlp_gradients_within_the_bf16_bound():
    """Random values: every entry of every gradient lies within the bound of the FP64 reference at
    the training pass's rounding points (oracle/mlp_oracle.py, grads_bf16), given the pass's own
    BF16 activations -- computed here by the same tensor-core GEMM (bl_gemm_bf16) the training
    forward runs, and checked first against the forward's bound."""
    from paper_1909_10286_gb300 import mlp
    import mlp_cases as MC
    import torch

    p, x, t = MC.random_case()
    # the activations the training forward computes: BF16 GEMM + bias + ReLU, BF16 out
    a = _bf16_tensor(x)
    acts = []
    for l in range(3):
        a = mlp.gemm_bf16(a, _bf16_tensor(R.bf16(p[2 * l])), torch.tensor(p[2 * l + 1], dtype=torch.float32).cuda(),
                          relu=True, out_f32=False, out_bf16=True)
        acts.append(a.float().cpu().numpy().astype(np.float64))
    # each layer's activations within the forward bound of the layer below's (exact) GPU values
    prev = x
    for l in range(3):
        W = R.bf16(p[2 * l])
        z = prev @ W.T + p[2 * l + 1]
        ez = 2 * W.shape[1] * R.U32 * (np.abs(prev) @ np.abs(W).T + np.abs(p[2 * l + 1]))
        lo, hi = R.bf16(np.maximum(z - ez, 0)), R.bf16(np.maximum(z + ez, 0))
        assert np.all((acts[l] >= lo) & (acts[l] <= hi)), l
        prev = acts[l]
    g_ref, E, loss_ref = R.grads_bf16(p, x, t, acts=acts)
    g, loss, _ = _gpu_grads(p, x, t)
    assert loss == pytest.approx(loss_ref, rel=1e-5)
    names = ["dW1", "db1", "dW2", "db2", "dW3", "db3", "dw4", "db4"]
    for k in range(8):
        d = np.abs(g[k] - g_ref[k])
        assert np.all(d <= E[k]), (names[k], int(np.sum(d > E[k])), float(np.max(d / np.maximum(E[k], 1e-300))))


def test_mlp_training_reduces_loss():
    from paper_1909_10286_gb300 import mlp
    import torch

    M, I = 2048, 16
    rng = np.random.default_rng(2)
    x = rng.standard_normal((M, I))
    t = np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2] - np.abs(x[:, 3])
    net = mlp.MLP(I, 64, max_batch=M, seed=0)
    xt, tt = _bf16_tensor(x), torch.tensor(t, dtype=torch.float32).cuda()
    first = net.train_step(xt, tt, 3e-3)
    for _ in range(300):
        last = net.train_step(xt, tt, 3e-3)
    assert last < 0.25 * first, (first, last)
    net.close()


def _set_random(net, rng, I, H):
    params = [0.5 * rng.standard_normal((H, I)) / np.sqrt(I), 0.1 * rng.standard_normal(H),
              rng.standard_normal((H, H)) / np.sqrt(H), 0.1 * rng.standard_normal(H),
              rng.standard_normal((H, H)) / np.sqrt(H), 0.1 * rng.standard_normal(H),
              rng.standard_normal(H) / np.sqrt(H), np.array([0.3])]
    params = [p.astype(np.float32) for p in params]
    net.set(params)
    # the kernels multiply BF16 copies of the three layer weights
    return [R.bf16(params[0]), params[1], R.bf16(params[2]), params[3], R.bf16(params[4]), params[5], params[6],
            params[7]]


def _check_rows(y, ref, x_rows):
    y_ref, (_, _, h3) = R.forward_bf16(ref, x_rows)
    # FP32 accumulation in the tensor cores and the head; a hidden value whose FP32 sum
    # lands next to a BF16 rounding boundary may round one BF16 ulp (2^-8) the other way
    scale = np.abs(h3) @ np.abs(ref[6]) + abs(float(ref[7][0]))
    err = np.abs(y - y_ref)
    assert np.all(err <= 4e-3 * scale + 1e-6), float(np.max(err / (scale + 1e-30)))
    assert np.median(err / (scale + 1e-30)) < 1e-4


@pytest.mark.parametrize("M,I,H,max_batch", [(1000, 64, 256, 1024), (300, 60, 96, 512), (129, 256, 32, 256),
                                             (200, 16, 48, 256), (70000, 64, 256, 4096)])
def test_inference_forward_matches_bf16_hidden_reference(M, I, H, max_batch):
    """bl_mlp_forward: the fused three-layer kernel (hidden a multiple of 32; any M,
    ragged last tile, in_dim not a multiple of 16) and the layer-by-layer path
    (hidden 48) against the FP64 forward with BF16-rounded hidden layers."""
    from paper_1909_10286_gb300 import mlp

    rng = np.random.default_rng(M + I + H)
    net = mlp.MLP(I, H, max_batch=max_batch, seed=1)
    ref = _set_random(net, rng, I, H)
    x = R.bf16(rng.standard_normal((M, I)))
    y = net.forward(_bf16_tensor(x)).cpu().numpy()
    rows = np.arange(M) if M <= 4096 else np.unique(np.concatenate([rng.integers(0, M, 3000), np.arange(M - 200, M)]))
    _check_rows(y[rows], ref, x[rows])
    # new weights after a forward: the packed copy must follow them
    ref2 = _set_random(net, rng, I, H)
    y2 = net.forward(_bf16_tensor(x[:300])).cpu().numpy()
    _check_rows(y2, ref2, x[:300])
    net.close()


def test_inference_after_training_step_uses_updated_weights():
    from paper_1909_10286_gb300 import mlp
    import torch

    M, I, H = 512, 64, 256
    rng = np.random.default_rng(11)
    net = mlp.MLP(I, H, max_batch=M, seed=2)
    x = _bf16_tensor(R.bf16(rng.standard_normal((M, I))))
    y0 = net.forward(x).cpu().numpy()
    net.train_step(x, torch.zeros(M, dtype=torch.float32, device="cuda") + 5.0, 1e-2)
    p = net.get()
    ref = [R.bf16(p[0]), p[1], R.bf16(p[2]), p[3], R.bf16(p[4]), p[5], p[6], p[7]]
    y1 = net.forward(x).cpu().numpy()
    assert not np.allclose(y0, y1)
    _check_rows(y1, ref, x.float().cpu().numpy())
    net.close()


def _splitmix64(z):
    m = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def test_sampled_train_step_draws_the_documented_rows():
    """bl_mlp_train_step_sampled equals bl_mlp_train_step on the rows its documented SplitMix64 draw
    selects (computed here in Python), bit for bit, over two Adam steps; and the same seed repeats."""
    from paper_1909_10286_gb300 import mlp
    import torch

    rng = np.random.default_rng(4)
    n, I, H, batch, seed = 5003, 64, 64, 256, 12345
    X = _bf16_tensor(rng.standard_normal((n, I)))
    T = torch.tensor(rng.standard_normal(n), dtype=torch.float32).cuda()
    a = mlp.MLP(I, H, max_batch=batch, seed=7)
    b = mlp.MLP(I, H, max_batch=batch, seed=7)
    c = mlp.MLP(I, H, max_batch=batch, seed=7)
    for step in range(2):
        rows = [(_splitmix64((seed + ((step * batch + r) * 0x9E3779B97F4A7C15)) & ((1 << 64) - 1)) * n) >> 64
                for r in range(batch)]
        idx = torch.tensor(rows, dtype=torch.int64, device="cuda")
        la = a.train_step_sampled(X, T, batch, seed, 1e-3)
        lb = b.train_step(X[idx].contiguous(), T[idx].contiguous(), 1e-3)
        lc = c.train_step_sampled(X, T, batch, seed, 1e-3)
        # the loss is summed with atomics (order-dependent in the last bits); the weights are exact
        assert la == pytest.approx(lb, rel=1e-6) and lc == pytest.approx(la, rel=1e-6)
    for pa, pb, pc in zip(a.get(), b.get(), c.get()):
        assert np.array_equal(pa, pb) and np.array_equal(pa, pc)
    for net in (a, b, c):
        net.close()
