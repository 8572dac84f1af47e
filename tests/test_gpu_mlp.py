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


def test_mlp_forward_and_gradients_match_fp64_backprop():
    from paper_1909_10286_gb300 import mlp
    import torch

    M, I, H = 512, 64, 256
    net = mlp.MLP(I, H, max_batch=M, seed=3)
    rng = np.random.default_rng(1)
    params = net.get()
    params = [p.astype(np.float32) for p in params]
    params[1] = (0.1 * rng.standard_normal(H)).astype(np.float32)   # nonzero biases
    params[3] = (0.1 * rng.standard_normal(H)).astype(np.float32)
    params[7] = np.array([0.3], np.float32)
    net.set(params)
    x = R.bf16(rng.standard_normal((M, I)))
    t = rng.standard_normal(M)
    xt = _bf16_tensor(x)
    y = net.forward(xt).cpu().numpy()
    # the reference sees the same BF16 weights of the three GEMM layers
    ref_params = [R.bf16(params[0]), params[1], R.bf16(params[2]), params[3], R.bf16(params[4]), params[5], params[6],
                  params[7]]
    y_ref, _ = R.forward(ref_params, x)
    assert np.allclose(y, y_ref, rtol=3e-2, atol=3e-2 * np.std(y_ref))
    loss = net.grads(xt, torch.tensor(t, dtype=torch.float32).cuda())
    g = net.get(grads=True)
    g_ref, loss_ref = R.grads(ref_params, x, t)
    assert loss == pytest.approx(loss_ref, rel=2e-2)
    for k, (a, b) in enumerate(zip(g, g_ref)):
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        cos = float(np.dot(a.ravel(), b.ravel()) / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-30))
        assert rel < 5e-2 and cos > 0.998, (k, rel, cos)
    net.close()


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
