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
