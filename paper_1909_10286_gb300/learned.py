"""Learned move proposal: data collection, training and evaluation of the MLP
ranker (an extension; the paper's Step 8 draws moves uniformly).

The network predicts, from a move's features (bl_features), the exact change
of the plan cost the move causes, in percent of the base plan's cost. Training
tuples come from the plain search itself: at every logged iteration a sample
of that iteration's candidates is featurised and scored exactly
(bl_score_candidates). Infeasible candidates and those the completion-time gate
discards are given the clipped target CLIP_HI, so they rank last. Every step
runs in the library's kernels; this module only sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import biolog
from .mlp import MLP

NFEAT = 64
CLIP_LO, CLIP_HI = -2.0, 0.2


def targets(cost, base_cost) -> np.ndarray:
    """Percent cost change of each candidate against its base plan, clipped."""
    cost = np.asarray(cost, dtype=np.float64)
    d = np.full(cost.shape, CLIP_HI)
    ok = np.isfinite(cost) & np.isfinite(base_cost)
    d[ok] = np.clip(100.0 * (cost[ok] - base_cost) / base_cost, CLIP_LO, CLIP_HI)
    return d.astype(np.float32)


def collect(instances, iters: int, sample: int, seed: int = 100, n_cand: int | None = None, eps: float = 0.5,
            stride: int = 1):
    """(X [N x 64] bf16 CUDA tensor, T [N] float32 CUDA tensor) from plain searches on `instances`: the
    features and exact targets of `sample` candidates at `iters` points of each search, `stride`
    iterations apart (a stride above 1 reaches the later, slower phase of the search)."""
    import torch

    xs, ts = [], []
    for k, inst in enumerate(instances):
        S = biolog.Search([inst], biolog.make_params(n_cand=n_cand or sample, eps=eps, seed=seed + k, gate=1))
        feat = torch.empty((sample, NFEAT), dtype=torch.bfloat16, device="cuda")
        bc = torch.empty(1, dtype=torch.float32, device="cuda")
        for _ in range(iters):
            st = S.get_state()
            if not np.isfinite(st["cstar"]):
                S.search_step(1)
                continue
            S.features(0, st["iter"], 0, sample, feat, bc)
            cost = S.score_candidates(0, st["iter"], st["tmaxstar"], 0, sample)["cost"]
            torch.cuda.synchronize()
            xs.append(feat.clone())
            ts.append(torch.tensor(targets(cost, float(bc.item())), device="cuda"))
            S.search_step(stride)
        S.close()
    return torch.cat(xs), torch.cat(ts)


def train(X, T, hidden: int = 256, steps: int = 2000, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          stream=None, max_batch: int = 1 << 18, log_every: int = 0):
    """Adam on mean squared error over random minibatches; returns (MLP, losses)."""
    net = MLP(NFEAT, hidden, max_batch=max(batch, max_batch), seed=seed, stream=stream)
    losses = []
    X, T = X.contiguous(), T.contiguous()
    for s in range(steps):
        rate = lr * (0.1 ** (s / max(steps, 1)))   # geometric decay to lr/10
        # the library draws the minibatch (uniform rows, with replacement) and takes the Adam step
        losses.append(net.train_step_sampled(X, T, batch, seed, rate))
        if log_every and s % log_every == 0:
            print(f"step {s}: loss {losses[-1]:.4f}")
    return net, losses


def ranking_quality(net, X, T, top_true: float = 0.01, top_pred: float = 0.10) -> dict:
    """How well predictions rank moves: Spearman correlation with the exact
    targets, and the share of the truly best `top_true` moves found among the
    best `top_pred` predicted (a random ranking finds `top_pred` of them)."""
    import torch

    y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    for i in range(0, X.shape[0], net.max_batch):
        j = min(X.shape[0], i + net.max_batch)
        net.forward(X[i:j].contiguous(), y[i:j])
    torch.cuda.synchronize()
    yp, t = y.cpu().numpy().astype(np.float64), T.cpu().numpy().astype(np.float64)
    rp = np.argsort(np.argsort(yp))
    rt = np.argsort(np.argsort(t + 1e-9 * np.arange(len(t))))
    spearman = float(np.corrcoef(rp, rt)[0, 1])
    n = len(t)
    best_true = set(np.argsort(t, kind="stable")[: max(1, int(top_true * n))].tolist())
    best_pred = set(np.argsort(yp, kind="stable")[: max(1, int(top_pred * n))].tolist())
    recall = len(best_true & best_pred) / len(best_true)
    return {"spearman": spearman, "recall": recall, "random_recall": top_pred, "n": n}
