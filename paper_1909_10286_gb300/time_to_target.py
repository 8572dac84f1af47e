"""Time to reach within 1 % of the best cost: plain search against the batched
and the learned-plus-batched forms, on the same GPU and instances.

For each instance, C_ref is the best C* of a long plain search, 10x the
configured iteration budget, with all instances in one handle. Each form then
runs from the initial plan. The C* trajectory comes from a fresh handle, and it
is deterministic: moves come from a counter-based generator and the ranker is
fixed. The device time per iteration is measured with CUDA events on a
separate, warmed-up handle of the same shape. An instance's time to target is
the number of iterations until C* <= (1 + tol) * C_ref, times that per-iteration
time. Setup (plan init, graph build, ranker training) is reported but not
counted.

Forms:
  plain          one instance per handle, n candidates per iteration (the paper's loop)
  batched        all instances in one handle (one launch per iteration), n_batched each
  learned_batched  all instances in one handle; per instance a Philox pool of `pool`
                 moves is ranked by the MLP, and about `keep` of them plus a random
                 fraction are scored exactly
"""
from __future__ import annotations

import time

import numpy as np

from . import biolog, instances as I, learned


def _per_iter_ms(insts, params, iters, net=None, pool=0, keep=0, rf=0.0):
    import torch

    S = biolog.Search(insts, params)
    netS = net.copy(stream=S.stream, max_batch=pool * len(insts)) if net is not None else None
    step = (lambda k: S.search_step_learned(netS, k, pool, keep, rf)) if netS else (lambda k: S.search_step(k))
    step(3)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(S.stream)
    step(iters)
    b.record(S.stream)
    b.synchronize()
    ms = a.elapsed_time(b) / iters
    if netS is not None:
        netS.close()
    S.close()
    return ms


def _trajectories(insts, params, iters, net=None, pool=0, keep=0, rf=0.0):
    S = biolog.Search(insts, params)
    netS = net.copy(stream=S.stream, max_batch=pool * len(insts)) if net is not None else None
    c0 = [S.get_state(inst=k)["cstar"] for k in range(len(insts))]
    if netS is not None:
        S.search_step_learned(netS, iters, pool, keep, rf)
    else:
        S.search_step(iters)
    tr = [np.concatenate([[c0[k]], S.get_log(0, iters, inst=k)["cstar"].astype(np.float64)])
          for k in range(len(insts))]
    if netS is not None:
        netS.close()
    S.close()
    return tr   # tr[k][j] = C* after j iterations


def _final_best(insts, params, iters):
    """C* of every instance after `iters` iterations (C* never increases)."""
    S = biolog.Search(insts, params)
    S.search_step(iters)
    c = np.array([S.get_state(inst=k)["cstar"] for k in range(len(insts))], dtype=np.float64)
    S.close()
    return c


def _iters_to(tr, target):
    hit = np.nonzero(tr <= target)[0]
    return int(hit[0]) if len(hit) else None


def study(workload: str = "paper", seeds=range(10), n: int = 1 << 20, iters: int = 300, budget: int = 1000,
          n_batched: int = 1 << 16, pool: int = 1 << 16, keep: int = 7373, rand_frac: float = 0.014,
          train_seeds=range(100, 110), train_iters: int = 25, train_sample: int = 8192, train_steps: int = 1500,
          tol: float = 0.01, eps: float = 0.5, seed_offset: int = 1000, time_iters: int = 30,
          ref_n: int | None = None) -> dict:
    """Runs the study; returns a JSON-able dict (times in ms)."""
    insts = I.make_batch(workload, seeds)
    kw = dict(eps=eps, gate=1)
    t0 = time.time()
    # C_ref: a long plain run, 10x the configured budget
    ref_n = ref_n or n
    c_ref = _final_best(insts, biolog.make_params(n_cand=ref_n, seed=seed_offset, **kw), 10 * budget)
    t_ref = time.time() - t0

    forms = {}
    # plain: one handle per instance, the paper's search seed (instance seed + 1000)
    ms_plain = _per_iter_ms(insts[:1], biolog.make_params(n_cand=n, seed=seed_offset, **kw), time_iters)
    its = []
    for k, (s, inst) in enumerate(zip(seeds, insts)):
        tr = _trajectories([inst], biolog.make_params(n_cand=n, seed=seed_offset + int(s), **kw), iters)[0]
        its.append(_iters_to(tr, (1 + tol) * c_ref[k]))
    forms["plain"] = dict(n_cand=n, ms_per_iter=ms_plain, iters=its)

    # batched: all instances in one handle
    pb = biolog.make_params(n_cand=n_batched, seed=seed_offset, **kw)
    ms_b = _per_iter_ms(insts, pb, time_iters)
    trs = _trajectories(insts, pb, iters)
    forms["batched"] = dict(n_cand=n_batched, ms_per_iter=ms_b,
                            iters=[_iters_to(t, (1 + tol) * c) for t, c in zip(trs, c_ref)])

    # learned + batched: ranker trained on plain searches of other instances
    t1 = time.time()
    X, T = learned.collect(I.make_batch(workload, train_seeds), iters=train_iters, sample=train_sample)
    net, losses = learned.train(X, T, hidden=256, steps=train_steps, batch=4096, lr=1e-3,
                                max_batch=pool * len(insts))
    t_train = time.time() - t1
    pl = biolog.make_params(n_cand=pool, seed=seed_offset, **kw)
    ms_l = _per_iter_ms(insts, pl, time_iters, net, pool, keep, rand_frac)
    trs = _trajectories(insts, pl, iters, net, pool, keep, rand_frac)
    forms["learned_batched"] = dict(pool=pool, keep=keep, rand_frac=rand_frac, ms_per_iter=ms_l,
                                    iters=[_iters_to(t, (1 + tol) * c) for t, c in zip(trs, c_ref)],
                                    train_tuples=int(X.shape[0]), train_s=round(t_train, 1),
                                    train_loss_first_last=[float(np.mean(losses[:50])), float(np.mean(losses[-50:]))])
    net.close()

    for f in forms.values():
        times = [i * f["ms_per_iter"] for i in f["iters"] if i is not None]
        f["reached"] = len(times)
        f["median_ms"] = float(np.median(times)) if len(times) == len(insts) else None
        f["median_ms_reached"] = float(np.median(times)) if times else None
        # every instance solved: one after another for plain, concurrently for the batched forms
        f["all_instances_ms"] = (float(np.sum(times)) if f is forms["plain"] else float(np.max(times))) \
            if len(times) == len(insts) else None
    return dict(workload=workload, seeds=[int(s) for s in seeds], tol=tol, iters_per_form=iters,
                c_ref=[float(c) for c in c_ref], c_ref_run=dict(n_cand=ref_n, iters=10 * budget,
                                                                s=round(t_ref, 1)),
                forms=forms)


def _wall_to_target(S, targets, max_iters, step):
    """Host wall time, through the API, until each instance's C* is within its target: one iteration per
    call, then every instance's C* read back in one transfer (bl_get_states). Returns (ms per instance or
    None, iterations per instance or None, total iterations run, total ms)."""
    n_inst = len(targets)
    reached_ms = [None] * n_inst
    reached_it = [None] * n_inst
    states = S.get_states()
    for k in range(n_inst):
        if states[k]["cstar"] <= targets[k]:
            reached_ms[k], reached_it[k] = 0.0, 0
    t0 = time.perf_counter()
    it = 0
    while it < max_iters and any(r is None for r in reached_ms):
        step(1)
        it += 1
        S.get_states(states)
        for k in range(n_inst):
            if reached_ms[k] is None and float(states[k]["cstar"]) <= targets[k]:
                reached_ms[k] = (time.perf_counter() - t0) * 1e3
                reached_it[k] = it
    return reached_ms, reached_it, it, (time.perf_counter() - t0) * 1e3


def study_wall(workload: str = "large", seeds=range(5), n: int = 1 << 20, n_batched: int = 1 << 16,
               max_iters: int = 400, ref_iters: int = 4000, ref_n: int = 1 << 16, pool: int = 1 << 18,
               keep: int = 2359, rand_frac: float = 0.001, train_seeds=range(100, 104), train_iters: int = 30,
               train_sample: int = 8192, train_steps: int = 1500, tol: float = 0.01, eps: float = 0.5,
               seed_offset: int = 1000, k_values=(1, 2), forms=None, train_stride: int = 1) -> dict:
    """Time to within `tol` of the best cost, measured as host wall time through the API (every
    iteration a bl_search_step call and one read of every instance's C*), from handles already set up; set-up and the
    ranker's training are reported beside it, not counted. C_ref per instance is the best C* of a
    plain batched run of ref_iters iterations of ref_n candidates. Forms: plain (one handle per
    instance, run one after the other) and batched (all instances in one launch per iteration) with
    k = 1, 2 ... chained moves per candidate, and learned + batched (MLP-ranked proposals). `forms`, if
    given, names the forms to run (e.g. ("batched", "plain_k2", "learned_batched"))."""
    import torch

    insts = I.make_batch(workload, seeds)
    kw = dict(eps=eps, gate=1)
    t0 = time.time()
    c_ref = _final_best(insts, biolog.make_params(n_cand=ref_n, seed=seed_offset, **kw), ref_iters)
    t_ref = time.time() - t0
    targets = [(1 + tol) * c for c in c_ref]
    wanted = None if forms is None else frozenset(forms)

    def want(name):
        return wanted is None or name in wanted

    forms = {}

    def summarise(name, ms, its, total_ms, setup_s, sequential, **extra):
        reached = [m for m in ms if m is not None]
        forms[name] = dict(reached=len(reached), iters=its, ms=[None if m is None else round(m, 3) for m in ms],
                           median_ms=float(np.median(ms)) if len(reached) == len(ms) else None,
                           all_instances_ms=(float(sum(ms)) if sequential else float(max(ms)))
                           if len(reached) == len(ms) else None,
                           run_ms=round(total_ms, 1), setup_s=round(setup_s, 2), **extra)

    # warm the kernels of every form once (module loading, attributes), outside the timed runs
    for k in k_values:
        if not (want("plain" if k == 1 else f"plain_k{k}") or want("batched" if k == 1 else f"batched_k{k}")):
            continue
        W = biolog.Search(insts[:1], biolog.make_params(n_cand=4096, seed=seed_offset, k_moves=k, **kw))
        W.search_step(2)
        W.close()
    for k in k_values:
        suffix = "" if k == 1 else f"_k{k}"
        ms_all, it_all, run_ms, setup = [], [], 0.0, 0.0
        for s, inst, tg in zip(seeds, insts, targets) if want("plain" + suffix) else ():
            t1 = time.time()
            S = biolog.Search([inst], biolog.make_params(n_cand=n, seed=seed_offset + int(s), k_moves=k, **kw))
            torch.cuda.synchronize()
            setup += time.time() - t1
            ms, its, _, tot = _wall_to_target(S, [tg], max_iters, S.search_step)
            ms_all += ms
            it_all += its
            run_ms += tot
            S.close()
        if want("plain" + suffix):
            summarise("plain" + suffix, ms_all, it_all, run_ms, setup, True, n_cand=n, k_moves=k)
        if not want("batched" + suffix):
            continue
        t1 = time.time()
        S = biolog.Search(insts, biolog.make_params(n_cand=n_batched, seed=seed_offset, k_moves=k, **kw))
        torch.cuda.synchronize()
        setup = time.time() - t1
        ms, its, _, tot = _wall_to_target(S, targets, max_iters, S.search_step)
        S.close()
        summarise("batched" + suffix, ms, its, tot, setup, False, n_cand=n_batched, k_moves=k)

    if want("learned_batched"):
        t1 = time.time()
        X, T = learned.collect(I.make_batch(workload, train_seeds), iters=train_iters, sample=train_sample,
                               stride=train_stride)
        net, losses = learned.train(X, T, hidden=256, steps=train_steps, batch=4096, lr=1e-3,
                                    max_batch=pool * len(insts))
        t_train = time.time() - t1
        t1 = time.time()
        S = biolog.Search(insts, biolog.make_params(n_cand=pool, seed=seed_offset, **kw))
        netS = net.copy(stream=S.stream, max_batch=pool * len(insts))
        torch.cuda.synchronize()
        setup = time.time() - t1
        ms, its, _, tot = _wall_to_target(S, targets, max_iters,
                                          lambda c: S.search_step_learned(netS, c, pool, keep, rand_frac))
        netS.close()
        S.close()
        net.close()
        summarise("learned_batched", ms, its, tot, setup, False, pool=pool, keep=keep, rand_frac=rand_frac,
                  train_tuples=int(X.shape[0]), train_s=round(t_train, 1),
                  train_loss_first_last=[float(np.mean(losses[:50])), float(np.mean(losses[-50:]))])
    return dict(workload=workload, seeds=[int(s) for s in seeds], tol=tol, max_iters=max_iters,
                c_ref=[float(c) for c in c_ref], c_ref_run=dict(n_cand=ref_n, iters=ref_iters, s=round(t_ref, 1)),
                timing="host wall clock through the API: per iteration one bl_search_step call and one bl_get_states read of every instance's C*",
                forms=forms)
