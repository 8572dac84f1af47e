"""Element-wise parity of the timed search kernel with the oracle.

bl_search_step_inspect runs one iteration with the kernel, launch shape and
work items bl_search_step replays, and writes each candidate's {C_i, Tmax_i}
where the kernel decides it: at the Eq. 2 check of the draw phase, at the
completion-time gate of the first stage (Sec. 2.5), or after the full score of
the second stage, resumed from the survivor record (shapes of up to 6 tours)
or recomputed (more tours). Every candidate of the iteration is compared:
  - with the inspection kernel (bl_score_candidates), bit for bit: the queue
    and survivor-record path gives the same FP32 results as the plain path;
  - with the oracle's FP64 score of the same candidate under the
    decision-margin protocol (strict candidates within 1e-5 and with the same
    verdicts and assignments; excluded ones within 1e-5 where they reach the
    oracle's assignments, at most 2 % resolved differently);
  - and the iteration's i* (the log) is the argmin of the written costs.
One workload per kernel shape (four, three, six, ten and sixteen tours), at
the bench's sizes and launch configurations for the paper and batched
workloads, plus the paper's own scale (1200 fields, Table 1 fleet)."""
import os

import numpy as np
import pytest

from gpu_common import REL_TOL, TAU, check_candidates, gpu_plan
from oracle import oracle as O
from paper_1909_10286_gb300 import biolog
from paper_1909_10286_gb300 import instances as I

pytestmark = pytest.mark.gpu
THREADS = os.cpu_count() or 1
KW = dict(eps=0.5, seed=1000, gate=1)


def _argmin_key(cost):
    bits = cost.astype(np.float32).view(np.uint32).astype(np.uint64)
    keys = (bits << np.uint64(32)) | np.arange(len(cost), dtype=np.uint64)
    return int(keys.min())


def _inspect_and_compare(S, insts, n, warm_iters, check_insts=None, limit=0.02):
    import torch

    if warm_iters:
        S.search_step(warm_iters)
    states = [S.get_state(inst=k) for k in range(len(insts))]
    out = torch.full((len(insts), n, 2), float("nan"), dtype=torch.float32, device="cuda")
    S.search_step_inspect(out, n)
    torch.cuda.synchronize()
    out = out.cpu().numpy()
    assert not np.isnan(out).any(), "a candidate was left unwritten"
    check = list(check_insts if check_insts is not None else range(len(insts)))
    logs = {k: S.get_log(states[k]["iter"], 1, inst=k) for k in check}
    # the plain inspection path stages the handle's current plans: score the iteration's candidates
    # from the state before the step, then put the state after it back
    after = {k: S.get_state(inst=k) for k in check}
    dumps = {}
    for k in check:
        S.set_state(states[k], inst=k)
        dumps[k] = S.score_candidates(int(logs[k]["use_best"][0]), states[k]["iter"], states[k]["tmaxstar"], 0, n,
                                      inst=k, units=True)
        S.set_state(after[k], inst=k)
    report = []
    for k in check:
        inst, st, log, g = insts[k], states[k], logs[k], dumps[k]
        use_best = int(log["use_best"][0])
        cost, tmax = out[k, :, 0], out[k, :, 1]
        # i* of the iteration is the argmin of the costs the kernel wrote
        key = _argmin_key(cost)
        assert int(log["istar"][0]) == key & 0xFFFFFFFF
        assert np.float32(log["c_istar"][0]) == np.uint32(key >> 32).view(np.float32)
        # the timed kernel's queue and record path equals the plain inspection path bit for bit
        assert np.array_equal(cost.view(np.uint32), g["cost"].view(np.uint32)), "C_i differs from the plain path"
        assert np.array_equal(tmax.view(np.uint32), g["tmax"].view(np.uint32)), "Tmax_i differs from the plain path"
        # and the oracle, candidate by candidate
        o = O.Oracle(inst)
        op = O.make_params(inst_idx=k, **KW)
        base = gpu_plan(st, "xbest" if use_best else "xold")
        tstar = o.score(gpu_plan(st, "xbest"), op, gate=0)["tmax"] if np.isfinite(st["cstar"]) else np.inf
        r = o.score_batch(op, st["iter"], base, n, tmax_star=tstar, threads=THREADS, details=True)
        assert np.array_equal(g["moves"], r["moves"]), "Philox moves differ"
        g2 = dict(cost=cost, tmax=tmax, hu_tour=g["hu_tour"], su_tour=g["su_tour"])
        base_margin = o.score(base, op, gate=0)["margin"]
        n_cmp, n_ex, n_diff, worst = check_candidates(g2, r, n, base_margin, limit=limit)
        decided = dict(infeasible=int((~np.isfinite(tmax)).sum()),
                       gated=int((np.isfinite(tmax) & ~np.isfinite(cost)).sum()),
                       scored=int(np.isfinite(cost).sum()))
        report.append((k, n_cmp, n_ex, n_diff, worst, decided))
    for row in report:
        print("instance %d: strict %d, excluded %d, resolved differently %d, worst %.2e, %s" % row)
    return report


def test_timed_kernel_paper_full_size():
    """The default bench line: paper instance 0 (three tours, shape with distances in shared
    memory and survivor records), 2^20 candidates, after 2 iterations."""
    inst = I.make_instance("paper", 0)
    n = I.SEARCH["paper"][0]
    S = biolog.Search([inst], biolog.make_params(n_cand=n, **KW))
    rep = _inspect_and_compare(S, [inst], n, 2)
    assert rep[0][5]["scored"] > 0 and rep[0][5]["gated"] > 0 and rep[0][5]["infeasible"] > 0
    S.close()


def test_timed_kernel_batched_full_size():
    """bench.py --workload batched: 256 uneven instances (up to six tours: the six-tour shape,
    distances through L2, survivor records), 2^16 candidates each, autotuned launch shape; the
    oracle scores every candidate of 8 of the instances, the largest among them."""
    from paper_1909_10286_gb300 import autotune

    insts = I.make_batch("batched", range(256))
    n = I.SEARCH["batched"][0]
    S = biolog.Search(insts, autotune.tuned_params(insts, n, **KW))
    sizes = np.array([i.n_fields * i.n_tours for i in insts])
    pick = sorted(set(np.argsort(-sizes)[:4].tolist() + [0, 1, 2, 255]))
    _inspect_and_compare(S, insts, n, 1, check_insts=pick)
    S.close()


@pytest.mark.parametrize("F,B,T,H,S_,n,lanes", [(140, 5, 5, 10, 20, 20000 + 37, 0),
                                                 (186, 5, 8, 10, 20, 12000 + 5, 0),
                                                 (300, 20, 16, 64, 128, 6000 + 11, 0),
                                                 (120, 8, 6, 12, 40, 10000 + 3, 16)])
def test_timed_kernel_sized_shapes(F, B, T, H, S_, n, lanes):
    """Five, eight and sixteen tours (the six-, ten- and sixteen-tour shapes), and the cooperative
    kernel (16 lanes per candidate), ragged candidate counts, after 3 iterations."""
    inst = I.make_sized(F, B, T, H, S_, seed=F + T)
    S = biolog.Search([inst], biolog.make_params(n_cand=n, lanes_per_cand=lanes, **KW))
    _inspect_and_compare(S, [inst], n, 3)
    S.close()


def test_timed_kernel_large():
    """The large workload (300 fields, 10 tours, 60 HUs, 120 SUs: the ten-tour shape), 2^18
    candidates, after 2 iterations."""
    inst = I.make_instance("large", 0)
    n = 1 << 18
    S = biolog.Search([inst], biolog.make_params(n_cand=n, **KW))
    _inspect_and_compare(S, [inst], n, 2)
    S.close()


def test_timed_kernel_replica_scale():
    """The paper's experiment scale (Sec. 3.1, Table 1): 1200 fields, 20 BPs, 7 tours, 7 HUs and
    the 14 + 28 two-class SU fleet; N = 1221 nodes, the distances (5.96 MB) read through L2.
    8,192 candidates per iteration, compared after 1 and after 4 iterations."""
    inst = I.make_instance("replica", 0)
    n = 8192
    S = biolog.Search([inst], biolog.make_params(n_cand=n, **KW))
    _inspect_and_compare(S, [inst], n, 1)
    _inspect_and_compare(S, [inst], n, 2)
    S.close()
