"""The cooperative scorer (a group of lanes per candidate, one lane per tour)
computes value for value what the one-thread scorer computes, so a search with
it follows the same trajectory bit for bit: the same i*, C_{i*}, base choices,
C* and plans, iteration after iteration. The one-thread scorer itself is
checked against the oracle in test_gpu_parity.py; a mismatch here is a
mismatch with the oracle's trajectory too."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1909_10286_gb300 import biolog
from paper_1909_10286_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _trajectory(insts, lanes, iters, **kw):
    S = biolog.Search(insts, biolog.make_params(lanes_per_cand=lanes, **kw))
    assert S.config()["lanes_per_cand"] == max(1, lanes)
    S.search_step(iters)
    logs = [S.get_log(0, iters, inst=k) for k in range(len(insts))]
    states = [S.get_state(inst=k) for k in range(len(insts))]
    S.close()
    return logs, states


def _same(a, b):
    (la, sa), (lb, sb) = a, b
    for x, y in zip(la, lb):
        for key in ("istar", "c_istar", "use_best", "cstar", "indicator"):
            assert np.array_equal(x[key], y[key]), key
    for x, y in zip(sa, sb):
        assert x["cstar"] == y["cstar"] and x["tmaxstar"] == y["tmaxstar"] and x["iter"] == y["iter"]
        for w in ("xold", "xbest"):
            for p, q in zip(x[w], y[w]):
                assert np.array_equal(p, q), w


@pytest.mark.parametrize("workload,seeds,lanes,n_cand,iters,kw", [
    ("large", [0], 16, 5000, 6, {}),
    ("large", [1], 32, 3000, 5, {}),
    ("large", [2], 16, 2048, 4, dict(gate=2, p_swap=0.3)),
    ("large", [3], 16, 2048, 4, dict(gate=0, fix_resources=1)),
    ("batched", [3, 5, 8, 11], 8, 3000, 5, {}),
    ("batched", [13, 21], 16, 2500, 5, dict(p_swap=0.2)),
    ("paper", [4], 4, 4096, 8, {}),
    ("paper", [6], 8, 3333, 8, dict(fix_field_bp=1)),
    ("tiny", [0], 4, 700, 12, {}),
])
def test_cooperative_search_follows_the_one_thread_trajectory(workload, seeds, lanes, n_cand, iters, kw):
    insts = I.make_batch(workload, seeds)
    kw = dict(dict(n_cand=n_cand, eps=0.5, seed=1000, gate=1), **kw)
    _same(_trajectory(insts, lanes, iters, **kw), _trajectory(insts, 1, iters, **kw))


def test_cooperative_search_matches_the_oracle_argmin():
    """Independently of the one-thread kernel: the first cooperative iterations'
    argmins on a large instance are the oracle's wherever the best two costs are
    apart, and C_{i*} agrees within the FP32 tolerance."""
    import os

    inst = I.make_instance("large", 4)
    n, iters = 2048, 3
    S = biolog.Search([inst], biolog.make_params(n_cand=n, eps=0.5, seed=1000, gate=1, lanes_per_cand=16))
    S.search_step(iters)
    log = S.get_log(0, iters)
    o = O.Oracle(inst)
    op = O.make_params(eps=0.5, seed=1000, gate=1)
    res = o.search(op, o.start(op), iters, n, threads=os.cpu_count() or 1, force_istar=log["istar"])
    for it in range(iters):
        if res["gap"][it] > 1e-5:
            assert int(log["istar"][it]) == int(res["istar"][it]), it
        c_o, c_g = float(res["c_istar"][it]), float(log["c_istar"][it])
        assert np.isfinite(c_o) == np.isfinite(c_g)
        if np.isfinite(c_o):
            assert c_g == pytest.approx(c_o, rel=1e-5), it
    S.close()


def test_cooperative_learned_iteration_equals_one_thread_learned_iteration():
    from paper_1909_10286_gb300.mlp import MLP

    inst = I.make_instance("large", 5)
    pool, keep, rf = 8192, 700, 0.02
    outs = []
    for lanes in (1, 16):
        S = biolog.Search([inst], biolog.make_params(n_cand=pool, eps=0.5, seed=1000, gate=1, lanes_per_cand=lanes))
        S.search_step(2)
        net = MLP(64, 256, max_batch=pool, seed=5, stream=S.stream)
        S.search_step_learned(net, 3, pool, keep, rf)
        outs.append((S.get_log(2, 3), S.get_state()))
        net.close()
        S.close()
    (la, sa), (lb, sb) = outs
    for key in ("istar", "c_istar", "cstar"):
        assert np.array_equal(la[key], lb[key]), key
    assert sa["cstar"] == sb["cstar"]


@pytest.mark.parametrize("workload,lanes", [("large", 8), ("large", 4), ("paper", 32), ("batched", 4)])
def test_unsupported_lane_counts_are_rejected(workload, lanes):
    insts = I.make_batch(workload, [7]) if workload == "batched" else [I.make_instance(workload, 0)]
    if workload == "batched" and max(i.n_tours for i in insts) <= lanes:
        insts = [i for i in I.make_batch("batched", range(40)) if i.n_tours > lanes][:1]
    with pytest.raises(biolog.BiologError) as e:
        biolog.Search(insts, biolog.make_params(n_cand=1024, lanes_per_cand=lanes))
    assert e.value.code == biolog.BL_EINVAL
