"""ShapedBatch: a batch split by launch shape into one handle per group on one stream. Each instance of
the batch follows exactly the trajectory its group's handle gives it on its own, the state calls map
the batch's instance indices correctly, and a resume through get_states / set_states continues
exactly."""
import numpy as np
import pytest

from gpu_common import gpu_plan
from paper_1909_10286_gb300 import biolog, shaped
from paper_1909_10286_gb300 import instances as I

pytestmark = pytest.mark.gpu
KW = dict(eps=0.5, seed=1000, gate=1)


def _params(group):
    return biolog.make_params(n_cand=4096, **KW)


def _same(a, b):
    return (gpu_plan(a, "xold") == gpu_plan(b, "xold") and gpu_plan(a, "xbest") == gpu_plan(b, "xbest")
            and a["cstar"] == b["cstar"] and a["iter"] == b["iter"])


def test_groups_split_by_shape_and_map_every_instance():
    insts = I.make_batch("batched", range(24))
    gs = shaped.groups(insts)
    assert len(gs) == 2 and sorted(gs[0] + gs[1]) == list(range(24))
    assert all(shaped.small(insts[i]) for i in gs[0]) and not any(shaped.small(insts[i]) for i in gs[1])
    B = shaped.ShapedBatch(insts, _params)
    cfg = B.config()
    assert [g["n_instances"] for g in cfg["groups"]] == [len(g) for g in gs]
    assert cfg["groups"][0]["block_threads"] == 256 and cfg["groups"][1]["block_threads"] == 128
    assert cfg["launches_per_iter"] == 2
    B.search_step(6)
    # each group's instances follow the trajectories a Search of that group alone gives them
    for g in gs:
        S = biolog.Search([insts[i] for i in g], _params(None))
        S.search_step(6)
        for k, i in enumerate(g):
            assert _same(B.get_state(inst=i), S.get_state(inst=k))
            np.testing.assert_array_equal(B.get_log(0, 6, inst=i)["cstar"], S.get_log(0, 6, inst=k)["cstar"])
            assert B.best_plan(inst=i)["cost_km"] == S.best_plan(inst=k)["cost_km"]
        S.close()
    # packed states in the batch's order, and the same dicts refilled
    st = B.get_states()
    for i in range(len(insts)):
        assert _same(st[i], B.get_state(inst=i))
    B.search_step(2)
    st2 = B.get_states(st)
    assert st2[0] is st[0] and all(_same(st2[i], B.get_state(inst=i)) for i in range(len(insts)))
    B.close()


def test_resume_through_packed_states_continues_exactly():
    insts = I.make_batch("batched", range(40, 56))
    A = shaped.ShapedBatch(insts, _params)
    A.search_step(4)
    ck = [dict(s, xold=tuple(np.copy(a) for a in s["xold"]), xbest=tuple(np.copy(a) for a in s["xbest"]))
          for s in A.get_states()]
    A.search_step(5)
    want = A.get_states()
    B = shaped.ShapedBatch(insts, _params)
    B.set_states(ck)
    B.search_step(5)
    got = B.get_states()
    assert all(_same(a, b) for a, b in zip(got, want))
    A.close()
    B.close()
