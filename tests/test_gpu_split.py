"""Split iterations on one GPU: the candidates of one instance scored in slices by separate handles
(bl_search_score_slice), their keys reduced to the minimum, and every handle updated from that key
(bl_search_apply), follow the unsplit search bit for bit. The slices run one after another in one
process -- no kernel waits for another."""
import numpy as np
import pytest

from gpu_common import gpu_plan
from paper_1909_10286_gb300 import biolog
from paper_1909_10286_gb300 import instances as I
from paper_1909_10286_gb300.split import GpuSlice, SplitSearch, slice_of

pytestmark = pytest.mark.gpu
KW = dict(eps=0.5, seed=1000, gate=1)


@pytest.mark.parametrize("wl,n,parts,iters,k", [("paper", 1 << 16, 2, 12, 1), ("paper", 50001, 3, 8, 2),
                                                ("batched", 30011, 4, 8, 1), ("large", 1 << 15, 2, 4, 1)])
def test_split_iterations_follow_the_unsplit_search(wl, n, parts, iters, k):
    import torch

    inst = I.make_instance(wl, 7)
    ref = biolog.Search([inst], biolog.make_params(n_cand=n, k_moves=k, **KW), stream=torch.cuda.current_stream())
    slices = [GpuSlice(inst, n, parts, r, k_moves=k, **KW) for r in range(parts)]
    assert sum(s.count for s in slices) == n
    for it in range(iters):
        ref.search_step(1)
        keys = [s.score_slice().clone() for s in slices]
        key = torch.stack(keys).min(dim=0).values
        for s in slices:
            s.apply(key)
        want = ref.get_state()
        log = ref.get_log(it, 1)
        assert int(key.item()) & 0xFFFFFFFF == int(log["istar"][0])
        for s in slices:
            got = s.search.get_state()
            assert gpu_plan(got, "xold") == gpu_plan(want, "xold") and gpu_plan(got, "xbest") == gpu_plan(want, "xbest")
            assert got["cstar"] == want["cstar"] and got["tmaxstar"] == want["tmaxstar"] and got["iter"] == it + 1
            glog = s.search.get_log(it, 1)
            assert int(glog["istar"][0]) == int(log["istar"][0]) and glog["use_best"][0] == log["use_best"][0]
    for s in slices:
        s.close()
    ref.close()


def test_split_search_driver_with_one_rank():
    """SplitSearch without a process group: one slice, the whole range, the same trajectory."""
    import torch

    inst = I.make_instance("paper", 3)
    n = 20000
    ref = biolog.Search([inst], biolog.make_params(n_cand=n, **KW), stream=torch.cuda.current_stream())
    ref.search_step(6)
    one = GpuSlice(inst, n, 1, 0, **KW)
    SplitSearch(one).step(6)
    a, b = ref.get_state(), one.search.get_state()
    assert gpu_plan(a, "xbest") == gpu_plan(b, "xbest") and a["cstar"] == b["cstar"] and b["iter"] == 6
    one.close()
    ref.close()


def test_apply_rejects_a_key_that_is_not_this_iterations():
    """A key whose cost does not match its candidate's score leaves the handle refusing work."""
    import torch

    inst = I.make_instance("paper", 3)
    s = GpuSlice(inst, 4096, 1, 0, **KW)
    key = s.score_slice().clone()
    bad = torch.tensor([int(key.item()) ^ (1 << 40)], dtype=torch.int64, device="cuda")   # another cost
    s.apply(bad)
    with pytest.raises(biolog.BiologError) as e:
        s.search.get_state()
    assert e.value.code == biolog.BL_ESTATE
    with pytest.raises(biolog.BiologError):
        s.search.search_step(1)
    assert slice_of(4096, 1, 0) == (0, 4096)
