"""bl_get_states / bl_set_states: every instance's search state in one transfer each way equals the
per-instance calls, a resume through them continues the search exactly, and an invalid plan writes
nothing."""
import numpy as np
import pytest

from gpu_common import gpu_plan
from paper_1909_10286_gb300 import biolog
from paper_1909_10286_gb300 import instances as I

pytestmark = pytest.mark.gpu
KW = dict(eps=0.5, seed=1000, gate=1)


def _same(a, b):
    return (gpu_plan(a, "xold") == gpu_plan(b, "xold") and gpu_plan(a, "xbest") == gpu_plan(b, "xbest")
            and a["cstar"] == b["cstar"] and a["tmaxstar"] == b["tmaxstar"] and a["iter"] == b["iter"])


def test_packed_states_equal_the_per_instance_calls_and_resume_exactly():
    insts = I.make_batch("batched", range(40, 64))
    A = biolog.Search(insts, biolog.make_params(n_cand=4096, **KW))
    A.search_step(5)
    packed = A.get_states()
    assert len(packed) == len(insts)
    for k in range(len(insts)):
        assert _same(packed[k], A.get_state(inst=k))
    A.search_step(7)
    full = A.get_states()
    # resume a fresh handle from the packed checkpoint after 5 iterations
    B = biolog.Search(insts, biolog.make_params(n_cand=4096, **KW))
    B.set_states(packed)
    B.search_step(7)
    res = B.get_states()
    for k in range(len(insts)):
        assert _same(res[k], full[k]), k
    # an invalid plan in one instance: rejected, nothing written
    bad = [dict(x) for x in res]
    xo = [a.copy() for a in bad[3]["xold"]]
    xo[0][0] = xo[0][1]          # a BP twice
    bad[3]["xold"] = tuple(xo)
    bad[0]["cstar"] = 1.0
    with pytest.raises(biolog.BiologError) as e:
        B.set_states(bad)
    assert e.value.code == biolog.BL_EINVAL
    after = B.get_states()
    for k in range(len(insts)):
        assert _same(after[k], res[k])
    A.close()
    B.close()


def test_packed_state_calls_read_and_write_the_arrays_passed_each_time():
    """The binding keeps the ctypes state array while the same arrays come back: an edit made in place
    between calls is what bl_set_states takes, bl_get_states refills the same arrays, and other arrays
    (copies) are used as given."""
    insts = I.make_batch("batched", range(8, 11))
    A = biolog.Search(insts, biolog.make_params(n_cand=4096, **KW))
    A.search_step(4)
    st = A.get_states()
    arrays = [a for s in st for a in (*s["xold"], *s["xbest"])]
    for a, b in zip(st[1]["xold"], st[1]["xbest"]):
        a[:] = b                                    # x_old := x* of instance 1, in place
    st[1]["iter"] = 77
    A.set_states(st)
    one = A.get_state(inst=1)
    assert gpu_plan(one, "xold") == gpu_plan(one, "xbest") and one["iter"] == 77
    A.search_step(2)
    st2 = A.get_states(st)
    assert st2 is st and all(x is y for x, y in zip([a for s in st2 for a in (*s["xold"], *s["xbest"])], arrays))
    for k in range(len(insts)):
        assert _same(st2[k], A.get_state(inst=k))
    copies = [dict(s, xold=tuple(a.copy() for a in s["xold"]), xbest=tuple(a.copy() for a in s["xbest"]))
              for s in st2]
    A.search_step(3)
    A.set_states(copies)
    for k in range(len(insts)):
        assert _same(A.get_state(inst=k), copies[k])
    A.close()
