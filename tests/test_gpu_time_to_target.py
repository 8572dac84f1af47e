"""The time-to-target harness: the iteration at which it sees each instance reach its target (one
bl_get_states read of every instance's C* per iteration) is the first iteration whose logged C* is
at or below the target, on a search that runs the same iterations."""
import numpy as np
import pytest

from paper_1909_10286_gb300 import biolog
from paper_1909_10286_gb300 import instances as I
from paper_1909_10286_gb300 import time_to_target as TT

pytestmark = pytest.mark.gpu
KW = dict(eps=0.5, seed=1000, gate=1)


def test_wall_to_target_reports_the_first_logged_iteration_at_or_below_the_target():
    insts = I.make_batch("batched", range(3))
    n_it = 40
    A = biolog.Search(insts, biolog.make_params(n_cand=4096, **KW))
    A.search_step(n_it)
    logs = [A.get_log(0, n_it, inst=k)["cstar"] for k in range(len(insts))]
    A.close()
    # per instance: a target reached part-way (the C* logged after iteration 12), and one never reached
    targets = [float(c[11]) for c in logs]
    want = [int(np.argmax(c <= t)) + 1 for c, t in zip(logs, targets)]
    B = biolog.Search(insts, biolog.make_params(n_cand=4096, **KW))
    ms, its, n, total = TT._wall_to_target(B, targets, n_it, B.search_step)
    B.close()
    assert its == want
    assert all(m is not None and 0.0 < m <= total for m in ms)
    assert n == max(want)
    C = biolog.Search(insts[:1], biolog.make_params(n_cand=4096, **KW))
    ms, its, n, _ = TT._wall_to_target(C, [0.5 * float(logs[0][-1])], 5, C.search_step)
    C.close()
    assert ms == [None] and its == [None] and n == 5
