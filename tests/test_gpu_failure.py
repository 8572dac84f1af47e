"""Failure detection without a GPU fault: a bounded device wait that nothing
completes gives up after its limit and comes back as BL_ETIMEOUT, and the
context stays usable for the search afterwards."""
import pytest

from paper_1909_10286_gb300 import biolog
from paper_1909_10286_gb300 import instances as I

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    rc, ns = biolog.wait_selftest(2_000_000)   # 2 ms
    assert rc == biolog.BL_ETIMEOUT
    assert 2_000_000 <= ns < 500_000_000
    S = biolog.Search([I.make_instance("tiny", 0)], biolog.make_params(n_cand=4096, seed=1000))
    S.search_step(3)
    assert S.get_state()["iter"] == 3
    rc, _ = biolog.wait_selftest(1_000_000)
    assert rc == biolog.BL_ETIMEOUT
    S.search_step(2)
    st = S.get_state()
    assert st["iter"] == 5 and st["cstar"] > 0
    S.close()


def test_wait_selftest_rejects_bad_limits():
    assert biolog.wait_selftest(0)[0] == biolog.BL_EINVAL
    assert biolog.wait_selftest(11_000_000_000)[0] == biolog.BL_EINVAL
