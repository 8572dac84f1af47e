"""The launch-shape autotuner: it tries lanes per candidate, blocks per SM and
work-item sizes on the real search, and whatever it picks changes the speed
only -- the tuned search follows the default search's trajectory bit for bit."""
import numpy as np
import pytest

from paper_1909_10286_gb300 import autotune, biolog
from paper_1909_10286_gb300 import instances as I

pytestmark = pytest.mark.gpu


def test_autotuner_picks_a_built_shape_and_keeps_the_results():
    insts = I.make_batch("batched", range(8))
    kw = dict(eps=0.5, seed=1000, gate=1)
    best = autotune.tune(insts, 2048, base_params=kw, iters=2, use_cache=False)
    assert best["lanes_per_cand"] in autotune.LANES and best["tried"] >= 16
    assert best["ms_per_iter"] > 0
    p = biolog.make_params(n_cand=2048, blocks_per_sm=best["blocks_per_sm"], tile=best["tile"],
                           lanes_per_cand=best["lanes_per_cand"], **kw)
    runs = []
    for params in (p, biolog.make_params(n_cand=2048, **kw)):
        S = biolog.Search(insts, params)
        S.search_step(4)
        runs.append([S.get_log(0, 4, inst=k) for k in range(len(insts))])
        S.close()
    for a, b in zip(*runs):
        for key in ("istar", "c_istar", "cstar"):
            assert np.array_equal(a[key], b[key]), key
