"""The four-case experiment driver (Sec. 3.2 structure) on small budgets."""
import numpy as np
import pytest

from paper_1909_10286_gb300 import biolog, experiment
from paper_1909_10286_gb300 import instances as I

pytestmark = pytest.mark.gpu


def test_four_cases_over_the_eps_grid():
    r = experiment.run("paper", seeds=range(3), iters=30, n_cand=2048)
    c1 = [p["cost_km"] for p in r["cases"][1]["per_instance"]]
    for case in (2, 3, 4):
        per = r["cases"][case]["per_instance"]
        assert len(per) == 3
        for k, p in enumerate(per):
            assert p["eps"] in experiment.EPS_GRID
            if np.isfinite(c1[k]):
                assert p["cost_km"] <= c1[k] * (1 + 1e-6)   # C* never increases from the initial plan
        assert r["cases"][case]["t_solve_s"] > 0
    # Case 2 keeps the round-robin dealing of the units over the active tours (no local minimisation)
    insts = I.make_batch("paper", range(3))
    S2 = biolog.Search(insts, biolog.make_params(n_cand=2048, eps=0.5, seed=1000, **experiment.CASES[2]))
    S2.search_step(30)
    for k, inst in enumerate(insts):
        b = S2.best_plan(inst=k)
        if not np.isfinite(b["cost_km"]):
            continue   # an infeasible initial plan stays so when the field -> BP assignment is fixed
        na = int((b["tour_cnt"] > 0).sum())
        for units, got in ((inst.n_hu, b["tour_n_hu"]), (inst.n_su, b["tour_n_su"])):
            want = sorted(units // na + (1 if j < units % na else 0) for j in range(na))
            assert sorted(int(x) for x in got[b["tour_cnt"] > 0]) == want
    S2.close()
    assert r["cases"][4]["feasible"] >= r["cases"][1]["feasible"]
