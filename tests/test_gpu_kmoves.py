"""Candidates of k chained moves (Step 8 repeated, Sec. 2.5) on the GPU against the oracle:
move records and decoded plans bit for bit, costs under the decision-margin protocol, the timed
kernel candidate by candidate, and whole search trajectories, for k = 2 and 3 on the kernel
shapes of three, five and ten tours."""
import numpy as np
import pytest

from gpu_common import REL_TOL, check_candidates, gpu_plan, pair
from paper_1909_10286_gb300 import biolog
from paper_1909_10286_gb300 import instances as I
from test_gpu_parity import _trajectory

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("wl,seed,n,k,p_swap,fix", [("paper", 1, 8192 + 17, 2, 0.0, 0), ("paper", 2, 6001, 3, 0.3, 0),
                                                 ("paper", 3, 4096, 2, 0.0, 1), ("batched", 11, 5003, 2, 0.2, 0),
                                                 ("batched", 12, 4001, 3, 0.0, 0), ("large", 1, 3001, 2, 0.1, 0)])
def test_chained_moves_decode_and_costs(wl, seed, n, k, p_swap, fix):
    inst = I.make_instance(wl, seed)
    S, o, op = pair(inst, n, p_swap=p_swap, fix_field_bp=fix, k_moves=k)
    S.search_step(2)
    st = S.get_state()
    for use_best in (0, 1):
        base = gpu_plan(st, "xbest" if use_best else "xold")
        it = st["iter"]
        tstar = o.score(gpu_plan(st, "xbest"), op, gate=0)["tmax"] if np.isfinite(st["cstar"]) else np.inf
        g = S.score_candidates(use_best, it, st["tmaxstar"], 0, n, units=True)
        r = o.score_batch(op, it, base, n, tmax_star=tstar, threads=8, details=True)
        assert g["moves"].shape == (n, 4 * k)
        assert np.array_equal(g["moves"], r["moves"]), "chained move records differ"
        base_margin = o.score(base, op, gate=0)["margin"]
        n_cmp, n_ex, n_diff, worst = check_candidates(g, r, n, base_margin)
        print(f"{wl}/{seed} k={k} base={use_best}: strict {n_cmp}, excluded {n_ex}, resolved differently {n_diff}, "
              f"worst {worst:.2e}")
        rng = np.random.default_rng(seed)
        idx = np.unique(np.concatenate([rng.integers(0, n, 300), np.arange(max(0, n - 40), n), [0]])).astype(np.int32)
        plans = S.decode_candidates(use_best, it, idx)
        F, B, T = inst.n_fields, inst.n_bps, inst.n_tours
        for row, i in zip(plans, idx):
            want, mv = o.candidate(op, it, int(i), base)
            assert np.array_equal(mv.ravel(), r["moves"][i])
            got = O_plan(row, B, T, F)
            assert got == want, (int(i), mv.tolist())
    S.close()


def O_plan(row, B, T, F):
    from oracle import oracle as O
    return O.Plan(row[:B], row[B:B + T], row[B + T:B + T + F], row[B + T + F:])


@pytest.mark.parametrize("wl,seed,n,iters,k,kw", [("paper", 0, 4096, 12, 2, {}), ("paper", 4, 2048, 8, 3, dict(p_swap=0.2)),
                                                ("batched", 3, 2500, 8, 2, {}),
                                                ("large", 2, 2048, 4, 3, dict(eps=0.25))])
def test_chained_move_trajectory_matches_oracle(wl, seed, n, iters, k, kw):
    _, _, n_ties = _trajectory(I.make_instance(wl, seed), n, iters, k_moves=k, **kw)
    assert n_ties <= 1


def test_chained_moves_timed_kernel_candidate_by_candidate():
    """The timed kernel with two chained moves writes, for every candidate, exactly what the plain
    path computes, and the iteration's i* is the argmin."""
    import torch

    inst = I.make_instance("paper", 5)
    n = 1 << 16
    S, o, op = pair(inst, n, k_moves=2)
    S.search_step(2)
    st = S.get_state()
    out = torch.full((1, n, 2), float("nan"), dtype=torch.float32, device="cuda")
    S.search_step_inspect(out, n)
    torch.cuda.synchronize()
    out = out.cpu().numpy()[0]
    log = S.get_log(st["iter"], 1)
    after = S.get_state()
    S.set_state(st)
    g = S.score_candidates(int(log["use_best"][0]), st["iter"], st["tmaxstar"], 0, n)
    S.set_state(after)
    assert np.array_equal(out[:, 0].view(np.uint32), g["cost"].view(np.uint32))
    assert np.array_equal(out[:, 1].view(np.uint32), g["tmax"].view(np.uint32))
    bits = g["cost"].view(np.uint32).astype(np.uint64)
    key = int(((bits << np.uint64(32)) | np.arange(n, dtype=np.uint64)).min())
    assert int(log["istar"][0]) == key & 0xFFFFFFFF
    S.close()


def test_chained_moves_rejected_where_unsupported():
    inst = I.make_instance("paper", 0)
    with pytest.raises(biolog.BiologError) as e:
        biolog.Search([inst], biolog.make_params(n_cand=1024, k_moves=4))
    assert e.value.code == biolog.BL_EINVAL
    with pytest.raises(biolog.BiologError) as e:
        biolog.Search([inst], biolog.make_params(n_cand=1024, k_moves=2, lanes_per_cand=8))
    assert e.value.code == biolog.BL_EINVAL


@pytest.mark.parametrize("wl,seed", [("paper", 0), ("batched", 3), ("large", 2)])
def test_chained_moves_keep_the_initial_plan_and_its_report(wl, seed):
    """The number of moves per candidate changes neither Step 4 (x*, C*, Tmax* of the initial plan)
    nor the report of x*: both score the plan itself."""
    inst = I.make_instance(wl, seed)
    A, _, _ = pair(inst, 256)
    B, _, _ = pair(inst, 256, k_moves=3)
    a, b = A.get_state(), B.get_state()
    assert gpu_plan(a, "xbest") == gpu_plan(b, "xbest")
    assert a["cstar"] == b["cstar"] and a["tmaxstar"] == b["tmaxstar"]
    ra, rb = A.best_plan(), B.best_plan()
    for key in ("tour_cost_km", "tour_tcompl_h", "hu_tour", "su_tour"):
        assert np.array_equal(ra[key], rb[key]), key
    A.close()
    B.close()
