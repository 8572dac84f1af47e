"""Helpers shared by the GPU parity tests: the CUDA search and the oracle on
the same seeded inputs."""
import numpy as np

from oracle import oracle as O
from paper_1909_10286_gb300 import biolog

# FP32 GPU vs FP64 oracle: costs within 1e-5 relative wherever every discrete
# decision of the candidate has a relative margin above TAU (see the decision
# margins recorded by the oracle).
REL_TOL = 1e-5
TAU = 1e-5


def pair(inst, n_cand, eps=0.5, seed=1000, gate=1, p_swap=0.0, fix_field_bp=0, fix_resources=0, inst_idx=0,
         k_moves=1, **kw):
    p = biolog.make_params(n_cand=n_cand, eps=eps, seed=seed, gate=gate, p_swap=p_swap, fix_field_bp=fix_field_bp,
                           fix_resources=fix_resources, inst_idx=inst_idx, k_moves=k_moves, **kw)
    op = O.make_params(eps=eps, seed=seed, gate=gate, p_swap=p_swap, fix_field_bp=fix_field_bp,
                       fix_resources=fix_resources, inst_idx=inst_idx, k_moves=k_moves)
    return biolog.Search([inst], p), O.Oracle(inst), op


def gpu_plan(state, which="xold"):
    return O.Plan(*state[which])


def compare_costs(gc, oc, margin, feas_g=None, feas_o=None):
    """Returns (n_compared, n_excluded, worst relative error) and asserts parity."""
    gc = gc.astype(np.float64)
    strict = margin > TAU
    fin_o = np.isfinite(oc)
    fin_g = np.isfinite(gc)
    assert np.array_equal(fin_o[strict], fin_g[strict]), "feasibility / gate decisions differ"
    both = strict & fin_o
    rel = np.abs(gc[both] - oc[both]) / np.abs(oc[both])
    worst = float(rel.max()) if rel.size else 0.0
    assert worst <= REL_TOL, f"relative cost error {worst:.3e}"
    return int(strict.sum()), int((~strict).sum()), worst


def check_candidates(g, r, n, base_margin=np.inf, limit=0.02):
    """Parity of per-candidate GPU results g (cost, tmax; optionally hu_tour, su_tour) with the oracle's
    r (cost, tmax, margin, hu_tour, su_tour) under the decision-margin protocol:
      - strict candidates (every decision's relative gap > TAU): the same feasibility and gate verdict,
        C_i within REL_TOL, Tmax_i within REL_TOL where the candidate is feasible, and (when given) the
        same HU and SU assignments;
      - excluded candidates (some gap <= TAU) whose assignments equal the oracle's: C_i within REL_TOL;
        those resolved differently (another assignment or verdict) may be at most `limit` of n, unless
        the base plan itself holds a near-tie (base_margin <= TAU), which every candidate inherits.
    Returns (n_strict, n_excluded, n_resolved_differently, worst relative error)."""
    gc = g["cost"].astype(np.float64)
    gt = g["tmax"].astype(np.float64)
    n_cmp, n_ex, worst = compare_costs(gc, r["cost"], r["margin"])
    strict = r["margin"] > TAU
    feas = np.isfinite(r["tmax"]) & np.isfinite(gt)
    both = strict & feas
    assert np.array_equal(np.isfinite(gt)[strict], np.isfinite(r["tmax"])[strict]), "Eq. 2 verdicts differ"
    if both.any():
        rel_t = np.abs(gt[both] - r["tmax"][both]) / np.abs(r["tmax"][both])
        assert rel_t.max() <= REL_TOL, f"Tmax error {rel_t.max():.3e}"
    same = np.isfinite(gc) == np.isfinite(r["cost"])
    if "hu_tour" in g:
        same_units = np.all(g["hu_tour"] == r["hu_tour"], axis=1) & np.all(g["su_tour"] == r["su_tour"], axis=1)
        st_fin = strict & np.isfinite(r["tmax"])
        assert same_units[st_fin].all(), "assignments of strict candidates differ"
        same &= same_units
    ex = ~strict
    agree_ex = ex & same & np.isfinite(r["cost"])
    if agree_ex.any():
        rel = np.abs(gc[agree_ex] - r["cost"][agree_ex]) / np.abs(r["cost"][agree_ex])
        assert rel.max() <= REL_TOL, f"excluded candidate with the oracle's outcome off by {rel.max():.3e}"
        worst = max(worst, float(rel.max()))
    n_diff = int((ex & ~same).sum())
    if base_margin > TAU:
        assert n_diff <= limit * n + 5, f"{n_diff} of {n} near-ties resolved differently"
    else:
        assert n_cmp >= 0.01 * n, "almost nothing left to compare strictly"
    return n_cmp, n_ex, n_diff, worst
