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


def pair(inst, n_cand, eps=0.5, seed=1000, gate=1, p_swap=0.0, fix_field_bp=0, fix_resources=0, inst_idx=0, **kw):
    p = biolog.make_params(n_cand=n_cand, eps=eps, seed=seed, gate=gate, p_swap=p_swap, fix_field_bp=fix_field_bp,
                           fix_resources=fix_resources, inst_idx=inst_idx, **kw)
    op = O.make_params(eps=eps, seed=seed, gate=gate, p_swap=p_swap, fix_field_bp=fix_field_bp,
                       fix_resources=fix_resources, inst_idx=inst_idx)
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
