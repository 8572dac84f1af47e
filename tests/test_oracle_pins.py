"""Pins of the CPU oracle against values fixed by the paper, by published
test vectors or by hand derivation -- never by the oracle itself.

Each hand-derived expectation is worked out in the comments next to it so a
reader can re-check it with pencil and paper.
"""
import math
import os

import numpy as np
import pytest

from conftest import GOLDEN
from paper_1909_10286_gb300 import instances as I


def _load_kat():
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle_mod):
    """Random123's published Philox4x32-10 vectors."""
    rows = _load_kat()
    assert len(rows) == 3
    for ctr, key, expect in rows:
        assert list(oracle_mod.philox4x32_10(ctr, key)) == expect


def test_first_move_from_known_answer(oracle_mod):
    """Counter (i=0, iter=0, inst=0, 0) with seed 0 is the all-zero KAT input,
    so the first move of the tiny instance follows from the published output
    words: v = floor(0x6627e8d5 * 8 / 2^32) = 3 (field 3, since F=6, B=2),
    BP = floor(0xe169c58d * 2 / 2^32) = 1, slot = floor(0xbc57ac4c * (len'+1) / 2^32)."""
    inst = I.make_instance("tiny", 0)
    o = oracle_mod.Oracle(inst)
    x = o.init_plan()
    p = oracle_mod.make_params(seed=0, inst_idx=0, p_swap=0.0)
    mv = o.move(p, 0, 0, x)
    assert mv[0] == 0 and mv[1] == 3 and mv[2] == 1
    tours, bps = x.to_lists()
    src = [b for b in range(2) if 3 in bps[b]][0]
    len_after = len(bps[1]) - (1 if src == 1 else 0)
    assert mv[3] == (0xBC57AC4C * (len_after + 1)) >> 32
    # with p_swap = 1 the same counter gives a swap: (0x9b00dbd8 >> 8) * 2^-24 = 0.6055 < 1
    ps = oracle_mod.make_params(seed=0, p_swap=1.0)
    mv2 = o.move(ps, 0, 0, x)
    assert mv2[0] == 2 and mv2[1] == 3 and mv2[2] == (0xE169C58D * 6) >> 32
    # and with p_swap = 0.6 it is not (0.6055 >= 0.6)
    assert o.move(oracle_mod.make_params(seed=0, p_swap=0.6), 0, 0, x)[0] == 0


def test_two_move_candidate_hand_trace(oracle_mod):
    """Step 8 repeated (Sec. 2.5's second application), traced by hand on the tiny instance,
    seed 0, candidate 0. Base: tours [[b0], [b1]], BP fields [[f0, f1], [f2, f4, f5, f3]].
    Move 0, counter (0, 0, 0, 0) = the all-zero KAT input: v = floor(0x6627e8d5 * 8 / 2^32) = 3
      (field 3, in b1 at position 3); BP = floor(0xe169c58d * 2 / 2^32) = 1; b1 has 3 fields
      left, slot = floor(0xbc57ac4c * 4 / 2^32) = 2: b1 -> [f2, f4, f3, f5].
    Move 1 is drawn on that plan from counter (0, 0, 0, 2) (word 3 = 1 is the eps rule's):
      with its output words w0..w2, v = floor(w0 * 8 / 2^32) = 6, i.e. BP 0 (in tour 0);
      tour = floor(w1 * 2 / 2^32) = 1; tour 1 holds 1 BP, slot = floor(w2 * 2 / 2^32) = 1:
      tour 0 -> [], tour 1 -> [b1, b0]."""
    inst = I.make_instance("tiny", 0)
    o = oracle_mod.Oracle(inst)
    base = o.init_plan()
    assert base.to_lists() == ([[0], [1]], [[0, 1], [2, 4, 5, 3]])
    w = [int(x) for x in oracle_mod.philox4x32_10([0, 0, 0, 2], [0, 0])]
    assert (w[0] * 8) >> 32 == 6 and (w[1] * 2) >> 32 == 1 and (w[2] * 2) >> 32 == 1
    cand, mv = o.candidate(oracle_mod.make_params(seed=0, k_moves=2), 0, 0, base)
    assert mv.tolist() == [[0, 3, 1, 2], [1, 0, 1, 1]]
    assert cand.to_lists() == ([[], [1, 0]], [[0, 1], [2, 4, 3, 5]])
    # with one move the candidate stops after move 0
    one, mv1 = o.candidate(oracle_mod.make_params(seed=0), 0, 0, base)
    assert mv1.tolist() == [[0, 3, 1, 2]] and one.to_lists() == ([[0], [1]], [[0, 1], [2, 4, 3, 5]])


def _fig1():
    """Fig. 1 as an instance: node positions read from the figure."""
    pos = {}
    for line in open(os.path.join(GOLDEN, "fig1_layout.txt")):
        if line.startswith("#") or not line.strip():
            continue
        n, x, y = line.split()
        pos[n] = (float(x), float(y))
    # node order: HQ, B1..B3, F1..F11 (BP b -> node 1+b-1, field f -> node 4+f-1)
    names = ["HQ", "B1", "B2", "B3"] + [f"F{k}" for k in range(1, 12)]
    xy = [pos[n] for n in names]
    F, B = 11, 3
    inst = I.custom_instance(xy, area=[1.0] * F, supply=[10.0] * F, demand=[1.0] * B, hu_rate=[1.0, 1.0],
                             hu_speed=40.0, su_cap=[4.0] * 4, su_fill=[0.1] * 4, su_speed=[40.0] * 4, n_tours=2)
    return inst, names


def test_fig1_edge_topology(oracle_mod):
    """The traced cost edges of the Fig. 1 plan equal the arrows of Fig. 1."""
    inst, names = _fig1()
    o = oracle_mod.Oracle(inst)
    f = lambda k: k - 1  # noqa: E731  field number in the figure -> field id
    plan = oracle_mod.Plan.from_lists(
        tours=[[1, 0], [2]],                                  # tour 1: B2 then B1; tour 2: B3
        bps=[[f(6), f(4), f(3)], [f(9), f(5), f(1), f(2)], [f(7), f(11), f(8), f(10)]])
    kinds = {0: "hu", 1: "esu", 2: "lsu", 3: "esu"}
    got = sorted((g + 1, kinds[k], names[a], names[b]) for k, a, b, g in o.trace_edges(plan))
    want = []
    for line in open(os.path.join(GOLDEN, "fig1_edges.txt")):
        if line.startswith("#") or not line.strip():
            continue
        t, k, a, b = line.split()
        want.append((int(t), k, a, b))
    assert got == sorted(want)


def _hand_one_tour():
    # HQ (0,0), BP b0 (3,0), fields f0 (0,4), f1 (3,4): a 3-4-5 layout.
    xy = [(0, 0), (3, 0), (0, 4), (3, 4)]
    return I.custom_instance(xy, area=[1.25, 1.0], supply=[50.0, 40.0], demand=[80.0], hu_rate=[2.0, 3.0],
                             hu_speed=40.0, su_cap=[10.0, 20.0, 30.0], su_fill=[0.25, 0.5, 0.75],
                             su_speed=[30.0, 40.0, 50.0], n_tours=1)


def test_cost_hand_example_one_tour(oracle_mod):
    """One tour, one BP, two fields (Sec. 2.2, Eq. 4, Eq. 6), by hand:
    HU route HQ->f0->f1->HQ = 4+3+5 = 12 km, 2 HUs;
    SU route HQ->f0 + b0->HQ = 4+3 = 7 km, 3 SUs;
    mean capacity 60/3 = 20 t: f0 ceil(50/20) = 3 drives x 2 x 5 km = 30,
                               f1 ceil(40/20) = 2 drives x 2 x 4 km = 16 (exact integer ratio);
    C = 2*12 + 3*7 + 30 + 16 = 91 km.
    T_compl = 12/40 + (1.25+1)/(2+3) = 0.75 h.
    T_wait: Dbar = (5+4)/2 = 4.5 km, critical SU = fill 0.75 ha at 50 km/h:
            2*4.5/50 - (0.25+0.5+0.75-0.75)/5 = 0.18 - 0.15 = 0.03 h."""
    o = oracle_mod.Oracle(_hand_one_tour())
    s = o.score(oracle_mod.Plan.from_lists([[0]], [[0, 1]]))
    assert s["feasible"]
    assert s["cost"] == pytest.approx(91.0, rel=1e-12)
    assert s["tmax"] == pytest.approx(0.75, rel=1e-12)
    assert s["twait"][0] == pytest.approx(0.03, abs=1e-12)
    assert list(s["n_hu"]) == [2] and list(s["n_su"]) == [3]
    assert s["tcost"][0] == pytest.approx(91.0, rel=1e-12)
    # the other field order: HQ->f1->f0->HQ = 5+3+4 = 12, SU HQ->f1 + b0->HQ = 5+3 = 8
    s2 = o.score(oracle_mod.Plan.from_lists([[0]], [[1, 0]]))
    assert s2["cost"] == pytest.approx(2 * 12 + 3 * 8 + 30 + 16, rel=1e-12)


def _hand_two_bps():
    # explicit distances; node 0 HQ, 1 b0, 2 b1, 3 f0, 4 f1, 5 f2, 6 f3
    N = 7
    d = np.full((N, N), 50.0)
    np.fill_diagonal(d, 0.0)

    def s(i, j, v):
        d[i, j] = d[j, i] = v
    s(0, 3, 10); s(3, 4, 6); s(4, 5, 1); s(5, 6, 1); s(6, 0, 12)   # HU route
    s(1, 4, 7); s(2, 0, 9)                                          # b0 -> first field of b1, b1 -> HQ
    s(3, 1, 2); s(4, 2, 4); s(5, 2, 4); s(6, 2, 4)                  # field -> own BP
    return I.custom_instance(np.zeros((N, 2)), area=[2, 3, 1, 2], supply=[25, 10, 15, 30], demand=[20, 50],
                             hu_rate=[4.0], hu_speed=30.0, su_cap=[10.0], su_fill=[0.5], su_speed=[20.0],
                             n_tours=1, dist=d)


def test_cost_hand_example_two_bps(oracle_mod):
    """One tour serving b0 (field f0) then b1 (fields f1, f2, f3), by hand:
    HU: HQ->f0->f1->f2->f3->HQ = 10+6+1+1+12 = 30 km (HUs never visit BPs);
    SU: HQ->f0 (10) + b0->f1 (7, previous BP to first field of the next BP) + b1->HQ (9) = 26 km;
    shuttles with capacity 10 t: f0 3x2x2=12, f1 1x2x4=8, f2 2x2x4=16, f3 3x2x4=24 -> 60 km;
    C = 30 + 26 + 60 = 116 km.  T_compl = 30/30 + 8/4 = 3 h.
    Mean of per-BP means (Algorithm 2, Step 1): (2 + 4)/2 = 3 km, not the field mean 3.5 km;
    T_wait = 2*3/20 - 0 = 0.3 h."""
    o = oracle_mod.Oracle(_hand_two_bps())
    s = o.score(oracle_mod.Plan.from_lists([[0, 1]], [[0], [1, 2, 3]]))
    assert s["cost"] == pytest.approx(116.0, rel=1e-12)
    assert s["tmax"] == pytest.approx(3.0, rel=1e-12)
    assert s["twait"][0] == pytest.approx(0.3, rel=1e-12)
    # Eq. 2: b0 with only f1 (10 t < 20 t) is infeasible and not evaluated
    bad = o.score(oracle_mod.Plan.from_lists([[0, 1]], [[1], [0, 2, 3]]))
    assert not bad["feasible"] and math.isinf(bad["cost"])


def _hu_trace_instance():
    # three tours with one BP and one field each, 20 km from the HQ: road time 40/40 = 1 h
    xy = [(0, 0), (20, 5), (5, 20), (-20, -5), (20, 0), (0, 20), (-20, 0)]
    return I.custom_instance(xy, area=[12.0, 30.0, 180.0], supply=[100.0] * 3, demand=[50.0] * 3,
                             hu_rate=[1, 2, 3, 4, 5, 6, 7, 8, 9], hu_speed=40.0, su_cap=[10.0] * 3,
                             su_fill=[0.25] * 3, su_speed=[40.0] * 3, n_tours=3)


def test_hu_local_min_hand_trace(oracle_mod):
    """HU assignment (Sec. 2.5; Algorithm 2 applied to HUs in rising rate order), traced by hand.
    Deal rates 1..9 round robin: t0 {1,4,7} R=12, t1 {2,5,8} R=15, t2 {3,6,9} R=18;
    T = 1 + A/R = [2, 3, 11].
    Round 1: g_max=t2, g_max2=t1, g_min=t0. Try 1: T(t2)=1+180/19=10.47 not < 3; try 4:
      9.18 not < 3; 7 is the last: accept, T(t2)=1+180/25=8.2, T(t0)=1+12/5=3.4; max 8.2 < 11 keep.
    Round 2: g_max=t2, g_max2=t0 (3.4), g_min=t1 (3). Try 2: 7.67 not < 3.4; try 5: 7 not < 3.4;
      8 last: accept, T(t2)=1+180/33=6.4545, T(t1)=1+30/7=5.2857; max 6.4545 < 8.2 keep.
    Round 3: g_max=t2, g_max2=t1, g_min=t0 {1,4}. Try 1: 6.29 not < 5.29; 4 last: accept,
      T(t0)=1+12/1=13; max 13 is not < 6.4545: undo and stop.
    Result: t0 {1,4}, t1 {2,5}, t2 {3,6,7,8,9}; Tmax = 71/11."""
    o = oracle_mod.Oracle(_hu_trace_instance())
    s = o.score(oracle_mod.Plan.from_lists([[0], [1], [2]], [[0], [1], [2]]))
    assert list(s["hu_tour"]) == [0, 1, 2, 0, 1, 2, 2, 2, 2]
    assert list(s["n_hu"]) == [2, 2, 5]
    assert s["tcompl"] == pytest.approx([3.4, 1 + 30 / 7, 71 / 11], rel=1e-12)
    assert s["tmax"] == pytest.approx(71 / 11, rel=1e-12)
    # Case 2 (fixed resources): the round-robin dealing is kept
    f = o.score(oracle_mod.Plan.from_lists([[0], [1], [2]], [[0], [1], [2]]),
                oracle_mod.make_params(fix_resources=1))
    assert list(f["hu_tour"]) == [0, 1, 2, 0, 1, 2, 0, 1, 2]


def _gaps(rows):
    return [abs(a - b) / sc for _, a, b, sc in rows]


def _check_trace(got, want, rel=1e-12):
    """The traced decision gaps equal the hand-derived ones (site, a, b, scale), as multisets."""
    key = lambda r: (r[0], round(r[1], 9), round(r[2], 9))  # noqa: E731
    g, w = sorted(got, key=key), sorted(want, key=key)
    assert [r[0] for r in g] == [r[0] for r in w], (g, w)
    for (sg, ag, bg, cg), (sw, aw, bw, cw) in zip(g, w):
        assert (ag, bg, cg) == pytest.approx((aw, bw, cw), rel=rel), (sg, (ag, bg, cg), (aw, bw, cw))


def test_hu_decision_margins_hand_trace(oracle_mod):
    """The decision gaps of the HU trace above (Algorithm 2's Steps 2, 4 and 5 applied to HUs),
    derived by hand from the same rounds. A pick's gap compares the picked tour's T with each
    competitor's, scaled by the larger of their T; an acceptance test compares T(g_max) after the
    trial move with T(g_max2), scaled by the larger; the last member of g_min is accepted without a
    test; the termination test compares the new maximum with the old one, scaled by the larger.
      R1: T = [2, 3, 11]; max t2 vs t0, t1; max2 t1 vs t0; no min competitor with 3 tours;
          trials 1, 4 (not 7, the last); stop: 8.2 vs 11.
      R2: T = [3.4, 3, 8.2]; max t2 vs t0, t1; max2 t0 vs t1; trials 2, 5; stop: 1+180/33 vs 8.2.
      R3: T = [3.4, 1+30/7, 1+180/33]; max t2 vs t0, t1; max2 t1 vs t0; trial 1; stop: 13 vs 1+180/33.
    The margin is the smallest gap: 0.4/3.4 (R2, max2)."""
    o = oracle_mod.Oracle(_hu_trace_instance())
    rows, sc = o.decision_trace(oracle_mod.Plan.from_lists([[0], [1], [2]], [[0], [1], [2]]))
    t1 = 1 + 30 / 7
    t2 = 1 + 180 / 33
    want = [
        ("hu_max", 11, 2, 11), ("hu_max", 11, 3, 11), ("hu_max2", 3, 2, 3),
        ("hu_accept", 1 + 180 / 19, 3, 1 + 180 / 19), ("hu_accept", 1 + 180 / 22, 3, 1 + 180 / 22),
        ("hu_stop", 8.2, 11, 11),
        ("hu_max", 8.2, 3.4, 8.2), ("hu_max", 8.2, 3, 8.2), ("hu_max2", 3.4, 3, 3.4),
        ("hu_accept", 1 + 180 / 27, 3.4, 1 + 180 / 27), ("hu_accept", 7, 3.4, 7),
        ("hu_stop", t2, 8.2, 8.2),
        ("hu_max", t2, 3.4, t2), ("hu_max", t2, t1, t2), ("hu_max2", t1, 3.4, t1),
        ("hu_accept", 1 + 180 / 34, t1, 1 + 180 / 34),
        ("hu_stop", 13, t2, 13),
    ]
    _check_trace(rows, want)
    assert sc["margin"] == pytest.approx(0.4 / 3.4, rel=1e-12)
    assert sc["margin"] == pytest.approx(min(_gaps(want)), rel=1e-12)


def test_hu_decision_margins_four_and_two_tours(oracle_mod):
    """The g_min pick (four tours) and the two-tour branch of the HU step, by hand.
    Four tours, 1 h of road each, areas [3, 2, 12, 8], rates 1..4 dealt one per tour:
      T = 1 + A/R = [4, 2, 5, 3]; g_max t2 vs t0, t1, t3; g_max2 t0 vs t1, t3; g_min t1 vs t3
      (scale 3); g_min keeps a single HU, so the round ends there.
    Two tours, areas [10, 40], rates 1..4 dealt round robin: t0 {1, 3} R = 4, t1 {2, 4} R = 6;
      T = [3.5, 1 + 40/6]; g_max t1 vs t0; with two tours g_min = g_max2 = t0 (no pick of its own),
      and the acceptance test compares against T(g_min) after the trial move:
      trial 1: T(t1) = 1 + 40/7 vs T(t0) = 1 + 10/3; 3 is the last: T(t0) = 11, stop: 11 vs 1 + 40/6."""
    four = I.custom_instance([(0, 0), (20, 5), (5, 20), (-20, -5), (-5, -20), (20, 0), (0, 20), (-20, 0), (0, -20)],
                             area=[3.0, 2.0, 12.0, 8.0], supply=[100.0] * 4, demand=[50.0] * 4,
                             hu_rate=[1.0, 2.0, 3.0, 4.0], hu_speed=40.0, su_cap=[10.0] * 4, su_fill=[0.25] * 4,
                             su_speed=[40.0] * 4, n_tours=4)
    o = oracle_mod.Oracle(four)
    rows, sc = o.decision_trace(oracle_mod.Plan.from_lists([[0], [1], [2], [3]], [[0], [1], [2], [3]]))
    want = [("hu_max", 5, 4, 5), ("hu_max", 5, 2, 5), ("hu_max", 5, 3, 5),
            ("hu_max2", 4, 2, 4), ("hu_max2", 4, 3, 4), ("hu_min", 2, 3, 3)]
    _check_trace(rows, want)
    assert sc["margin"] == pytest.approx(min(_gaps(want)), rel=1e-12)
    two = I.custom_instance([(0, 0), (20, 5), (5, 20), (20, 0), (0, 20)], area=[10.0, 40.0], supply=[100.0] * 2,
                            demand=[50.0] * 2, hu_rate=[1.0, 2.0, 3.0, 4.0], hu_speed=40.0, su_cap=[10.0] * 2,
                            su_fill=[0.25] * 2, su_speed=[40.0] * 2, n_tours=2)
    o2 = oracle_mod.Oracle(two)
    rows, sc = o2.decision_trace(oracle_mod.Plan.from_lists([[0], [1]], [[0], [1]]))
    want = [("hu_max", 1 + 40 / 6, 3.5, 1 + 40 / 6), ("hu_accept", 1 + 40 / 7, 1 + 10 / 3, 1 + 40 / 7),
            ("hu_stop", 11, 1 + 40 / 6, 11)]
    _check_trace(rows, want)
    assert sc["tmax"] == pytest.approx(1 + 40 / 6, rel=1e-12)
    assert sc["margin"] == pytest.approx(min(_gaps(want)), rel=1e-12)


def test_gate_decision_margin(oracle_mod):
    """The gate's gap compares Tmax with Tmax*, scaled by the larger (Sec. 2.5); without the
    gate there is no such decision. One tour: no pick, so the gate is the only decision."""
    o = oracle_mod.Oracle(_hand_one_tour())
    plan = oracle_mod.Plan.from_lists([[0]], [[0, 1]])
    rows, sc = o.decision_trace(plan, tmax_star=0.8, gate=1)
    _check_trace(rows, [("gate", 0.75, 0.8, 0.8)])
    assert sc["margin"] == pytest.approx(0.05 / 0.8, rel=1e-12)
    rows, sc = o.decision_trace(plan, tmax_star=0.7, gate=2)
    _check_trace(rows, [("gate", 0.75, 0.7, 0.75)])
    assert math.isinf(sc["cost"])
    rows, sc = o.decision_trace(plan, tmax_star=0.7, gate=0)
    assert rows == [] and math.isinf(sc["margin"])


def _su_trace_instance():
    # field-to-BP distances 15, 23.75, 60 km; SU speed 40 km/h -> round trips 0.75, 1.1875, 3 h
    xy = [(0, 0), (10, 15), (23.75, 10), (-10, -60), (10, 0), (0, 10), (-10, 0)]
    fills = [k / 8 for k in range(1, 10)]
    return I.custom_instance(xy, area=[1.0] * 3, supply=[100.0] * 3, demand=[50.0] * 3, hu_rate=[1.0] * 3,
                             hu_speed=40.0, su_cap=[10.0] * 9, su_fill=fills, su_speed=[40.0] * 9, n_tours=3)


def test_su_local_min_hand_trace(oracle_mod):
    """Algorithm 2 with Eq. 6, traced by hand (all numbers dyadic, so exact).
    One HU per tour (R = 1 ha/h). Fill areas k/8, k=1..9, dealt round robin:
      t0 {1/8,4/8,7/8} T_wait = 0.75 - (1.5-0.875) = 0.125
      t1 {2/8,5/8,8/8} T_wait = 1.1875 - 0.875 = 0.3125
      t2 {3/8,6/8,9/8} T_wait = 3 - 1.125 = 1.875
    R1: max t2, 2nd t1, min t0: 1/8 -> 1.75 no; 4/8 -> 1.375 no; 7/8 last -> t2 1.0, t0 0.625; keep.
    R2: max t2 (1.0), 2nd t0 (0.625), min t1: 2/8 -> 0.75 no; 5/8 -> t2 0.375 < 0.625 accept,
        t1 0.9375; max 0.9375 < 1.0 keep.
    R3: max t1, 2nd t0, min t2: 3/8 -> t1 0.5625 < 0.625 accept, t2 0.75; max 0.75 keep.
    R4: max t2, 2nd t0, min t1: 2/8 -> t2 0.5 < 0.625 accept, t1 0.8125; 0.8125 is not < 0.75: undo, stop.
    Result (by SU id): t0 {0,3}, t1 {1,2,7}, t2 {4,5,6,8}; T_wait = [0.625, 0.5625, 0.75]."""
    o = oracle_mod.Oracle(_su_trace_instance())
    s = o.score(oracle_mod.Plan.from_lists([[0], [1], [2]], [[0], [1], [2]]))
    assert list(s["hu_tour"]) == [0, 1, 2]
    assert list(s["su_tour"]) == [0, 1, 1, 0, 2, 2, 2, 1, 2]
    assert list(s["n_su"]) == [2, 3, 4]
    assert list(s["twait"]) == [0.625, 0.5625, 0.75]


def test_su_decision_margins_hand_trace(oracle_mod):
    """The decision gaps of the SU trace above (Algorithm 2, Eq. 6), derived by hand. The scale
    of a tour's T_wait is |drive| + |fill|, the size of the two terms Eq. 6 subtracts (T_wait can be
    near zero). A pick's gap is scaled by the larger of the two tours' scales; an acceptance test by
    the larger of the trial g_max's scale and g_max2's; the termination test by the larger of the
    new maximum's scale and the old g_max's. All values are dyadic, so they are exact.
      R1: T_wait = [1/8, 5/16, 15/8], scales [11/8, 33/16, 33/8]; trials 1/8 -> 7/4 (scale 17/4)
          and 4/8 -> 11/8 (37/8) against 5/16; stop: 1 (scale 5) vs 15/8.
      R2: [5/8, 5/16, 1], scales [7/8, 33/16, 5]; trials 2/8 -> 3/4 (21/4), 5/8 -> 3/8 (45/8)
          against 5/8; stop: 15/16 (23/16) vs 1 (5).
      R3: [5/8, 15/16, 3/8], scales [7/8, 23/16, 45/8]; max t1; trial 3/8 -> 9/16 (29/16) against
          5/8; stop: 3/4 (21/4) vs 15/16 (23/16).
      R4: [5/8, 9/16, 3/4], scales [7/8, 29/16, 21/4]; trial 2/8 -> 1/2 (11/2) against 5/8;
          stop: 13/16 (25/16) vs 3/4 (21/4): not lower, undone.
    The HU step has three equal completion times (1.5 h each): ties, so no gap.
    The margin is the smallest gap: (1/16)/(21/4) (R4, stop)."""
    o = oracle_mod.Oracle(_su_trace_instance())
    rows, sc = o.decision_trace(oracle_mod.Plan.from_lists([[0], [1], [2]], [[0], [1], [2]]))
    want = [
        ("su_max", 15 / 8, 1 / 8, 33 / 8), ("su_max", 15 / 8, 5 / 16, 33 / 8), ("su_max2", 5 / 16, 1 / 8, 33 / 16),
        ("su_accept", 7 / 4, 5 / 16, 17 / 4), ("su_accept", 11 / 8, 5 / 16, 37 / 8), ("su_stop", 1, 15 / 8, 5),
        ("su_max", 1, 5 / 8, 5), ("su_max", 1, 5 / 16, 5), ("su_max2", 5 / 8, 5 / 16, 33 / 16),
        ("su_accept", 3 / 4, 5 / 8, 21 / 4), ("su_accept", 3 / 8, 5 / 8, 45 / 8), ("su_stop", 15 / 16, 1, 5),
        ("su_max", 15 / 16, 5 / 8, 23 / 16), ("su_max", 15 / 16, 3 / 8, 45 / 8), ("su_max2", 5 / 8, 3 / 8, 45 / 8),
        ("su_accept", 9 / 16, 5 / 8, 29 / 16), ("su_stop", 3 / 4, 15 / 16, 21 / 4),
        ("su_max", 3 / 4, 5 / 8, 21 / 4), ("su_max", 3 / 4, 9 / 16, 21 / 4), ("su_max2", 5 / 8, 9 / 16, 29 / 16),
        ("su_accept", 1 / 2, 5 / 8, 11 / 2), ("su_stop", 13 / 16, 3 / 4, 21 / 4),
    ]
    _check_trace(rows, want, rel=0)
    assert sc["margin"] == (1 / 16) / (21 / 4)
    assert sc["margin"] == min(_gaps(want))


def test_init_hand_trace(oracle_mod):
    """Algorithm 1, Steps 1-3, traced by hand.
    BPs b0 (10,0), b1 (-10,0), b2 (0,30); both b0 and b1 are 10 km from the HQ -> tie to b0;
    then b1 (20 km), then b2: chain [b0, b1, b2], cut for 2 tours into [b0] and [b1, b2].
    Fields in id order (demand 100 t each): f0 (12,1) 60 t -> b0; f1 (-12,1) 120 t -> b1 (met);
    f2 (1,28) 150 t -> b2 (met); f3 (-9,1) 50 t -> b0, the only BP still short although b1 is
    closer; f4 (9,3) -> every BP met, so the closest, b0.
    Order of b0's fields from the HQ: f3 (9.06 km), then from f3: f4 (18.1) before f0 (21)."""
    xy = [(0, 0), (10, 0), (-10, 0), (0, 30), (12, 1), (-12, 1), (1, 28), (-9, 1), (9, 3)]
    inst = I.custom_instance(xy, area=[1.0] * 5, supply=[60, 120, 150, 50, 30], demand=[100] * 3,
                             hu_rate=[1.0, 1.0], hu_speed=40.0, su_cap=[10.0] * 2, su_fill=[0.25] * 2,
                             su_speed=[40.0] * 2, n_tours=2)
    o = oracle_mod.Oracle(inst)
    tours, bps = o.init_plan().to_lists()
    assert tours == [[0], [1, 2]]
    assert bps == [[3, 4, 0], [1], [2]]


def test_gate_rule(oracle_mod):
    """Completion-time gate (Sec. 2.5): gate 1 discards Tmax > Tmax*, gate 2 also Tmax == Tmax*."""
    o = oracle_mod.Oracle(_hand_one_tour())
    plan = oracle_mod.Plan.from_lists([[0]], [[0, 1]])
    assert o.score(plan, tmax_star=0.75, gate=1)["cost"] == pytest.approx(91.0)
    assert math.isinf(o.score(plan, tmax_star=0.75, gate=2)["cost"])
    assert math.isinf(o.score(plan, tmax_star=0.7, gate=1)["cost"])
    assert o.score(plan, tmax_star=0.7, gate=0)["cost"] == pytest.approx(91.0)


def test_replica_magnitudes_table3(oracle_mod):
    """Case 1 of Table 3 (10 random replicas of Sec. 3.1 with the Table 1 fleet, 1 HU and
    2 small + 4 large SUs per tour): mean cost 461,048.6 km, mean completion time 360.9 h,
    mean worst completion time 411.3 h, waiting times of tenths of an hour. The paper's
    instances are unseeded, so only the magnitudes are compared (cost within 10 %,
    completion times within 5 %)."""
    costs, avg, worst, wait = [], [], [], []
    for seed in range(10):
        inst = I.make_instance("replica", seed)
        o = oracle_mod.Oracle(inst)
        s = o.score(o.init_plan(), oracle_mod.make_params(fix_resources=1))
        assert s["feasible"]
        assert list(s["n_hu"]) == [1] * 7 and list(s["n_su"]) == [6] * 7
        costs.append(s["cost"]); avg.append(s["tcompl"].mean()); worst.append(s["tcompl"].max())
        wait.append(np.abs(s["twait"]).max())
    assert np.mean(costs) == pytest.approx(461048.6, rel=0.10)
    assert np.mean(avg) == pytest.approx(360.9, rel=0.05)
    assert np.mean(worst) == pytest.approx(411.3, rel=0.05)
    assert max(wait) < 1.5
