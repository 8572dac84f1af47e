"""Python front of the CPU oracle (``biolog_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg use it. The product path never imports this module, and this
module imports nothing from the product package. Instances are taken by duck
typing (any object with the fields of an instance record).

Every function here only marshals arguments; the arithmetic lives in the C
file, in FP64, following the paper passage named at each C function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "biolog_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

i16p = np.ctypeslib.ndpointer(dtype=np.int16, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with the system C compiler (plain C11 + OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-std=gnu11", "-O2", "-fPIC", "-shared", "-fopenmp", "-Wall", "-Wno-unused-variable",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _InstIn(C.Structure):
    _fields_ = [("F", C.c_int32), ("B", C.c_int32), ("T", C.c_int32), ("H", C.c_int32), ("S", C.c_int32),
                ("xy", C.c_void_p), ("dist", C.c_void_p), ("area", C.c_void_p), ("supply", C.c_void_p),
                ("demand", C.c_void_p), ("hu_rate", C.c_void_p), ("hu_speed", C.c_float),
                ("su_cap", C.c_void_p), ("su_fill", C.c_void_p), ("su_speed", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("p_swap", C.c_double), ("seed", C.c_uint64), ("inst_idx", C.c_uint32),
                ("fix_field_bp", C.c_int32), ("fix_resources", C.c_int32), ("gate", C.c_int32),
                ("k_moves", C.c_int32)]


class _Score(C.Structure):
    _fields_ = [("feasible", C.c_int), ("cost", C.c_double), ("tmax", C.c_double), ("margin", C.c_double),
                ("ops", C.c_double)]


class _Gap(C.Structure):
    _fields_ = [("site", C.c_int32), ("pad", C.c_int32), ("a", C.c_double), ("b", C.c_double),
                ("scale", C.c_double)]


# decision sites of the gap trace (the C file's GAP_* numbering)
GAP_SITES = {1: "hu_max", 2: "hu_max2", 3: "hu_min", 4: "hu_accept", 5: "hu_stop",
             6: "su_max", 7: "su_max2", 8: "su_min", 9: "su_accept", 10: "su_stop", 11: "gate"}


class _State(C.Structure):
    _fields_ = [("xold_bp_order", C.c_void_p), ("xold_tour_cnt", C.c_void_p), ("xold_field_order", C.c_void_p),
                ("xold_bp_cnt", C.c_void_p), ("xbest_bp_order", C.c_void_p), ("xbest_tour_cnt", C.c_void_p),
                ("xbest_field_order", C.c_void_p), ("xbest_bp_cnt", C.c_void_p), ("cstar", C.c_double),
                ("tmaxstar", C.c_double), ("iter", C.c_uint32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB lets the mutation test load a deliberately broken copy
            path = os.environ.get("ORACLE_LIB") or build()
            L = C.CDLL(path)
            L.or_new.restype = C.c_void_p
            L.or_new.argtypes = [C.POINTER(_InstIn), C.c_char_p, C.c_int]
            L.or_free.argtypes = [C.c_void_p]
            L.or_philox4x32_10.argtypes = [np.ctypeslib.ndpointer(np.uint32), np.ctypeslib.ndpointer(np.uint32),
                                           np.ctypeslib.ndpointer(np.uint32)]
            L.or_init_plan.argtypes = [C.c_void_p, i16p, i16p, i16p, i16p]
            L.or_move.argtypes = [C.c_void_p, C.POINTER(Params), C.c_uint32, C.c_uint32, i16p, i16p, i16p, i16p, i16p]
            L.or_apply.argtypes = [C.c_void_p, i16p, i16p, i16p, i16p, i16p, i16p, i16p, i16p, i16p]
            L.or_candidate.argtypes = [C.c_void_p, C.POINTER(Params), C.c_uint32, C.c_uint32, i16p, i16p, i16p, i16p,
                                       i16p, i16p, i16p, i16p, i16p]
            L.or_score_plan.argtypes = [C.c_void_p, C.POINTER(Params), i16p, i16p, i16p, i16p, C.c_double, C.c_int32,
                                        C.POINTER(_Score), i32p, i32p, f64p, f64p, f64p, i32p, i32p]
            L.or_score_plan_trace.argtypes = [C.c_void_p, C.POINTER(Params), i16p, i16p, i16p, i16p, C.c_double,
                                              C.c_int32, C.POINTER(_Score), C.c_void_p, C.c_int32]
            L.or_trace_edges.argtypes = [C.c_void_p, i16p, i16p, i16p, i16p, i32p, i32p, i32p, i32p, C.c_int32]
            L.or_eps_select.argtypes = [C.POINTER(Params), C.c_uint32]
            L.or_validate_enc.argtypes = [C.c_int, C.c_int, C.c_int, i16p, i16p, i16p, i16p]
            vp = C.c_void_p
            L.or_score_batch.argtypes = [C.c_void_p, C.POINTER(Params), C.c_uint32, i16p, i16p, i16p, i16p,
                                         C.c_double, C.c_int32, C.c_int32, C.c_int32, vp, vp, vp, vp, vp, vp, vp, vp,
                                         vp, vp]
            L.or_search.argtypes = [C.c_void_p, C.POINTER(Params), C.POINTER(_State), C.c_int32, C.c_int32, C.c_int32,
                                    vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
            L.or_max_threads.restype = C.c_int
            _lib = L
    return _lib


def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, dtype=np.uint32), np.asarray(key, dtype=np.uint32), out)
    return out


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class Plan:
    """Plan encoding (Sec. 2.4): BP order by tour, BPs per tour, field order grouped by BP id, fields per BP."""

    def __init__(self, bp_order, tour_cnt, field_order, bp_cnt):
        self.bp_order = np.ascontiguousarray(bp_order, dtype=np.int16)
        self.tour_cnt = np.ascontiguousarray(tour_cnt, dtype=np.int16)
        self.field_order = np.ascontiguousarray(field_order, dtype=np.int16)
        self.bp_cnt = np.ascontiguousarray(bp_cnt, dtype=np.int16)

    def arrays(self):
        return self.bp_order, self.tour_cnt, self.field_order, self.bp_cnt

    def copy(self):
        return Plan(*(a.copy() for a in self.arrays()))

    def __eq__(self, other):
        return all(np.array_equal(a, b) for a, b in zip(self.arrays(), other.arrays()))

    @classmethod
    def from_lists(cls, tours, bps):
        """tours: list of BP-id lists per tour; bps: list of field-id lists per BP id."""
        bp_order = [b for t in tours for b in t]
        field_order = [f for fl in bps for f in fl]
        return cls(bp_order, [len(t) for t in tours], field_order, [len(fl) for fl in bps])

    def to_lists(self):
        tours, k = [], 0
        for n in self.tour_cnt:
            tours.append([int(x) for x in self.bp_order[k:k + n]]); k += n
        bps, k = [], 0
        for n in self.bp_cnt:
            bps.append([int(x) for x in self.field_order[k:k + n]]); k += n
        return tours, bps


def make_params(eps=0.5, seed=0, inst_idx=0, fix_field_bp=0, fix_resources=0, gate=1, p_swap=0.0,
                k_moves=1) -> Params:
    assert 1 <= k_moves <= 8
    return Params(float(np.float32(eps)), float(np.float32(p_swap)), int(seed), int(inst_idx), int(fix_field_bp),
                  int(fix_resources), int(gate), int(k_moves))


class Oracle:
    """FP64 model of one instance."""

    def __init__(self, inst):
        self.inst = inst
        self.F, self.B, self.T, self.H, self.S = inst.n_fields, inst.n_bps, inst.n_tours, inst.n_hu, inst.n_su
        self._keep = [np.ascontiguousarray(a, dtype=np.float32) for a in (
            inst.xy, inst.area_ha, inst.supply_t, inst.demand_t, inst.hu_rate_ha_h, inst.su_cap_t,
            inst.su_fill_ha, inst.su_speed_kmh)]
        xy, area, sup, dem, hur, cap, fill, spd = self._keep
        dist = getattr(inst, "dist", None)
        if dist is not None:
            dist = np.ascontiguousarray(dist, dtype=np.float32)
            self._keep.append(dist)
        s = _InstIn(self.F, self.B, self.T, self.H, self.S, _p(xy), _p(dist), _p(area), _p(sup), _p(dem), _p(hur),
                    float(inst.hu_speed_kmh), _p(cap), _p(fill), _p(spd))
        err = C.create_string_buffer(256)
        self._h = lib().or_new(C.byref(s), err, 256)
        if not self._h:
            raise ValueError("oracle: " + err.value.decode())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_free(h)
            self._h = None

    # -- Algorithm 1, Steps 1-3
    def init_plan(self) -> Plan:
        p = Plan(np.zeros(self.B), np.zeros(self.T), np.zeros(self.F), np.zeros(self.B))
        lib().or_init_plan(self._h, *p.arrays())
        return p

    def validate(self, plan: Plan) -> int:
        return lib().or_validate_enc(self.T, self.B, self.F, *plan.arrays())

    # -- Step 8
    def move(self, params: Params, iter_: int, i: int, base: Plan) -> np.ndarray:
        mv = np.zeros(4, dtype=np.int16)
        rc = lib().or_move(self._h, C.byref(params), iter_, i, *base.arrays(), mv)
        if rc:
            raise ValueError("bad plan")
        return mv

    def candidate(self, params: Params, iter_: int, i: int, base: Plan):
        """Candidate i (Step 8 applied params.k_moves times): its plan and its k x 4 move records."""
        k = max(1, params.k_moves)
        mv = np.zeros(4 * k, dtype=np.int16)
        out = Plan(np.zeros(self.B), np.zeros(self.T), np.zeros(self.F), np.zeros(self.B))
        rc = lib().or_candidate(self._h, C.byref(params), iter_, i, *base.arrays(), mv, *out.arrays())
        if rc:
            raise ValueError("bad plan")
        return out, mv.reshape(k, 4)

    def apply(self, base: Plan, mv) -> Plan:
        out = Plan(np.zeros(self.B), np.zeros(self.T), np.zeros(self.F), np.zeros(self.B))
        rc = lib().or_apply(self._h, *base.arrays(), np.ascontiguousarray(mv, dtype=np.int16), *out.arrays())
        if rc:
            raise ValueError("bad plan")
        return out

    # -- scoring (Sec. 2.2, 2.5)
    def score(self, plan: Plan, params: Params | None = None, tmax_star=np.inf, gate=0) -> dict:
        params = params or make_params()
        T, H, S = self.T, self.H, self.S
        r = _Score()
        n_hu = np.zeros(T, np.int32); n_su = np.zeros(T, np.int32)
        tc = np.zeros(T); tw = np.zeros(T); tcost = np.zeros(T)
        hu = np.zeros(H, np.int32); su = np.zeros(S, np.int32)
        rc = lib().or_score_plan(self._h, C.byref(params), *plan.arrays(), float(tmax_star), int(gate), C.byref(r),
                                 n_hu, n_su, tc, tw, tcost, hu, su)
        if rc:
            raise ValueError("bad plan")
        return dict(feasible=bool(r.feasible), cost=r.cost, tmax=r.tmax, margin=r.margin, ops=r.ops,
                    n_hu=n_hu, n_su=n_su, tcompl=tc, twait=tw, tcost=tcost, hu_tour=hu, su_tour=su)

    def decision_trace(self, plan: Plan, params: Params | None = None, tmax_star=np.inf, gate=0, cap=4096):
        """Every decision gap the score of `plan` counts, in order: (site, a, b, scale), where the
        site names the decision (GAP_SITES) and |a - b| / scale is its relative gap; plus the score."""
        params = params or make_params()
        buf = (_Gap * cap)()
        r = _Score()
        n = lib().or_score_plan_trace(self._h, C.byref(params), *plan.arrays(), float(tmax_star), int(gate),
                                      C.byref(r), C.cast(buf, C.c_void_p), int(cap))
        if n < 0:
            raise ValueError("bad plan")
        if n > cap:
            raise ValueError("trace longer than cap")
        rows = [(GAP_SITES[buf[k].site], buf[k].a, buf[k].b, buf[k].scale) for k in range(n)]
        return rows, dict(feasible=bool(r.feasible), cost=r.cost, tmax=r.tmax, margin=r.margin)

    def trace_edges(self, plan: Plan):
        cap = 8 * (self.F + self.B + self.T) + 16
        k = np.zeros(cap, np.int32); a = np.zeros(cap, np.int32); b = np.zeros(cap, np.int32); g = np.zeros(cap, np.int32)
        n = lib().or_trace_edges(self._h, *plan.arrays(), k, a, b, g, cap)
        return [(int(k[j]), int(a[j]), int(b[j]), int(g[j])) for j in range(n)]

    def score_batch(self, params: Params, iter_: int, base: Plan, n: int, tmax_star=np.inf, i0=0, threads=1,
                    details=False) -> dict:
        cost = np.zeros(n); tmax = np.zeros(n); margin = np.zeros(n); feas = np.zeros(n, np.int32)
        moves = np.zeros((n, 4 * max(1, params.k_moves)), np.int16)
        n_hu = np.zeros((n, self.T), np.int32) if details else None
        n_su = np.zeros((n, self.T), np.int32) if details else None
        hu = np.zeros((n, self.H), np.int32) if details else None
        su = np.zeros((n, self.S), np.int32) if details else None
        ops = C.c_double(0.0)
        rc = lib().or_score_batch(self._h, C.byref(params), iter_, *base.arrays(), float(tmax_star), int(i0), int(n),
                                  int(threads), _p(cost), _p(tmax), _p(margin), _p(feas), _p(moves), _p(n_hu),
                                  _p(n_su), _p(hu), _p(su), C.cast(C.pointer(ops), C.c_void_p))
        if rc:
            raise ValueError("bad plan")
        out = dict(cost=cost, tmax=tmax, margin=margin, feasible=feas.astype(bool), moves=moves, ops=ops.value)
        if details:
            out.update(n_hu=n_hu, n_su=n_su, hu_tour=hu, su_tour=su)
        return out

    def eps_select(self, params: Params, iter_: int) -> bool:
        return bool(lib().or_eps_select(C.byref(params), iter_))

    # -- Algorithm 1, Steps 5-16
    def search(self, params: Params, state: "SearchState", n_iters: int, n_cand: int, threads=1,
               force_istar=None) -> dict:
        st = _State(*[_p(a) for a in state.xold.arrays()], *[_p(a) for a in state.xbest.arrays()],
                    float(state.cstar), float(state.tmaxstar), int(state.iter))
        use_best = np.zeros(n_iters, np.int32); istar = np.zeros(n_iters, np.int32)
        c_istar = np.zeros(n_iters); cstar = np.zeros(n_iters); tstar = np.zeros(n_iters)
        ind = np.zeros(n_iters, np.int32); mbest = np.zeros(n_iters); gap = np.zeros(n_iters)
        follow = np.zeros(n_iters)
        force = None
        if force_istar is not None:
            force = np.ascontiguousarray(force_istar, dtype=np.int32)
        rc = lib().or_search(self._h, C.byref(params), C.byref(st), int(n_iters), int(n_cand), int(threads),
                             _p(use_best), _p(istar), _p(c_istar), _p(cstar), _p(tstar), _p(ind), _p(mbest), _p(gap),
                             _p(force), _p(follow))
        if rc:
            raise ValueError("bad state")
        state.cstar, state.tmaxstar, state.iter = st.cstar, st.tmaxstar, st.iter
        return dict(use_best=use_best.astype(bool), istar=istar, c_istar=c_istar, cstar=cstar, tmaxstar=tstar,
                    indicator=ind, margin_best=mbest, gap=gap, c_follow=follow)

    def start(self, params: Params | None = None) -> "SearchState":
        """Algorithm 1, Step 4: x* = x_old = initial plan, C* and Tmax* from the scorer (no gate)."""
        x = self.init_plan()
        s = self.score(x, params, gate=0)
        return SearchState(x.copy(), x.copy(), s["cost"], s["tmax"], 0)


class SearchState:
    def __init__(self, xold: Plan, xbest: Plan, cstar: float, tmaxstar: float, iter_: int):
        self.xold, self.xbest, self.cstar, self.tmaxstar, self.iter = xold, xbest, cstar, tmaxstar, iter_

    def copy(self):
        return SearchState(self.xold.copy(), self.xbest.copy(), self.cstar, self.tmaxstar, self.iter)


def max_threads() -> int:
    return int(lib().or_max_threads())
