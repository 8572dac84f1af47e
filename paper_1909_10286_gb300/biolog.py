"""Python binding of the C ABI in ``include/biolog.h`` (argument marshalling only).

Every step of the search runs in the CUDA library ``_lib/libbiolog.so``; this
module converts numpy arrays and torch streams/buffers to the plain pointers
the ABI takes. There is no fallback: if the library is missing or no CUDA
device is present, the calls raise.

PyTorch supplies the device memory (the workspace is a torch uint8 tensor,
so it comes from torch's caching allocator) and the stream.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbiolog.so")
_lib = None
_lock = threading.Lock()

BL_OK, BL_EINVAL, BL_EINFEASIBLE_INSTANCE, BL_ETOO_LARGE, BL_ECUDA, BL_ETIMEOUT, BL_ESTATE = 0, -1, -2, -3, -4, -5, -6
EXPORTS = ("bl_workspace_bytes", "bl_plan_init", "bl_plan_init_batch", "bl_search_step", "bl_best_plan",
           "bl_get_state", "bl_set_state", "bl_get_log", "bl_score_candidates", "bl_decode_candidates",
           "bl_get_config", "bl_plan_free", "bl_last_error", "bl_global_error", "bl_argmin_noalloc", "bl_wait_selftest",
           "bl_search_step_inspect", "bl_search_score_slice", "bl_search_apply", "bl_get_states", "bl_set_states",
           "bl_mlp_create", "bl_mlp_forward", "bl_mlp_grads", "bl_mlp_train_step", "bl_mlp_get", "bl_mlp_set",
           "bl_mlp_free", "bl_mlp_last_error", "bl_gemm_bf16", "bl_features", "bl_search_step_learned",
           "bl_mlp_train_step_sampled")


class BiologError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"biolog error {code}: {msg}")
        self.code = code


class bl_instance(C.Structure):
    _fields_ = [("n_fields", C.c_int32), ("n_bps", C.c_int32), ("n_tours", C.c_int32), ("n_hu", C.c_int32),
                ("n_su", C.c_int32), ("xy", C.c_void_p), ("dist", C.c_void_p), ("area_ha", C.c_void_p),
                ("supply_t", C.c_void_p), ("demand_t", C.c_void_p), ("hu_rate_ha_h", C.c_void_p),
                ("hu_speed_kmh", C.c_float), ("su_cap_t", C.c_void_p), ("su_fill_ha", C.c_void_p),
                ("su_speed_kmh", C.c_void_p)]


class bl_params(C.Structure):
    _fields_ = [("eps", C.c_float), ("p_swap", C.c_float), ("seed", C.c_uint64), ("inst_idx", C.c_uint32),
                ("n_cand", C.c_int32), ("fix_field_bp", C.c_int32), ("fix_resources", C.c_int32),
                ("gate", C.c_int32), ("block_threads", C.c_int32), ("blocks_per_sm", C.c_int32), ("tile", C.c_int32),
                ("log_capacity", C.c_int32), ("lanes_per_cand", C.c_int32), ("k_moves", C.c_int32),
                ("cand_offset", C.c_uint32), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t)]


class bl_plan(C.Structure):
    _fields_ = [("bp_order", C.c_void_p), ("tour_cnt", C.c_void_p), ("field_order", C.c_void_p),
                ("bp_cnt", C.c_void_p), ("hu_tour", C.c_void_p), ("su_tour", C.c_void_p),
                ("tour_cost_km", C.c_void_p), ("tour_tcompl_h", C.c_void_p), ("tour_twait_h", C.c_void_p),
                ("tour_n_hu", C.c_void_p), ("tour_n_su", C.c_void_p), ("cost_km", C.c_float), ("tmax_h", C.c_float),
                ("iter", C.c_uint32)]


class bl_state(C.Structure):
    _fields_ = [("xold_bp_order", C.c_void_p), ("xold_tour_cnt", C.c_void_p), ("xold_field_order", C.c_void_p),
                ("xold_bp_cnt", C.c_void_p), ("xbest_bp_order", C.c_void_p), ("xbest_tour_cnt", C.c_void_p),
                ("xbest_field_order", C.c_void_p), ("xbest_bp_cnt", C.c_void_p), ("cstar", C.c_float),
                ("tmaxstar", C.c_float), ("iter", C.c_uint32)]


def load(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise BiologError(BL_ESTATE, f"CUDA library not built: {p} (run paper_1909_10286_gb300.build.build())")
            L = C.CDLL(p)
            vp = C.c_void_p
            L.bl_workspace_bytes.argtypes = [C.POINTER(bl_instance), C.c_int32, C.POINTER(bl_params),
                                             C.POINTER(C.c_size_t)]
            L.bl_plan_init.argtypes = [C.POINTER(bl_instance), C.POINTER(bl_params), vp, C.POINTER(vp)]
            L.bl_plan_init_batch.argtypes = [C.POINTER(bl_instance), C.c_int32, C.POINTER(bl_params), vp, C.POINTER(vp)]
            L.bl_search_step.argtypes = [vp, C.c_int32]
            L.bl_search_step_inspect.argtypes = [vp, vp, C.c_int32]
            L.bl_search_score_slice.argtypes = [vp, vp]
            L.bl_search_apply.argtypes = [vp, vp]
            L.bl_best_plan.argtypes = [vp, C.c_int32, C.POINTER(bl_plan)]
            L.bl_get_state.argtypes = [vp, C.c_int32, C.POINTER(bl_state)]
            L.bl_set_state.argtypes = [vp, C.c_int32, C.POINTER(bl_state)]
            L.bl_get_states.argtypes = [vp, vp]
            L.bl_set_states.argtypes = [vp, vp]
            L.bl_get_log.argtypes = [vp, C.c_int32, C.c_uint32, C.c_int32, vp, vp, vp, vp, vp]
            L.bl_score_candidates.argtypes = [vp, C.c_int32, C.c_int32, C.c_uint32, C.c_float, C.c_int32, C.c_int32,
                                              vp, vp, vp, vp, vp, vp, vp]
            L.bl_decode_candidates.argtypes = [vp, C.c_int32, C.c_int32, C.c_uint32, vp, C.c_int32, vp]
            L.bl_get_config.argtypes = [vp, vp, vp, vp, vp, vp]
            L.bl_wait_selftest.argtypes = [vp, C.c_uint64, C.POINTER(C.c_uint64)]
            L.bl_argmin_noalloc.argtypes = [vp, C.c_int32, C.c_int32, C.c_uint32, C.c_float, C.c_int32, C.c_int32,
                                            vp, vp]
            L.bl_features.argtypes = [vp, C.c_int32, C.c_int32, C.c_uint32, C.c_int32, C.c_int32, vp, vp]
            L.bl_search_step_learned.argtypes = [vp, vp, C.c_int32, C.c_int32, C.c_int32, C.c_float]
            L.bl_plan_free.argtypes = [vp]
            L.bl_last_error.argtypes = [vp]
            L.bl_last_error.restype = C.c_char_p
            L.bl_global_error.restype = C.c_char_p
            _lib = L
    return _lib


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


class _InstanceArgs:
    """Keeps the numpy buffers of one bl_instance alive."""

    def __init__(self, inst):
        self.arrays = [_f32(inst.xy), _f32(inst.area_ha), _f32(inst.supply_t), _f32(inst.demand_t),
                       _f32(inst.hu_rate_ha_h), _f32(inst.su_cap_t), _f32(inst.su_fill_ha), _f32(inst.su_speed_kmh)]
        xy, area, sup, dem, hur, cap, fill, spd = self.arrays
        dist = getattr(inst, "dist", None)
        if dist is not None:
            dist = _f32(dist)
            self.arrays.append(dist)
        self.s = bl_instance(inst.n_fields, inst.n_bps, inst.n_tours, inst.n_hu, inst.n_su, _p(xy), _p(dist),
                             _p(area), _p(sup), _p(dem), _p(hur), float(inst.hu_speed_kmh), _p(cap), _p(fill), _p(spd))


def make_params(n_cand: int, eps: float = 0.5, seed: int = 0, inst_idx: int = 0, fix_field_bp: int = 0,
                fix_resources: int = 0, gate: int = 1, p_swap: float = 0.0, block_threads: int = 0,
                blocks_per_sm: int = 0, tile: int = 0, log_capacity: int = 0, lanes_per_cand: int = 0,
                k_moves: int = 1, cand_offset: int = 0) -> bl_params:
    return bl_params(float(eps), float(p_swap), int(seed), int(inst_idx), int(n_cand), int(fix_field_bp),
                     int(fix_resources), int(gate), int(block_threads), int(blocks_per_sm), int(tile),
                     int(log_capacity), int(lanes_per_cand), int(k_moves), int(cand_offset), None, 0)


def _check(rc: int, handle=None):
    if rc != BL_OK:
        L = load()
        msg = (L.bl_last_error(handle) if handle else L.bl_global_error()) or b""
        raise BiologError(rc, msg.decode())


def workspace_bytes(instances, params: bl_params) -> int:
    args = [_InstanceArgs(i) for i in instances]
    arr = (bl_instance * len(args))(*[a.s for a in args])
    n = C.c_size_t(0)
    _check(load().bl_workspace_bytes(arr, len(args), C.byref(params), C.byref(n)))
    return int(n.value)


class Search:
    """One handle of the library: a batch of instances searched together."""

    def __init__(self, instances, params: bl_params, stream=None, torch_workspace: bool = True):
        import torch  # device memory and streams only

        if not torch.cuda.is_available():
            raise BiologError(BL_ESTATE, "no CUDA device: the search runs only on the GPU")
        self.instances = list(instances)
        self._args = [_InstanceArgs(i) for i in self.instances]
        arr = (bl_instance * len(self._args))(*[a.s for a in self._args])
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        prm = bl_params.from_buffer_copy(params)
        self._ws = None
        if torch_workspace:
            nbytes = workspace_bytes(self.instances, params)
            self._ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            prm.workspace = C.c_void_p(self._ws.data_ptr())
            prm.workspace_bytes = nbytes
        self.params = prm
        h = C.c_void_p()
        L = load()
        if len(self._args) == 1:
            rc = L.bl_plan_init(arr, C.byref(prm), C.c_void_p(self._stream.cuda_stream), C.byref(h))
        else:
            rc = L.bl_plan_init_batch(arr, len(self._args), C.byref(prm), C.c_void_p(self._stream.cuda_stream),
                                      C.byref(h))
        _check(rc)
        self.h = h
        self._states_c = None   # (array ids, ctypes bl_state array, the arrays) of the last packed transfer

    # --- the three calls of the paper's loop
    def search_step(self, n_iters: int):
        _check(load().bl_search_step(self.h, int(n_iters)), self.h)

    def score_slice(self, d_key_ptr: int):
        """bl_search_score_slice: this handle's slice of the iteration, its argmin key into 8 bytes of device
        memory at d_key_ptr (e.g. an int64 CUDA tensor's data_ptr())."""
        _check(load().bl_search_score_slice(self.h, C.c_void_p(d_key_ptr)), self.h)

    def apply(self, d_key_ptr: int):
        """bl_search_apply: Steps 13-16 with the iteration's reduced argmin key (device memory)."""
        _check(load().bl_search_apply(self.h, C.c_void_p(d_key_ptr)), self.h)

    def search_step_inspect(self, out, stride: int):
        """bl_search_step_inspect: one iteration of the search kernel that also writes {C_i, Tmax_i}
        per candidate into `out`, a caller-owned float32 CUDA tensor of >= 2 * n_inst * stride values."""
        assert out.is_cuda and out.dtype.itemsize == 4 and out.numel() >= 2 * len(self.instances) * stride
        _check(load().bl_search_step_inspect(self.h, C.c_void_p(out.data_ptr()), int(stride)), self.h)

    def best_plan(self, inst: int = 0) -> dict:
        I = self.instances[inst]
        B, T, F, H, S = I.n_bps, I.n_tours, I.n_fields, I.n_hu, I.n_su
        o = dict(bp_order=np.zeros(B, np.int16), tour_cnt=np.zeros(T, np.int16), field_order=np.zeros(F, np.int16),
                 bp_cnt=np.zeros(B, np.int16), hu_tour=np.zeros(H, np.int16), su_tour=np.zeros(S, np.int16),
                 tour_cost_km=np.zeros(T, np.float32), tour_tcompl_h=np.zeros(T, np.float32),
                 tour_twait_h=np.zeros(T, np.float32), tour_n_hu=np.zeros(T, np.int16),
                 tour_n_su=np.zeros(T, np.int16))
        p = bl_plan(*[_p(o[k]) for k in ("bp_order", "tour_cnt", "field_order", "bp_cnt", "hu_tour", "su_tour",
                                         "tour_cost_km", "tour_tcompl_h", "tour_twait_h", "tour_n_hu",
                                         "tour_n_su")], 0.0, 0.0, 0)
        _check(load().bl_best_plan(self.h, int(inst), C.byref(p)), self.h)
        o.update(cost_km=p.cost_km, tmax_h=p.tmax_h, iter=p.iter)
        return o

    def get_state(self, inst: int = 0) -> dict:
        I = self.instances[inst]
        B, T, F = I.n_bps, I.n_tours, I.n_fields
        a = [np.zeros(n, np.int16) for n in (B, T, F, B, B, T, F, B)]
        s = bl_state(*[_p(x) for x in a], 0.0, 0.0, 0)
        _check(load().bl_get_state(self.h, int(inst), C.byref(s)), self.h)
        return dict(xold=tuple(a[:4]), xbest=tuple(a[4:]), cstar=s.cstar, tmaxstar=s.tmaxstar, iter=s.iter)

    def set_state(self, state: dict, inst: int = 0):
        a = [np.ascontiguousarray(x, dtype=np.int16) for x in (*state["xold"], *state["xbest"])]
        s = bl_state(*[_p(x) for x in a], float(state["cstar"]), float(state["tmaxstar"]), int(state["iter"]))
        _check(load().bl_set_state(self.h, int(inst), C.byref(s)), self.h)

    def _state_arrays(self):
        out = []
        for I in self.instances:
            B, T, F = I.n_bps, I.n_tours, I.n_fields
            a = [np.zeros(n, np.int16) for n in (B, T, F, B, B, T, F, B)]
            out.append(dict(xold=tuple(a[:4]), xbest=tuple(a[4:]), cstar=0.0, tmaxstar=0.0, iter=0))
        return out

    def _states_struct(self, arrays):
        """The ctypes bl_state array pointing at `arrays` (per instance: x_old's four, then x*'s four).
        Built once and reused while the same arrays come back, as in a loop that passes one state list
        to every bl_set_states / bl_get_states; the library reads and writes them through the pointers."""
        key = [tuple(id(x) for x in a) for a in arrays]
        c = self._states_c
        if c is not None and c[0] == key:
            return c[1]
        arr = (bl_state * len(arrays))(*[bl_state(*[_p(x) for x in a], 0.0, 0.0, 0) for a in arrays])
        self._states_c = (key, arr, arrays)   # the arrays stay referenced while the pointers are kept
        return arr

    def get_states(self, out=None) -> list:
        """bl_get_states: every instance's state in one transfer; fills and returns `out` (a list of state
        dicts as get_state returns, e.g. from an earlier call) or new arrays."""
        out = out if out is not None else self._state_arrays()
        arr = self._states_struct([(*o["xold"], *o["xbest"]) for o in out])
        _check(load().bl_get_states(self.h, C.cast(arr, C.c_void_p)), self.h)
        for o, s in zip(out, arr):
            o.update(cstar=s.cstar, tmaxstar=s.tmaxstar, iter=s.iter)
        return out

    def set_states(self, states: list):
        """bl_set_states: every instance's state in one transfer."""
        def i16(x):
            ok = isinstance(x, np.ndarray) and x.dtype == np.int16 and x.flags.c_contiguous
            return x if ok else np.ascontiguousarray(x, dtype=np.int16)

        arr = self._states_struct([tuple(i16(x) for x in (*st["xold"], *st["xbest"])) for st in states])
        for s, st in zip(arr, states):
            s.cstar, s.tmaxstar, s.iter = float(st["cstar"]), float(st["tmaxstar"]), int(st["iter"])
        _check(load().bl_set_states(self.h, C.cast(arr, C.c_void_p)), self.h)

    def get_log(self, first: int, n: int, inst: int = 0) -> dict:
        o = dict(istar=np.zeros(n, np.int32), c_istar=np.zeros(n, np.float32), use_best=np.zeros(n, np.int8),
                 cstar=np.zeros(n, np.float32), indicator=np.zeros(n, np.int8))
        _check(load().bl_get_log(self.h, int(inst), int(first), int(n), _p(o["istar"]), _p(o["c_istar"]),
                                 _p(o["use_best"]), _p(o["cstar"]), _p(o["indicator"])), self.h)
        return o

    # --- inspection (parity tests)
    def score_candidates(self, use_best: int, iter_: int, tmax_star: float, i0: int, n: int, inst: int = 0,
                         units: bool = False) -> dict:
        I = self.instances[inst]
        T = I.n_tours
        km = max(1, int(self.params.k_moves))
        o = dict(cost=np.zeros(n, np.float32), tmax=np.zeros(n, np.float32), moves=np.zeros((n, 4 * km), np.int16),
                 n_hu=np.zeros((n, T), np.int16), n_su=np.zeros((n, T), np.int16))
        if units:
            o.update(hu_tour=np.zeros((n, I.n_hu), np.int16), su_tour=np.zeros((n, I.n_su), np.int16))
        _check(load().bl_score_candidates(self.h, int(inst), int(use_best), int(iter_), float(tmax_star), int(i0),
                                          int(n), _p(o["cost"]), _p(o["tmax"]), _p(o["moves"]), _p(o["n_hu"]),
                                          _p(o["n_su"]), _p(o.get("hu_tour")), _p(o.get("su_tour"))), self.h)
        return o

    def decode_candidates(self, use_best: int, iter_: int, idx, inst: int = 0) -> np.ndarray:
        I = self.instances[inst]
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        row = 2 * I.n_bps + I.n_tours + I.n_fields
        out = np.zeros((len(idx), row), np.int16)
        _check(load().bl_decode_candidates(self.h, int(inst), int(use_best), int(iter_), _p(idx), len(idx), _p(out)),
               self.h)
        return out

    def argmin_noalloc(self, use_best: int, iter_: int, tmax_star: float, i0: int, n: int, key_ptr: int,
                       tmax_ptr: int, inst: int = 0):
        """bl_argmin_noalloc: argmin of candidates i0..i0+n-1 into caller-owned device memory
        (key_ptr: 8 bytes, tmax_ptr: 4 bytes); the library allocates nothing for it."""
        _check(load().bl_argmin_noalloc(self.h, int(inst), int(use_best), int(iter_), float(tmax_star), int(i0),
                                        int(n), C.c_void_p(key_ptr), C.c_void_p(tmax_ptr)), self.h)

    def features(self, use_best: int, iter_: int, i0: int, n: int, feat, base_cost=None, inst: int = 0):
        """bl_features into a caller-owned torch bf16 tensor feat [>= n x 64] (and base_cost [1] float32)."""
        _check(load().bl_features(self.h, int(inst), int(use_best), int(iter_), int(i0), int(n),
                                  C.c_void_p(feat.data_ptr()),
                                  None if base_cost is None else C.c_void_p(base_cost.data_ptr())), self.h)

    def search_step_learned(self, mlp, n_iters: int, pool: int, n_keep: int, rand_frac: float = 0.1):
        """bl_search_step_learned with a paper_1909_10286_gb300.mlp.MLP created on this handle's stream."""
        _check(load().bl_search_step_learned(self.h, mlp.h, int(n_iters), int(pool), int(n_keep), float(rand_frac)),
               self.h)

    @property
    def stream(self):
        return self._stream

    def config(self) -> dict:
        v = [C.c_int32() for _ in range(5)]
        _check(load().bl_get_config(self.h, *[C.byref(x) for x in v]), self.h)
        return dict(block_threads=v[0].value, grid_blocks=v[1].value, tile=v[2].value, launches_per_iter=v[3].value,
                    lanes_per_cand=v[4].value)

    def close(self):
        if getattr(self, "h", None):
            load().bl_plan_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# C-ABI names as plain functions
def plan_init(instance, params: bl_params, stream=None) -> Search:
    return Search([instance], params, stream)


def plan_init_batch(instances, params: bl_params, stream=None) -> Search:
    return Search(instances, params, stream)


def search_step(h: Search, n_iters: int):
    h.search_step(n_iters)


def wait_selftest(limit_ns: int, stream=None) -> tuple[int, int]:
    """bl_wait_selftest: (return code, nanoseconds waited); BL_ETIMEOUT is the expected code."""
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    el = C.c_uint64(0)
    rc = load().bl_wait_selftest(C.c_void_p(s.cuda_stream), int(limit_ns), C.byref(el))
    return int(rc), int(el.value)


def best_plan(h: Search, inst: int = 0) -> dict:
    return h.best_plan(inst)


def plan_free(h: Search):
    h.close()
