"""Autotuner for the launch shape of the search kernel.

The free launch parameters are (a) how many lanes score one candidate: one
thread, or a group of 4 to 32 lanes holding one tour each (the cooperative
kernel; same results, other latency and occupancy); (b) how many blocks the
grid keeps resident per SM -- more blocks hide latency, fewer leave registers
and shared memory to each; and (c) how many candidates one work item holds,
which trades per-item staging cost against load balance across uneven
instances.

`tune()` times a few iterations for each pair on the actual instances and
returns the fastest; results are cached in a JSON file keyed by the GPU name
and a size bucket of the workload (instances, largest field count, largest
tour count, candidates per instance), so a repeated workload shape is tuned
once. Every timing runs the real search (iterations advance the state of a
throw-away handle), timed with CUDA events.
"""
from __future__ import annotations

import json
import os
import threading

from . import biolog

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "autotune.json")
_lock = threading.Lock()

LANES = (1, 4, 8, 16, 32)       # lane counts the library builds (each for some tour counts)
BLOCKS_PER_SM = (1, 2, 3, 4)
TILE_FACTORS = (1, 4, 16, 64)   # candidates per work item, in units of the block size (of groups, cooperative)
COOP_BLOCKS_PER_SM = (1, 2)
COOP_TILE_FACTORS = (1, 4, 16)


def _bucket(instances, n_cand: int) -> str:
    f = max(i.n_fields for i in instances)
    t = max(i.n_tours for i in instances)
    fb = 1 << max(0, (f - 1).bit_length())
    nb = 1 << max(0, (n_cand - 1).bit_length())
    return f"n_inst={len(instances)}|F<={fb}|T<={t}|n_cand<={nb}"


def _load() -> dict:
    try:
        return json.load(open(CACHE))
    except (OSError, ValueError):
        return {}


def _time(instances, params, iters: int) -> float:
    import torch

    S = biolog.Search(instances, params)
    S.search_step(2)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    S.search_step(iters)
    b.record()
    torch.cuda.synchronize()
    cfg = S.config()
    S.close()
    return a.elapsed_time(b) / iters, cfg


def tune(instances, n_cand: int, base_params: dict | None = None, iters: int = 8, use_cache: bool = True) -> dict:
    """Returns {"lanes_per_cand", "blocks_per_sm", "tile", "ms_per_iter", ...} for this workload."""
    import torch

    gpu = torch.cuda.get_device_name()
    key = f"v4|{gpu}|{_bucket(instances, n_cand)}"   # v4: six- and ten-tour shapes, two blocks per SM
    with _lock:
        cache = _load() if use_cache else {}
        if key in cache:
            return cache[key]
    base_params = dict(base_params or {})
    results = []
    for lanes in LANES:
        try:   # lane counts that are not built for these tour counts are refused
            S = biolog.Search(instances, biolog.make_params(n_cand=n_cand, lanes_per_cand=lanes, **base_params))
        except biolog.BiologError:
            continue
        unit = S.config()["block_threads"] // max(1, lanes)   # threads, or lane groups, per block
        S.close()
        for bps in (BLOCKS_PER_SM if lanes == 1 else COOP_BLOCKS_PER_SM):
            for tf in (TILE_FACTORS if lanes == 1 else COOP_TILE_FACTORS):
                p = biolog.make_params(n_cand=n_cand, blocks_per_sm=bps, tile=tf * unit, lanes_per_cand=lanes,
                                       **base_params)
                try:
                    ms, cfg = _time(instances, p, iters)
                except biolog.BiologError:
                    continue
                results.append({"lanes_per_cand": lanes, "blocks_per_sm": bps, "tile": tf * unit, "ms_per_iter": ms,
                                "grid_blocks": cfg["grid_blocks"]})
    best = min(results, key=lambda r: r["ms_per_iter"])
    best = dict(best, tried=len(results), bucket=key)
    with _lock:
        cache = _load()
        cache[key] = best
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        tmp = CACHE + f".{os.getpid()}.tmp"
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, CACHE)
    return best


def tuned_params(instances, n_cand: int, **kw) -> "biolog.bl_params":
    """bl_params with the tuned launch shape for these instances."""
    best = tune(instances, n_cand, base_params=kw)
    return biolog.make_params(n_cand=n_cand, blocks_per_sm=best["blocks_per_sm"], tile=best["tile"],
                              lanes_per_cand=best.get("lanes_per_cand", 1), **kw)
