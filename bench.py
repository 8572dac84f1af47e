"""Benchmark of the candidate search: candidates scored per second.

One step = one iteration of Algorithm 1 (Steps 6-16) on the paper-scale plain
workload: 40 fields, 5 BPs, 3 tours, 10 HUs, 20 SUs in a 50 x 50 km square,
2^20 candidates per iteration, every candidate scored exactly (demand check,
Fig. 1 costs, HU/SU local minimisation, gate), then argmin and update.

Timing: W untimed warm-up iterations, then K iterations each bracketed by CUDA
events on the search stream; the L2 is flushed (a 256 MiB device write)
before every timed iteration, outside the events. Under torchrun every rank
searches its own instance (seed + rank): replicas, weak scaling, no
collective in the data path; the time is the max over ranks.

Extra keys: e2e (the same metric through the C ABI with the state copied
from and to pinned host buffers every iteration), roofline (the scoring
kernel against the issue rate of the SMs, with the work per candidate counted
by the instrumented CPU oracle on a sample of the same iteration), clocks,
gpu_launches and cpu_baseline (the oracle on the host cores).

--impl reference times the CPU oracle alone on this workload (a bounded
sample of candidates per iteration, all host cores).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidates scored/s; time to reach within 1% of best cost (learned+batched vs plain)"
UNIT = "candidates/s"
WORKLOAD = "paper-scale plain search: 40 fields, 5 BPs, 3 tours, 10 HUs, 20 SUs, 50x50 km, 2^20 candidates/iter"
WORKLOAD_BATCHED = ("batched uneven instances: 256 instances (fields U{10..120}, BPs U{2..10}, tours U{1..6}, "
                    "HUs U{2..20}, SUs U{4..40}), 2^16 candidates/instance/iter, one launch per iteration")
WORKLOAD_LARGE = ("large plain search: 300 fields, 20 BPs, 10 tours, 60 HUs, 120 SUs, 150x150 km, "
                  "2^24 candidates/iter")
L2_FLUSH_BYTES = 256 << 20


def workload_text(workload: str, n_inst: int, n_per_inst: int, n_groups: int = 1) -> str:
    """The workload description with the instance count, candidates per iteration and launches actually run."""
    k = n_per_inst.bit_length() - 1
    n = f"2^{k}" if n_per_inst == 1 << k else str(n_per_inst)
    base = {"paper": WORKLOAD, "batched": WORKLOAD_BATCHED, "large": WORKLOAD_LARGE}.get(workload)
    if base is None:
        return workload
    if workload == "batched":
        base = base.replace("256 instances", f"{n_inst} instances").replace("2^16 candidates", f"{n} candidates")
        if n_groups > 1:
            base = base.replace("one launch per iteration",
                                f"one launch per iteration for each of {n_groups} launch-shape groups")
        return base
    return base.replace("2^20 candidates", f"{n} candidates").replace("2^24 candidates", f"{n} candidates")
# time-to-1% study settings per workload (paper: seeds 0-9, the paper's 10 experiments)
STUDY = {
    "paper": dict(workload="paper", seeds=range(10), n=1 << 20, iters=300, budget=1000, n_batched=1 << 16,
                  pool=1 << 16, keep=7373, rand_frac=0.014, train_seeds=range(100, 110)),
    "large": dict(workload="large", seeds=range(5), n=1 << 20, iters=400, budget=400, n_batched=1 << 16,
                  pool=1 << 18, keep=2359, rand_frac=0.001, train_seeds=range(100, 104), train_iters=30,
                  ref_n=1 << 16),
}


# the wall-clock time-to-1% study on the large workload (the default line's time_to_1pct key): plain and
# batched search with one and two chained moves per candidate, and learned + batched
STUDY_WALL = dict(workload="large", seeds=range(5), n=1 << 20, n_batched=1 << 16, max_iters=400, ref_iters=4000,
                  ref_n=1 << 16, pool=1 << 14, keep=1024, rand_frac=0.06, train_seeds=range(100, 104),
                  train_iters=30, k_values=(1, 2))
# The learned form's pool, keep and random fraction were picked by a sweep on instances 0-4; the same
# comparison on instances 5-9, which the sweep did not see, is reported beside it.
HELD_OUT = dict(seeds=range(5, 10), forms=("batched", "plain_k2", "learned_batched"))


def _dist():
    import torch.distributed as dist

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1 and not dist.is_initialized():
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class NvmlSampler:
    """SM clock, power and clock-event reasons read through NVML (libnvidia-ml)
    every ~2 ms in a thread, so that a timed region of a few milliseconds gets
    samples inside it. Read-only: nothing on the GPU is changed."""

    BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}

    def __init__(self, device_index: int):
        import ctypes as C
        import threading

        self.C, self.lib, self.h = C, None, None
        self.samples = []
        self.stop_evt = threading.Event()
        self.thread = None
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                self.lib = C.CDLL(name)
                break
            except OSError:
                continue
        if self.lib is None or self.lib.nvmlInit_v2() != 0:
            self.lib = None
            return
        h = C.c_void_p()
        try:
            import torch
            p = torch.cuda.get_device_properties(device_index)
            bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
            ok = self.lib.nvmlDeviceGetHandleByPciBusId_v2(C.c_char_p(bus), C.byref(h)) == 0
        except Exception:
            ok = False
        if not ok and self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(device_index), C.byref(h)) != 0:
            self.lib = None
            return
        self.h = h
        self.reasons_fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def ok(self) -> bool:
        return self.lib is not None

    def _run(self):
        C = self.C
        mhz, mw, rs = C.c_uint(), C.c_uint(), C.c_ulonglong()
        while not self.stop_evt.is_set():
            if (self.lib.nvmlDeviceGetClockInfo(self.h, 1, C.byref(mhz)) == 0 and
                    self.reasons_fn(self.h, C.byref(rs)) == 0):
                self.lib.nvmlDeviceGetPowerUsage(self.h, C.byref(mw))
                self.samples.append((mhz.value, mw.value / 1000.0, rs.value))
            self.stop_evt.wait(0.002)

    def start(self):
        import threading

        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def stop(self) -> dict:
        self.stop_evt.set()
        self.thread.join(timeout=5)
        mx = self.C.c_uint()
        self.lib.nvmlDeviceGetMaxClockInfo(self.h, 1, self.C.byref(mx))
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": mx.value or None, "reasons": ["no samples"], "source": "nvml"}
        reasons = sorted({n for _, _, r in self.samples for n, b in self.BITS.items() if r & b})
        return {"sm_mhz": statistics.median(m for m, _, _ in self.samples), "sm_max_mhz": mx.value,
                "reasons": reasons, "samples": len(self.samples),
                "power_w_max": max(p for _, p, _ in self.samples), "source": "nvml, every ~2 ms"}


def clock_sampler(device_index: int):
    """NVML sampling where the library is present, else nvidia-smi."""
    s = NvmlSampler(device_index)
    return s if s.ok() else ClockSampler(device_index)


class ClockSampler:
    """nvidia-smi clock samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2])); power.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.remove(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")


def _traffic(line_name: str):
    """DRAM bytes per launch of a line's dominant kernel, from one ncu capture listed in
    profiles/dram_traffic.txt, or None if there is none or the kernel's source file has
    changed since (its SHA-256 is recorded beside the figure)."""
    import hashlib

    try:
        rows = [r.split() for r in open(TRAFFIC_FILE) if r.strip() and not r.startswith("#")]
    except OSError:
        return None
    for r in rows:
        if len(r) >= 4 and r[0] == line_name:
            src, want_sha, nbytes = r[1], r[2], r[3]
            try:
                sha = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
            except OSError:
                return None
            return int(nbytes) if sha == want_sha else None
    return None


def oracle_throughput(inst, params_kw, n_cand, budget_s, threads, max_iters=50, state=None):
    """The CPU oracle's Algorithm 1 on the host cores: iterations of m candidates
    (m <= n_cand, chosen so the run takes about budget_s). Returns (cand/s, m, iters, threads)."""
    from oracle import oracle as O

    o = O.Oracle(inst)
    op = O.make_params(**params_kw)
    st = state or o.start(op)
    probe = min(n_cand, 8192)
    t0 = time.perf_counter()
    o.search(op, st.copy(), 1, probe, threads=threads)
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    m = int(min(n_cand, max(1024, rate * budget_s / 3)))
    iters = int(max(1, min(max_iters, budget_s * rate / m)))
    t0 = time.perf_counter()
    o.search(op, st, iters, m, threads=threads)
    dt = time.perf_counter() - t0
    return m * iters / dt, m, iters, threads


WORKLOAD_LEARNED = ("learned proposals on the paper-scale instance: per iteration 2^20 Philox moves featurised and "
                    "ranked by the MLP 64-256-256-256-1 (BF16, tensor cores), the 0.9*2^18 best plus ~10% random "
                    "moves scored exactly")
WORKLOAD_SURROGATE = ("surrogate pre-filter on the large instance (300 fields, 20 BPs, 10 tours, 60 HUs, 120 SUs): "
                      "per iteration 2^24 Philox moves featurised and scored by the MLP 64-256-256-256-1 (BF16, "
                      "tensor cores), the best 1% scored exactly")
RANKED = {
    # config 4: ranked proposals on the paper-scale instance
    "learned": dict(text=WORKLOAD_LEARNED, inst="paper", pool=1 << 20, keep=int(0.9 * (1 << 18)),
                    rand=0.1 * (1 << 18), train_iters=12, train_steps=600, compare_iters=0),
    # config 5: the surrogate scores 2^24 candidates, the top 1 % are scored exactly; plain exact search
    # at equal wall time beside it
    "surrogate": dict(text=WORKLOAD_SURROGATE, inst="large", pool=1 << 24, keep=(1 << 24) // 100, rand=0.0,
                      train_iters=12, train_steps=1500, compare_iters=100),
}


def _equal_wall_time(inst, kw, net, pool, keep, rand_frac, iters):
    """C* after `iters` ranked iterations from the initial plan, and C* of plain exact searches (2^24 and
    2^20 candidates per iteration) from the same plan given the same device time."""
    import torch

    from paper_1909_10286_gb300 import biolog

    def timed(S, step, k):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(S.stream)
        step(k)
        b.record(S.stream)
        b.synchronize()
        return a.elapsed_time(b)

    S = biolog.Search([inst], biolog.make_params(n_cand=pool, **kw))
    netS = net.copy(stream=S.stream, max_batch=8192)
    wall = timed(S, lambda k: S.search_step_learned(netS, k, pool, keep, rand_frac), iters)
    out = {"device_ms": wall, "ranked": {"iters": iters, "cstar": S.get_state()["cstar"]}}
    netS.close()
    S.close()
    for n in (1 << 24, 1 << 20):
        # iterations in chunks until the device time reaches the ranked run's; C* after the same
        # number of iterations as the ranked run is kept too (quality per iteration)
        P = biolog.Search([inst], biolog.make_params(n_cand=n, **kw))
        ms, k, c_at = 0.0, 0, None
        while ms < wall:
            step = max(1, min(iters, int((wall - ms) / max(ms / k, 1e-3) / 2) if k else 2))
            if k < iters < k + step:
                step = iters - k
            ms += timed(P, P.search_step, step)
            k += step
            if k == iters:
                c_at = P.get_state()["cstar"]
        out[f"plain_2^{n.bit_length() - 1}"] = {"iters": k, "device_ms": ms, "cstar": P.get_state()["cstar"],
                                               f"cstar_after_{iters}_iters": c_at}
        P.close()
    return out


def run_learned(args, ws, rank, local):
    line = measure_learned(args, args.workload, ws, rank, local)
    if rank == 0:
        print(json.dumps(line), flush=True)


def measure_learned(args, workload, ws, rank, local):
    """Configs 4 and 5: ranked proposals. value = exactly scored candidates/s; the
    roofline is the fused MLP forward's (the dominant kernel), timed on its own
    with CUDA events on the same pool of features."""
    import numpy as np
    import torch

    from paper_1909_10286_gb300 import biolog, learned
    from paper_1909_10286_gb300 import instances as I

    spec = RANKED[workload]
    torch.cuda.set_device(local)
    pool, keep = spec["pool"], spec["keep"]
    rand_frac = spec["rand"] / (pool - keep)
    t0 = time.time()
    X, T = learned.collect(I.make_batch(spec["inst"], range(100 + 10 * rank, 104 + 10 * rank)),
                           iters=spec["train_iters"], sample=8192)
    net0, losses = learned.train(X, T, hidden=256, steps=spec["train_steps"], batch=4096, lr=1e-3, max_batch=8192)
    t_train = time.time() - t0
    inst = I.make_instance(spec["inst"], args.seed + rank)
    kw = dict(eps=0.5, seed=1000 + args.seed + rank, gate=1)
    S = biolog.Search([inst], biolog.make_params(n_cand=pool, **kw))
    # the fused forward takes any number of rows; max_batch only sizes the training buffers
    net = net0.copy(stream=S.stream, max_batch=8192)
    stream = S.stream
    S.search_step_learned(net, args.warmup, pool, keep, rand_frac)
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = clock_sampler(local)
    clocks.start()
    _barrier(ws)
    torch.cuda.synchronize()
    for a, b in evs:
        with torch.cuda.stream(stream):
            flush.zero_()
        a.record(stream)
        S.search_step_learned(net, 1, pool, keep, rand_frac)
        b.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    clk = clocks.stop()
    t_ms = _max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), ws)
    ms_step = t_ms / args.steps
    # exactly scored candidates per iteration: the kept list (its length is data dependent)
    feat = torch.empty((pool, 64), dtype=torch.bfloat16, device="cuda")
    S.features(-1, 0xFFFFFFFF, 0, pool, feat)
    y = torch.empty(pool, dtype=torch.float32, device="cuda")
    with torch.cuda.stream(stream):
        net.forward(feat, y)
    torch.cuda.synchronize()
    yv = y.cpu().numpy()
    sample = np.sort(yv[(np.arange(4096) * pool) // 4096])
    th = sample[min(4095, keep * 4096 // pool)]
    n_exact = int((yv <= th).sum()) + int(round(rand_frac * int((yv > th).sum())))
    del yv
    value = n_exact * args.steps * ws / (t_ms / 1e3)
    # the fused MLP forward alone, on the same features, timed with CUDA events on its stream
    fe = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a, b in fe:
        with torch.cuda.stream(stream):
            flush.zero_()
        a.record(stream)
        net.forward(feat, y)
        b.record(stream)
    torch.cuda.synchronize()
    ms_mlp = statistics.median(a.elapsed_time(b) for a, b in fe)
    del feat, y
    flop = 2.0 * (64 * 256 + 2 * 256 * 256 + 256) * pool
    peaks = _peaks()
    peak = float(peaks.get("bf16_tflops", 1900.0))
    achieved = flop / (ms_mlp / 1e3) / 1e12
    hbm_bytes = pool * (64 * 2 + 4)
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32 scorer, bf16 ranker", "data": "synthetic",
            "config": {"workload": spec["text"], "instance_seed": args.seed, "pool": pool, "keep": keep,
                       "rand_frac": rand_frac, "exact_per_iter": n_exact,
                       "l2": "flushed before every timed step (256 MiB device write)",
                       "ranker_training": {"tuples": int(X.shape[0]), "steps": spec["train_steps"],
                                           "s": round(t_train, 1)},
                       "kernel": S.config(), "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "proposals_per_s": pool * args.steps * ws / (t_ms / 1e3),
            "gpu_launches": args.steps * 5, "clocks": clk,
            "e2e": {"value": None, "note": "the end-to-end number is on the default paper line"},
            "roofline": {"bound": "tensor", "kernel": "fused_mlp_forward_kernel", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": _traffic(workload),
                         "ms_per_launch": ms_mlp,
                         "flop_per_launch": flop,
                         "peak_basis": "bf16_tflops (burst) of MEASURED_PEAKS.json; kernel timed alone",
                         # the same launch against HBM: the features are materialised, so it reads them once
                         # (BF16, 64 per row) and writes one FP32 prediction per row
                         "hbm": {"achieved": hbm_bytes / (ms_mlp / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                                 "frac": hbm_bytes / (ms_mlp / 1e3) / 1e9 / hbm_peak, "bytes_per_launch": hbm_bytes,
                                 "peak_basis": "hbm_gbs of MEASURED_PEAKS.json"}}}
    net.close()
    S.close()
    if spec["compare_iters"] and rank == 0:
        line["equal_wall_time"] = _equal_wall_time(inst, kw, net0, pool, keep, rand_frac, spec["compare_iters"])
    net0.close()
    return line


def rank_instances(workload: str, seed: int, rank: int, n_inst: int):
    """The instances one rank searches: replicas, each rank its own (no data exchange)."""
    from paper_1909_10286_gb300 import instances as I

    if workload == "batched":
        return I.make_batch("batched", range(seed * 1000 + rank * n_inst, seed * 1000 + (rank + 1) * n_inst))
    return [I.make_instance(workload, seed + rank)]


def run_reference(args, ws, rank):
    if rank != 0:
        return
    from paper_1909_10286_gb300 import instances as I
    from oracle import oracle as O

    inst = I.make_instance(args.workload, args.seed)
    n = args.n_cand or I.SEARCH[args.workload][0]
    threads = os.cpu_count() or 1
    kw = dict(eps=0.5, seed=1000 + args.seed, gate=1)
    o = O.Oracle(inst)
    op = O.make_params(**kw)
    st = o.start(op)
    # sample size: the whole run (warm-up + steps) within about --ref-budget seconds
    probe = min(n, 8192)
    t0 = time.perf_counter()
    o.search(op, st.copy(), 1, probe, threads=threads)
    rate = probe / max(time.perf_counter() - t0, 1e-6)
    m = int(min(n, max(1024, rate * args.ref_budget / max(1, args.steps + args.warmup))))
    o.search(op, st, args.warmup, m, threads=threads)
    t0 = time.perf_counter()
    o.search(op, st, args.steps, m, threads=threads)
    dt = time.perf_counter() - t0
    value = m * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "instance_seed": args.seed, "n_cand_per_iter": n},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{m} of the {n} candidates per iteration, {args.steps} timed iterations"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--n-cand", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--n-inst", type=int, default=256, help="instances of the batched workload")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-shape-split", action="store_true",
                    help="batched: one handle for the whole batch instead of one per launch shape")
    ap.add_argument("--no-time-to-target", action="store_true",
                    help="skip the time-to-1%% study (paper workload, rank 0, one GPU)")
    ap.add_argument("--no-extra-lines", action="store_true",
                    help="skip the batched and large lines that the default (paper) line carries")
    ap.add_argument("--study", action="store_true", help="print only the time-to-1%% study for --workload")
    ap.add_argument("--ref-budget", type=float, default=120.0, help="seconds of oracle work in --impl reference")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload in RANKED:
        run_learned(args, ws, rank, local)
        return
    if args.study:
        import torch

        from paper_1909_10286_gb300 import time_to_target

        torch.cuda.set_device(local)
        print(json.dumps(dict(study="time to within 1% of the best cost",
                              **time_to_target.study(**STUDY[args.workload]))), flush=True)
        return

    import torch

    torch.cuda.set_device(local)
    line = measure_plain(args, args.workload, ws, rank, local, args.cpu_budget)
    if rank == 0:
        if ws == 1 and args.workload == "paper" and not args.no_extra_lines:
            # the other single-GPU workloads, each with its own roofline, e2e and CPU baseline
            for wl in ("batched", "large"):
                sub = measure_plain(args, wl, ws, rank, local, args.cpu_budget / 2)
                line[wl] = {k: sub[k] for k in ("value", "unit", "ms_per_step", "config", "gpu_launches", "clocks",
                                                "e2e", "roofline", "cpu_baseline") if k in sub}
            # the batched workload also as one persistent launch for the whole batch (one handle), beside
            # the default of one launch per launch-shape group
            one = measure_plain(argparse.Namespace(**{**vars(args), "no_shape_split": True, "no_cpu_baseline": True}),
                                "batched", ws, rank, local, 0.0)
            line["batched"]["one_launch"] = {k: one[k] for k in ("value", "ms_per_step", "config", "gpu_launches",
                                                                 "e2e", "roofline") if k in one}
            # ranked proposals on the paper-scale instance (the MLP's tensor-core roofline)
            sub = measure_learned(args, "learned", ws, rank, local)
            line["learned"] = {k: sub[k] for k in ("value", "unit", "ms_per_step", "config", "proposals_per_s",
                                                   "gpu_launches", "clocks", "roofline") if k in sub}
        if ws == 1 and args.workload == "paper" and not args.no_time_to_target:
            from paper_1909_10286_gb300 import time_to_target

            r = time_to_target.study_wall(**STUDY_WALL)
            line["time_to_1pct"] = {
                "unit": "ms", "higher_is_better": False,
                "workload": "large instances (300 fields, 20 BPs, 10 tours, 60 HUs, 120 SUs, 150x150 km); "
                            "candidates per iteration of each form in `forms`", "tol": r["tol"],
                "instances": r["seeds"], "timing": r["timing"],
                "c_ref": f"best C* of a plain batched run of {r['c_ref_run']['iters']} iterations of "
                         f"{r['c_ref_run']['n_cand']} candidates per instance",
                "median_ms": {k: f["median_ms"] for k, f in r["forms"].items()},
                "all_instances_ms": {k: f["all_instances_ms"] for k, f in r["forms"].items()},
                "reached": {k: f["reached"] for k, f in r["forms"].items()},
                "iters_to_target": {k: f["iters"] for k, f in r["forms"].items()},
                "setup_s": {k: f["setup_s"] for k, f in r["forms"].items()},
                "forms": {k: {q: v for q, v in f.items() if q in ("n_cand", "k_moves", "pool", "keep", "rand_frac")}
                          for k, f in r["forms"].items()},
                "ranker_training": {k: r["forms"]["learned_batched"][k]
                                    for k in ("train_tuples", "train_s", "train_loss_first_last")}}
            h = time_to_target.study_wall(**{**STUDY_WALL, **HELD_OUT})
            line["time_to_1pct"]["held_out"] = {
                "instances": h["seeds"],
                "note": "the learned form's settings were picked on instances 0-4; these were not seen by that sweep",
                "median_ms": {k: f["median_ms"] for k, f in h["forms"].items()},
                "all_instances_ms": {k: f["all_instances_ms"] for k, f in h["forms"].items()},
                "reached": {k: f["reached"] for k, f in h["forms"].items()},
                "iters_to_target": {k: f["iters"] for k, f in h["forms"].items()}}
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_plain(args, workload, ws, rank, local, cpu_budget):
    """One plain-search line: device-timed throughput, e2e through the C ABI, and on rank 0 the
    roofline and the CPU baseline."""
    import numpy as np
    import torch

    from paper_1909_10286_gb300 import biolog
    from paper_1909_10286_gb300 import instances as I

    n = (args.n_cand if workload == args.workload else 0) or I.SEARCH[workload][0]
    kw = dict(eps=0.5, seed=1000 + args.seed + rank, gate=1)
    stream = torch.cuda.Stream()
    tuned = None
    insts = rank_instances(workload, args.seed, rank, args.n_inst)
    tuned_all = []

    def params_of(group):
        if workload != "batched" or args.no_autotune:
            return biolog.make_params(n_cand=n, **kw)
        from paper_1909_10286_gb300 import autotune
        t = autotune.tune(group, n, base_params=kw)
        tuned_all.append(t)
        return biolog.make_params(n_cand=n, blocks_per_sm=t["blocks_per_sm"], tile=t["tile"],
                                  lanes_per_cand=t.get("lanes_per_cand", 1), **kw)

    inst = insts[0]
    n_total = n * len(insts)
    if workload == "batched" and not args.no_shape_split:
        # one handle per launch shape (the instances that fit the four-tour shape, and the rest)
        from paper_1909_10286_gb300 import shaped
        S = shaped.ShapedBatch(insts, params_of, stream=stream)
    else:
        S = biolog.Search(insts, params_of(insts), stream=stream)
    tuned = (tuned_all[0] if len(tuned_all) == 1 else tuned_all) or None
    cfg = S.config()
    with torch.cuda.stream(stream):
        S.search_step(args.warmup)
    torch.cuda.synchronize()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = clock_sampler(local)
    clocks.start()
    _barrier(ws)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for a, b in evs:
            flush.zero_()
            a.record(stream)
            S.search_step(1)
            b.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    clk = clocks.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in evs)
    t_ms = _max_over_ranks(t_ms, ws)
    value = n_total * args.steps * ws / (t_ms / 1e3)
    ms_step = t_ms / args.steps
    del flush

    # e2e through the C ABI: every instance's state in from host memory, one iteration, every state
    # out (bl_set_states / bl_get_states: one transfer each way through the library's pinned staging)
    hstate = S.get_states()
    bytes_state = sum(sum(a.nbytes for a in h["xold"] + h["xbest"]) + 12 for h in hstate)
    e2e_steps = max(1, min(args.e2e_steps, int(2000 / max(ms_step, 1e-3))))
    _barrier(ws)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        S.set_states(hstate)
        with torch.cuda.stream(stream):
            S.search_step(1)
        S.get_states(hstate)
    e2e_s = _max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": n_total * e2e_steps * ws / e2e_s, "unit": UNIT, "h2d_bytes_per_step": bytes_state,
           "d2h_bytes_per_step": bytes_state, "steps": e2e_steps,
           "api": "bl_set_states + bl_search_step(1) + bl_get_states (all instances, one transfer each way)"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_text(workload, len(insts), n_total // max(1, len(insts)),
                                                 len(cfg.get("groups", [cfg]))),
                       "instance_seed": args.seed, "n_instances": len(insts), "n_cand_per_iter": n_total,
                       "eps": 0.5, "gate": 1, "autotuned": tuned,
                       "l2": "flushed before every timed step (256 MiB device write)",
                       "kernel": cfg, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
            "gpu_launches": args.steps * cfg["launches_per_iter"], "clocks": clk, "e2e": e2e}

    if rank == 0:
        # roofline: oracle-counted model operations per candidate on a sample of this iteration
        from oracle import oracle as O

        o = O.Oracle(inst)
        op = O.make_params(**kw)
        cur = S.get_state()
        base = O.Plan(*(cur["xbest"] if o.eps_select(op, cur["iter"]) else cur["xold"]))
        tstar = o.score(O.Plan(*cur["xbest"]), op, gate=0)["tmax"]
        m = 1 << 14
        r = o.score_batch(op, cur["iter"], base, m, tmax_star=tstar, threads=os.cpu_count() or 1)
        w_per = r["ops"] / m
        peaks = _peaks()
        f_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        peak = sms * 4 * 32 * f_mhz * 1e6 / 1e12            # lane-ops/s: 4 schedulers x 32 lanes per SM
        achieved = w_per * n_total / (ms_step / 1e3) / 1e12
        line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tlane-op/s",
                            "frac": achieved / peak,
                            "traffic": _traffic("batched_one" if workload == "batched" and args.no_shape_split
                                                else workload), "ops_per_candidate": w_per,
                            "peak_basis": f"{sms} SMs x 4 schedulers x 32 lanes x {f_mhz:.0f} MHz (sm_max_mhz of "
                                          "MEASURED_PEAKS.json)"}
        if len(insts) > 1:
            line["roofline"]["ops_per_candidate_basis"] = "oracle count on instance 0 of the batch"
        if ws == 1 and not args.no_cpu_baseline:
            rate, m_s, iters, thr = oracle_throughput(inst, kw, n, cpu_budget, os.cpu_count() or 1)
            line["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": thr, "kind": "oracle",
                                    "sample": f"{iters} oracle iterations of {m_s} candidates (of {n}) from the "
                                              "initial plan" + (" of instance 0" if len(insts) > 1 else "")}
    S.close()
    return line


if __name__ == "__main__":
    main()
