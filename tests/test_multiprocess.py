"""The N > 1 path of bench.py on the CPU with gloo (world size 2): replicas,
one instance (or batch) per rank, no data exchange, a barrier and the maximum
of the ranks' times, and only rank 0 printing."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    ws, r, local = bench._dist()
    bench._barrier(ws)
    t = bench._max_over_ranks(10.0 * (r + 1), ws)
    seeds = [i.seed for i in bench.rank_instances("paper", 3, r, 4)]
    bseeds = [i.seed for i in bench.rank_instances("batched", 0, r, 4)]
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump(dict(ws=ws, rank=r, local=local, tmax=t, seeds=seeds, bseeds=bseeds), f)
    import torch.distributed as dist
    dist.destroy_process_group()


def test_gloo_ranks_share_the_max_time_and_search_their_own_instances(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert (r0["ws"], r0["rank"], r1["rank"]) == (2, 0, 1)
    assert r0["tmax"] == r1["tmax"] == 20.0            # the max over ranks, on every rank
    assert r0["seeds"] == [3] and r1["seeds"] == [4]    # seed + rank: replicas of different instances
    assert set(r0["bseeds"]).isdisjoint(r1["bseeds"]) and len(r0["bseeds"]) == len(r1["bseeds"]) == 4


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "3", "--workload", "tiny", "--ref-budget", "2"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
