"""One iteration's candidates split over several processes, one GPU each.

The candidates of an iteration are independent (Sec. 2.5): every process
holds the same instance and state, scores its own contiguous slice of the
candidate numbers, and the iteration's argmin is the minimum of the slices'
keys ((cost bits << 32) | i, ties to the lowest i as in the unsplit
iteration). One all-reduce-min of a single 64-bit integer per iteration is
the only exchange: each process then replays move i* on its own copy of the
base plan (Steps 13-16), so the states stay identical without sending plans.

This module sequences the calls only: the scoring and the update run in the
library's kernels (bl_search_score_slice, bl_search_apply), the reduction in
torch.distributed (NCCL between GPUs).
"""
from __future__ import annotations


def slice_of(n_cand: int, world: int, rank: int) -> tuple[int, int]:
    """(first candidate number, count) of `rank`'s slice: contiguous, sizes differing by at most one."""
    if not (0 <= rank < world) or n_cand < world:
        raise ValueError("need 0 <= rank < world <= n_cand")
    lo = (rank * n_cand) // world
    hi = ((rank + 1) * n_cand) // world
    return lo, hi - lo


class GpuSlice:
    """This process's slice of a split search: a library handle over candidates offset .. offset+count-1."""

    def __init__(self, inst, n_cand: int, world: int, rank: int, **params):
        import torch

        from . import biolog

        self.offset, self.count = slice_of(n_cand, world, rank)
        self.search = biolog.Search([inst], biolog.make_params(n_cand=self.count, cand_offset=self.offset, **params),
                                    stream=torch.cuda.current_stream())
        self.key = torch.zeros(1, dtype=torch.int64, device="cuda")

    def score_slice(self):
        self.search.score_slice(self.key.data_ptr())
        return self.key

    def apply(self, key):
        self.search.apply(key.data_ptr())

    def close(self):
        self.search.close()


class SplitSearch:
    """Drives split iterations over a process group: score this rank's slice, all-reduce-min the key,
    apply it. `scorer` provides score_slice() -> a one-element int64 tensor and apply(key)."""

    def __init__(self, scorer, group=None):
        self.scorer = scorer
        self.group = group

    def step(self, n_iters: int = 1):
        import torch.distributed as dist

        for _ in range(n_iters):
            key = self.scorer.score_slice()
            if dist.is_initialized() and dist.get_world_size(self.group) > 1:
                dist.all_reduce(key, op=dist.ReduceOp.MIN, group=self.group)
            self.scorer.apply(key)
