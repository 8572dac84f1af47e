"""A batch of uneven instances split by launch shape: one library handle per group, all on one stream.

The library gives a handle one launch shape, the one its largest instance needs (tours, HUs, SUs,
distance table). In a batch of uneven instances the small ones then run on the large ones' shape:
on GB300, 128-thread blocks at 2 per SM (8 resident warps), where instances of at most 4 tours and
32 HUs and SUs fit the 256-thread shape with the distances in shared memory (16 resident warps).
ShapedBatch puts those instances in a handle of their own and the rest in another, on the same
stream, so one iteration is the groups' launches back to back. Host-side bookkeeping only: every
step runs in the library's kernels, each group's handle exactly as a Search of its own.

An instance's candidate stream depends on its index within its handle (the Philox counter carries
it), so a split batch draws other (equally valid) candidates than the same batch in one handle.
"""
from __future__ import annotations

from . import biolog

# limits of the four-tour shape (shape A) of the library's kernels
SMALL_TOURS, SMALL_UNITS = 4, 32


def small(inst) -> bool:
    """Whether an instance fits the four-tour shape by its tour and unit counts (the library still
    checks the distance table and the unit sums, and picks the next shape if they do not fit)."""
    return inst.n_tours <= SMALL_TOURS and inst.n_hu <= SMALL_UNITS and inst.n_su <= SMALL_UNITS


def groups(instances) -> list[list[int]]:
    """Instance indices of each group: those that fit the four-tour shape, then the others (empty
    groups left out)."""
    a = [i for i, x in enumerate(instances) if small(x)]
    b = [i for i, x in enumerate(instances) if not small(x)]
    return [g for g in (a, b) if g]


class ShapedBatch:
    """One biolog.Search per shape group on a shared stream, addressed by the batch's instance indices.

    `params_of(instances)` gives each group's bl_params (e.g. autotuned for that group)."""

    def __init__(self, instances, params_of, stream=None):
        import torch

        self.instances = list(instances)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        self.groups = groups(self.instances)
        self.handles = []
        try:
            for g in self.groups:
                sub = [self.instances[i] for i in g]
                self.handles.append(biolog.Search(sub, params_of(sub), stream=self._stream))
        except Exception:
            self.close()
            raise
        self._where = {}
        for h, g in enumerate(self.groups):
            for k, i in enumerate(g):
                self._where[i] = (h, k)

    @property
    def stream(self):
        return self._stream

    def search_step(self, n_iters: int):
        """n_iters iterations of every group (the groups' instances are independent, so running one
        group's iterations before the other's gives what interleaving them would)."""
        for S in self.handles:
            S.search_step(n_iters)

    def config(self) -> dict:
        cfgs = [S.config() for S in self.handles]
        return dict(groups=[dict(c, n_instances=len(g)) for c, g in zip(cfgs, self.groups)],
                    launches_per_iter=sum(c["launches_per_iter"] for c in cfgs))

    def _at(self, inst: int):
        h, k = self._where[inst]
        return self.handles[h], k

    def get_state(self, inst: int = 0) -> dict:
        S, k = self._at(inst)
        return S.get_state(inst=k)

    def set_state(self, state: dict, inst: int = 0):
        S, k = self._at(inst)
        S.set_state(state, inst=k)

    def best_plan(self, inst: int = 0) -> dict:
        S, k = self._at(inst)
        return S.best_plan(inst=k)

    def get_log(self, first: int, n: int, inst: int = 0) -> dict:
        S, k = self._at(inst)
        return S.get_log(first, n, inst=k)

    def get_states(self, out=None) -> list:
        """Every instance's state, one bl_get_states transfer per group, in the batch's order. With `out`
        (state dicts as get_state returns, e.g. from an earlier call) those dicts are filled and returned."""
        if out is None:
            parts = [S.get_states() for S in self.handles]
        else:
            parts = [S.get_states([out[i] for i in g]) for S, g in zip(self.handles, self.groups)]
        res = [None] * len(self.instances)
        for g, o in zip(self.groups, parts):
            for k, i in enumerate(g):
                res[i] = o[k]
        return res

    def set_states(self, states: list):
        """Every instance's state, in the batch's order; one bl_set_states transfer per group."""
        for S, g in zip(self.handles, self.groups):
            S.set_states([states[i] for i in g])

    def close(self):
        for S in getattr(self, "handles", []):
            S.close()
        self.handles = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
