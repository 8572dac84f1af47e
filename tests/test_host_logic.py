"""Host-side logic without a GPU: the shape groups of a batch (shaped.groups), the time-to-target
harness (time_to_target._wall_to_target) on a stand-in handle, and the bench's workload text."""
import pytest

from paper_1909_10286_gb300 import instances as I
from paper_1909_10286_gb300 import shaped
from paper_1909_10286_gb300 import time_to_target as TT


def test_shape_groups_partition_the_batch_by_the_four_tour_limits():
    insts = I.make_batch("batched", range(64))
    gs = shaped.groups(insts)
    assert sorted(i for g in gs for i in g) == list(range(64))
    assert len(gs) == 2
    for i in gs[0]:
        x = insts[i]
        assert x.n_tours <= 4 and x.n_hu <= 32 and x.n_su <= 32
    for i in gs[1]:
        x = insts[i]
        assert x.n_tours > 4 or x.n_hu > 32 or x.n_su > 32
    # order within a group follows the batch; a batch of one kind gives one group
    assert all(a < b for g in gs for a, b in zip(g, g[1:]))
    assert shaped.groups([insts[i] for i in gs[0]]) == [list(range(len(gs[0])))]
    assert shaped.groups(I.make_batch("large", range(3))) == [[0, 1, 2]]


class _FakeSearch:
    """C* per instance after each iteration from fixed traces; states as get_states returns them."""

    def __init__(self, traces):
        self.traces = traces
        self.it = 0

    def _fill(self, out):
        for k, tr in enumerate(self.traces):
            out[k]["cstar"] = tr[min(self.it, len(tr) - 1)]
        return out

    def get_states(self, out=None):
        return self._fill(out if out is not None else [dict() for _ in self.traces])

    def search_step(self, n):
        self.it += n


def test_wall_to_target_takes_the_first_iteration_at_or_below_each_target():
    traces = [[10.0, 9.0, 8.0, 8.0, 7.0, 7.0],     # reaches 8.0 after iteration 2
              [5.0, 5.0, 5.0, 4.5, 4.0, 4.0],      # reaches 4.0 after iteration 4
              [3.0, 3.0, 3.0, 3.0, 3.0, 3.0]]      # never reaches 1.0
    S = _FakeSearch(traces)
    ms, its, n, total = TT._wall_to_target(S, [8.0, 4.0, 1.0], 5, S.search_step)
    assert its == [2, 4, None] and n == 5
    assert ms[2] is None and 0.0 <= ms[0] <= ms[1] <= total
    # a target met by the initial plan counts at iteration 0; the loop stops once all are met
    S = _FakeSearch(traces[:2])
    ms, its, n, _ = TT._wall_to_target(S, [10.0, 4.5], 50, S.search_step)
    assert its == [0, 3] and n == 3 and ms[0] == 0.0


def test_bench_workload_text_names_the_sizes_run():
    import bench

    t = bench.workload_text("batched", 64, 1 << 15, 2)
    assert "64 instances" in t and "2^15 candidates" in t and "2 launch-shape groups" in t
    assert "2^20 candidates" in bench.workload_text("large", 1, 1 << 20)
    assert bench.workload_text("paper", 1, 1 << 20) == bench.WORKLOAD
    assert "3000 candidates" in bench.workload_text("paper", 1, 3000)
