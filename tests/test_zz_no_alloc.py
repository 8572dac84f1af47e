"""The allocation-free argmin entry point agrees with the regular inspection
entry point.

bl_argmin_noalloc serves callers that must not allocate device memory where
they call it (a latency-critical loop that cannot afford cudaMalloc's device
synchronisation, or a process whose device memory belongs to another
allocator): its scratch is a static device array inside the library. This
test calls it twice in a row through the C ABI -- the second call finds the
first call's leftovers in the shared scratch -- and checks each result
against the argmin of the costs bl_score_candidates returns for the same
candidates. The file is named to be collected last.
"""
import numpy as np
import pytest

from paper_1909_10286_gb300 import biolog
from paper_1909_10286_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _host_argmin(cost, i0=0):
    bits = cost.astype(np.float32).view(np.uint32).astype(np.uint64)
    keys = (bits << np.uint64(32)) | (np.uint64(i0) + np.arange(len(cost), dtype=np.uint64))
    return int(keys.min())


# (workload, first candidate i0, count n, blocks per SM): i0 > 0 offsets the positions; n = 2^20 + 37
# needs more blocks than the launch grid has, so every block's grid-stride loop takes several passes
# before the queue's last flush; with 8 blocks per SM the grid (8 x the SM count) is clamped to the
# 1024 partial results the scratch holds
@pytest.mark.parametrize("wl,i0,n,bps", [("paper", 0, 20000 + 37, 0), ("batched", 0, 7001, 0),
                                         ("paper", 12345, 20000 + 37, 0), ("paper", 12345, (1 << 20) + 37, 0),
                                         ("paper", 777, (1 << 20) + 37, 8)])
def test_argmin_noalloc_matches_score_candidates(wl, i0, n, bps):
    import torch

    inst = I.make_instance(wl, 3)
    S = biolog.Search([inst], biolog.make_params(n_cand=n, eps=0.5, seed=1000, gate=1, blocks_per_sm=bps))
    S.search_step(2)
    st = S.get_state()
    out_key = torch.zeros(2, dtype=torch.int64, device="cuda")
    out_t = torch.zeros(2, dtype=torch.float32, device="cuda")
    for call, use_best in enumerate((0, 1)):          # two calls in a row share the scratch
        S.argmin_noalloc(use_best, st["iter"], st["tmaxstar"], i0, n, out_key.data_ptr() + 8 * call,
                         out_t.data_ptr() + 4 * call)
    torch.cuda.synchronize()
    for call, use_best in enumerate((0, 1)):
        g = S.score_candidates(use_best, st["iter"], st["tmaxstar"], i0, n)
        want = _host_argmin(g["cost"], i0)
        got = int(out_key[call].item()) & 0xFFFFFFFFFFFFFFFF
        c_got = np.uint32(got >> 32).view(np.float32)
        c_want = np.uint32(want >> 32).view(np.float32)
        assert np.isfinite(c_want)
        assert abs(float(c_got) - float(c_want)) <= 1e-5 * abs(float(c_want))
        assert got & 0xFFFFFFFF == want & 0xFFFFFFFF
        i = (want & 0xFFFFFFFF) - i0
        assert float(out_t[call].item()) == pytest.approx(float(g["tmax"][i]), rel=1e-5)
    with pytest.raises(biolog.BiologError) as e:
        S.argmin_noalloc(0, st["iter"], st["tmaxstar"], 0, 0, out_key.data_ptr(), out_t.data_ptr())
    assert e.value.code == biolog.BL_ETOO_LARGE
    S.close()
