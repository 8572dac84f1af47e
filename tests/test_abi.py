"""The C-ABI library builds, loads and exports every entry point its header
declares, and its host-side validation answers without a GPU."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_1909_10286_gb300 import biolog, build
from paper_1909_10286_gb300 import instances as I


@pytest.fixture(scope="module")
def lib():
    build.build()
    return biolog.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "biolog.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bl_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    declared = _declared()
    assert len(declared) >= 14
    assert set(declared) == set(biolog.EXPORTS)
    for name in declared:
        assert hasattr(lib, name), name


def test_workspace_query_and_validation_without_gpu(lib):
    inst = I.make_instance("paper", 0)
    p = biolog.make_params(n_cand=1 << 20)
    assert biolog.workspace_bytes([inst], p) > 0
    bad = I.make_instance("paper", 0)
    bad.supply_t = bad.supply_t.copy(); bad.supply_t[3] = -1.0
    with pytest.raises(biolog.BiologError) as e:
        biolog.workspace_bytes([bad], p)
    assert e.value.code == biolog.BL_EINVAL
    infeas = I.make_instance("paper", 0)
    infeas.demand_t = (infeas.demand_t * 2).astype(np.float32)
    with pytest.raises(biolog.BiologError) as e:
        biolog.workspace_bytes([infeas], p)
    assert e.value.code == biolog.BL_EINFEASIBLE_INSTANCE
    # instances whose distance tables do not fit in shared memory next to the kernel's buffers: accepted
    for F, T in ((180, 5), (186, 8)):
        assert biolog.workspace_bytes([I.make_sized(F, 5, T, 10, 20, seed=F)], p) > 0
    big = I.make_instance("large", 0)
    big.n_tours = 17
    with pytest.raises(biolog.BiologError) as e:
        biolog.workspace_bytes([big], p)
    assert e.value.code == biolog.BL_ETOO_LARGE
    with pytest.raises(biolog.BiologError) as e:
        biolog.workspace_bytes([inst], biolog.make_params(n_cand=0))
    assert e.value.code == biolog.BL_EINVAL


def test_no_cpu_fallback():
    """Without a CUDA device the search refuses to run instead of falling back."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(biolog.BiologError):
        biolog.plan_init(I.make_instance("tiny", 0), biolog.make_params(n_cand=64))


def test_argmin_noalloc_size_checks_without_gpu(lib):
    """bl_argmin_noalloc checks n and i0 + n before it looks at the handle, so the
    limits are testable with a NULL handle and no GPU: positions up to INT32_MAX
    are legal, one past it is not."""
    import ctypes as C

    def call(i0, n):
        return lib.bl_argmin_noalloc(None, 0, 0, 0, C.c_float(0.0), int(i0), int(n), C.c_void_p(8), C.c_void_p(8))

    int32_max = 2**31 - 1
    max_cand = 1 << 28
    for i0, n in ((0, 0), (0, -1), (0, max_cand + 1), (-1, 10), (int32_max - 9, 11), (int32_max, 1),
                  (int32_max - max_cand + 1, max_cand)):
        assert call(i0, n) == biolog.BL_ETOO_LARGE, (i0, n)
        assert b"INT32_MAX" in lib.bl_global_error()
    # legal sizes reach the handle check (NULL handle -> BL_EINVAL), the last ones end at INT32_MAX
    for i0, n in ((0, 1), (0, max_cand), (int32_max - 10, 10), (int32_max - 1, 1), (int32_max - max_cand, max_cand)):
        assert call(i0, n) == biolog.BL_EINVAL, (i0, n)


def test_chained_move_parameters_without_gpu(lib):
    """k_moves: 1 to 3 chained moves are accepted; more, or chained moves with lane groups, are not."""
    inst = I.make_instance("paper", 0)
    for k in (0, 1, 2, 3):
        assert biolog.workspace_bytes([inst], biolog.make_params(n_cand=4096, k_moves=k)) > 0
    for p in (biolog.make_params(n_cand=4096, k_moves=4), biolog.make_params(n_cand=4096, k_moves=-1),
              biolog.make_params(n_cand=4096, k_moves=2, lanes_per_cand=8)):
        with pytest.raises(biolog.BiologError) as e:
            biolog.workspace_bytes([inst], p)
        assert e.value.code == biolog.BL_EINVAL


def test_candidate_offset_parameter_without_gpu(lib):
    """cand_offset + n_cand must stay within the 31-bit candidate numbers."""
    inst = I.make_instance("paper", 0)
    assert biolog.workspace_bytes([inst], biolog.make_params(n_cand=4096, cand_offset=(1 << 31) - 1 - 4096)) > 0
    with pytest.raises(biolog.BiologError) as e:
        biolog.workspace_bytes([inst], biolog.make_params(n_cand=4096, cand_offset=(1 << 31) - 4096))
    assert e.value.code == biolog.BL_EINVAL
