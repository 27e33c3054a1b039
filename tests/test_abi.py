"""C-ABI checks that need no GPU: the library loads, exports every function
include/dkm.h declares, validates arguments on the host, and the grid
planner honours the memory budget (the memory-tunable index of Section V-A)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dkm.h")


@pytest.fixture(scope="module")
def dkm():
    from paper_2412_02244_gb300 import build
    build.build()
    from paper_2412_02244_gb300 import dkm as m
    m.lib()
    return m


def declared_functions():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"DKM_API\s+[\w\s\*]+?\b(dkm_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for want in ("dkm_create", "dkm_assign", "dkm_update", "dkm_fit", "dkm_run", "dkm_destroy"):
        assert want in names


def test_every_declared_symbol_is_exported(dkm):
    lib = dkm.lib()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header(dkm):
    for n in declared_functions():
        assert hasattr(dkm, n), f"binding lacks {n}"


def test_default_options(dkm):
    o = dkm.dkm_default_options()
    assert o.mem_budget_bytes == 64 << 20
    assert o.cells_per_centroid == pytest.approx(1.0)
    assert o.algo == dkm.DKM_ALGO_INDEXED and o.early_stop == 1 and o.profile == 0
    assert dkm.dkm_status_string(1) == "DKM_EINVAL"


@pytest.mark.parametrize("n,d,k", [(0, 2, 1), (10, 4, 2), (10, 1, 2), (10, 2, 0), (10, 3, 11)])
def test_plan_rejects_bad_sizes(dkm, n, d, k):
    with pytest.raises(dkm.DkmError) as e:
        dkm.dkm_plan(n, d, k, [0] * d, [1] * d)
    assert e.value.status == dkm.DKM_EINVAL


def test_plan_rejects_bad_box(dkm):
    with pytest.raises(dkm.DkmError):
        dkm.dkm_plan(10, 2, 2, [1, 0], [0, 1])
    with pytest.raises(dkm.DkmError):
        dkm.dkm_plan(10, 2, 2, [float("nan"), 0], [1, 1])


@pytest.mark.parametrize("budget_mb", [0.5, 1, 4, 64, 1024])
def test_plan_respects_budget(dkm, budget_mb):
    k = 10_000
    o = dkm.dkm_default_options(mem_budget_bytes=int(budget_mb * (1 << 20)))
    p = dkm.dkm_plan(10_000_000, 3, k, [-100, -100, 0], [100, 100, 10], o)
    assert p.index_bytes <= o.mem_budget_bytes
    assert p.cells == p.dims[0] * p.dims[1] * p.dims[2]
    assert p.cells <= math.ceil(o.cells_per_centroid * k)
    # the grid covers the box: dims * cell >= extent on every axis
    for a, ext in enumerate([200, 200, 10]):
        assert p.dims[a] * p.cell >= ext * (1 - 1e-6)


def test_smaller_budget_gives_coarser_grid(dkm):
    cells = []
    for mb in (0.5, 1, 4, 16):
        o = dkm.dkm_default_options(mem_budget_bytes=int(mb * (1 << 20)))
        cells.append(dkm.dkm_plan(10_000_000, 3, 10_000, [0, 0, 0], [1, 1, 1], o).cells)
    assert cells == sorted(cells) and cells[0] < cells[-1]


def test_plan_budget_too_small(dkm):
    o = dkm.dkm_default_options(mem_budget_bytes=1024)
    with pytest.raises(dkm.DkmError) as e:
        dkm.dkm_plan(1000, 2, 500, [0, 0], [1, 1], o)
    assert e.value.status == dkm.DKM_ENOMEM


def test_plan_degenerate_axes(dkm):
    p = dkm.dkm_plan(1000, 3, 100, [0, 0, 5], [10, 10, 5])     # flat in z
    assert p.dims[2] == 1 and p.cells <= 200
    p = dkm.dkm_plan(1000, 2, 100, [3, 3], [3, 3])             # a single point
    assert p.cells == 1


def test_binding_type_checks(dkm):
    with pytest.raises(TypeError):
        dkm.dkm_create(np.zeros(8, np.float64), 4, 2, 1)
    with pytest.raises(ValueError):
        dkm.dkm_create(np.zeros(6, np.float32), 4, 2, 1)


def test_noalloc_rejects_k_beyond_its_scratch(dkm):
    # size checks come before any GPU work, so this runs without a GPU
    status = dkm.lib().dkm_lloyd_step_noalloc(None, 10, 3, dkm.DKM_NOALLOC_MAX_K + 1, None, None,
                                              None, None, None)
    assert status == dkm.DKM_EINVAL
    assert "DKM_NOALLOC_MAX_K" in dkm.dkm_last_error()


def test_create_validates_before_touching_the_gpu(dkm):
    with pytest.raises(dkm.DkmError) as e:
        dkm.dkm_create(np.zeros(8, np.float32), 4, 2, 5)     # k > n
    assert e.value.status == dkm.DKM_EINVAL
    assert "must not exceed" in dkm.dkm_last_error()


@pytest.mark.parametrize("offsets,ks,d,msg", [
    ([0, 5, 5, 9], [1, 1, 1], 3, "empty"),          # a cloud with no points
    ([0, 4, 9], [5, 2], 3, "exceeds"),               # k_b > n_b
    ([0, 4, 9], [0, 2], 3, ">= 1"),                  # k_b < 1
    ([1, 4, 9], [1, 2], 3, "offsets[0]"),            # offsets do not start at 0
    ([0, 4, 9], [1, 2], 4, "d must be"),             # d not 2 / 3
])
def test_batched_create_validates_before_touching_the_gpu(dkm, offsets, ks, d, msg):
    n = offsets[-1]
    with pytest.raises(dkm.DkmError) as e:
        dkm.dkm_create_batched(np.zeros(max(n, 1) * d, np.float32), offsets, d, ks)
    assert e.value.status == dkm.DKM_EINVAL
    assert msg in dkm.dkm_last_error()


def test_batched_create_rejects_bad_cloud_count(dkm):
    status = dkm.lib().dkm_create_batched(None, None, None, 0, 3, None, None)
    assert status == dkm.DKM_EINVAL
    h = ctypes.c_void_p()
    pts = np.zeros(3, np.float32)
    off = np.zeros(2, np.int64)
    ks = np.ones(1, np.int32)
    status = dkm.lib().dkm_create_batched(ctypes.byref(h), pts.ctypes.data, off.ctypes.data,
                                          70_000, 3, ks.ctypes.data, None)
    assert status == dkm.DKM_EINVAL and "B must be" in dkm.dkm_last_error()
