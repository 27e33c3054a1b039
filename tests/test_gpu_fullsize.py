"""Parity with the FP64 oracle at the stated sizes of the three single-cloud
workloads (GPU required):

  geo2d-blobs  n = 1e5,  k = 100,   up to 20 passes, early stop
  geo2d-roads  n = 1e6,  k = 1000,  50 passes, coordinates up to 1e5
  lidar3d      n = 1e7,  k = 1e4,   30 passes

Lock-step protocol (Eq. 1 assignment, Algorithm 1 refine step; Section
II-B: index acceleration returns exactly Lloyd's result): at every pass
every context receives the same FP32 centroids C_t.
  - Labels: every indexed setting equals the plain brute-force GPU kernel
    bit for bit on all points; the GPU labels equal the oracle's except at
    near-ties (relative best/second gap below 1e-5) -- on all points where
    the oracle is affordable, else on a seeded sample of 2e5 points every
    pass and on all points at the first and the last pass.
  - Update: dkm_update from the pass's own sums, for every indexed
    setting, matches the oracle's update of the same labels within 1e-5 of
    the bounding-box extent; the cluster sizes are equal.
  - SSE: the pass SSE within 1e-4 relative of the oracle's (its minimum
    distances where all points are checked, else the FP64 SSE of the GPU
    labels).
  - Then C_{t+1} = the oracle's update, rounded to FP32.
The index settings are the defaults, coarser tiles (tile_cut_div 8), the
autotuner's usual choice on these workloads (tile_cut_div 2, row filter
off), the bound layer (the tile stay test, and the tile and point stay
tests) and hierarchical tiles (tile_group 4).  The free-running runs of the
two 2D workloads are replayed pass by pass and compared with oracle.fit."""
import numpy as np
import pytest

from paper_2412_02244_gb300 import synth
from gpu_util import (CENTROID_TOL, SSE_RTOL, check_labels, extent, gpu_assign, gpu_update,
                      make_ctx, replay_free_running, torch_cuda)

pytestmark = pytest.mark.gpu

SAMPLE = 200_000
SETTINGS = {
    "default": {},
    "coarse": dict(tile_cut_div=8),
    "tuned": dict(tile_cut_div=2, row_filter_min=256),
    "stay": dict(tile_cut_div=2, row_filter_min=256, stay_test=1),
    "pstay": dict(tile_cut_div=2, row_filter_min=256, stay_test=2),
    "group4": dict(tile_group=4),
}


@pytest.fixture(scope="module")
def dkm():
    torch_cuda()
    from paper_2412_02244_gb300 import build
    build.build()
    from paper_2412_02244_gb300 import dkm as m
    return m


def _lockstep(dkm, oracle, w, passes, sample=None, seed=0, stop_when_stable=False):
    pts = w.points
    n = w.n
    ext = extent(pts)
    ctxs = {}
    for name, setting in SETTINGS.items():
        ctxs[name] = make_ctx(dkm, pts, w.k)
        if setting:
            dkm.dkm_set_tuning(ctxs[name], **setting)
    ctx_b = make_ctx(dkm, pts, w.k, algo=dkm.DKM_ALGO_BRUTE)
    idx = None
    if sample is not None and sample < n:
        idx = np.sort(np.random.default_rng(seed).choice(n, size=sample, replace=False))
    C = w.init.copy()
    flips = 0
    stays = 0
    pstays = 0
    prev_o = None
    for t in range(passes):
        C64 = C.astype(np.float64)
        lab_b, sse_b, _ = gpu_assign(dkm, ctx_b, C)
        full = idx is None or t == 0 or t == passes - 1
        if full:
            lab_o, best, second = oracle.assign(pts, C64)
            flips += check_labels(lab_b, lab_o, best, second)
            s_ref = best.sum()
        else:
            lab_o, best, second = oracle.assign_subset(pts, idx, C64)
            flips += check_labels(lab_b[idx], lab_o, best, second)
            s_ref = oracle.sse(pts, lab_b, C64)
        assert abs(sse_b - s_ref) <= SSE_RTOL * s_ref, f"pass {t}: brute-force SSE"
        C_o, cnt_o = oracle.update(pts, lab_b, C64)
        for name, ctx in ctxs.items():
            lab, sse, _ = gpu_assign(dkm, ctx, C)
            assert np.array_equal(lab, lab_b), f"pass {t}, {name}: labels differ from brute force"
            assert abs(sse - sse_b) <= 1e-6 * sse_b, f"pass {t}, {name}: SSE"
            C_g, cnt_g = gpu_update(dkm, ctx, None, C)   # the pass's own sums
            assert np.array_equal(cnt_g, cnt_o), f"pass {t}, {name}: cluster sizes"
            err = np.abs(C_g.astype(np.float64) - C_o).max()
            assert err <= CENTROID_TOL * ext, \
                f"pass {t}, {name}: centroid error {err:.3g} > {CENTROID_TOL * ext:.3g}"
            if name == "stay":
                stays = max(stays, dkm.dkm_last_stats(ctx).stayed_tiles)
            if name == "pstay":
                pstays = max(pstays, dkm.dkm_last_stats(ctx).stayed_points)
        C = C_o.astype(np.float32)
        if stop_when_stable and prev_o is not None and np.array_equal(lab_o, prev_o):
            break
        prev_o = lab_o
    for ctx in list(ctxs.values()) + [ctx_b]:
        ctx.close()
    assert pstays > 0
    return flips, stays


def test_geo2d_blobs_full_size(dkm, oracle):
    w = synth.geo2d_blobs(seed=1)
    assert (w.n, w.k) == (100_000, 100)
    flips, stays = _lockstep(dkm, oracle, w, 20, stop_when_stable=True)
    assert flips <= 10
    assert stays > 0


def test_geo2d_blobs_full_size_free_running(dkm, oracle):
    w = synth.geo2d_blobs(seed=1)
    flips, agree = replay_free_running(dkm, oracle, w.points, w.k, w.init, 20, 1)
    assert flips <= 10


def test_geo2d_roads_full_size(dkm, oracle):
    w = synth.geo2d_roads(seed=2)
    assert (w.n, w.k) == (1_000_000, 1_000)
    flips, stays = _lockstep(dkm, oracle, w, 50)
    assert flips <= 100
    assert stays > 0


def test_geo2d_roads_full_size_free_running(dkm, oracle):
    w = synth.geo2d_roads(seed=2)
    flips, agree = replay_free_running(dkm, oracle, w.points, w.k, w.init, 50, 0)
    assert flips <= 100


def test_lidar3d_full_size(dkm, oracle):
    w = synth.lidar3d(seed=3)
    assert (w.n, w.k) == (10_000_000, 10_000)
    flips, stays = _lockstep(dkm, oracle, w, 30, sample=SAMPLE, seed=33)
    assert flips <= 200
    assert stays > 0
