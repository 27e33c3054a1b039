"""Batched contexts (B independent clouds in one context) against the FP64
oracle, cloud by cloud.

Each cloud of a batch is its own Lloyd problem (Eq. 1, Algorithm 1); the
batch only shares launches.  So every check compares cloud b of the batch
with the oracle run on cloud b alone: lock-step labels and updates, the
graph-captured run against the per-pass composition, a free-running fit
with per-cloud early stop, and the 512-cloud uneven workload at full size
(all 25 passes in lock-step: labels on sampled points every pass and on all
points at the first and last pass, updates and SSE on all points)."""
import numpy as np
import pytest

from paper_2412_02244_gb300 import synth
from gpu_util import (CENTROID_TOL, SSE_RTOL, check_labels, dev, extent, gpu_assign,
                      gpu_update, torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dkm():
    torch_cuda()
    from paper_2412_02244_gb300 import build
    build.build()
    from paper_2412_02244_gb300 import dkm as m
    return m


def _batch(ws, d=3):
    P = np.ascontiguousarray(np.concatenate([w.points[:, :d] for w in ws]).astype(np.float32))
    off = np.zeros(len(ws) + 1, np.int64)
    off[1:] = np.cumsum([w.n for w in ws])
    ks = np.array([w.k for w in ws], np.int32)
    coff = np.zeros(len(ws) + 1, np.int64)
    coff[1:] = np.cumsum(ks)
    init = np.ascontiguousarray(np.concatenate([w.init[:, :d] for w in ws]).astype(np.float32))
    return P, off, ks, coff, init


def _small(d=3, seed=41, n_clouds=9):
    # uneven clouds of 256 .. 8192 points: ragged tails, clouds shorter than
    # a tile window, clouds spanning several windows
    ws = synth.batched3d(seed=seed, n_clouds=n_clouds, log2_lo=8.0, log2_hi=13.0)
    return _batch(ws, d)


def _ctx(dkm, P, off, ks, **opts):
    return dkm.dkm_create_batched(dev(P), off, P.shape[1], ks, dkm.dkm_default_options(**opts))


def _run(dkm, ctx, init, T):
    torch = torch_cuda()
    C = torch.empty(ctx.k * ctx.d, dtype=torch.float32, device="cuda")
    lab = torch.empty(ctx.n, dtype=torch.int32, device="cuda")
    it, sse = dkm.dkm_run_batched(ctx, dev(init), T, C, lab)
    return C.cpu().numpy().reshape(ctx.k, ctx.d), lab.cpu().numpy(), it, sse


@pytest.mark.parametrize("d", [2, 3])
def test_batched_lockstep_against_oracle(dkm, oracle, d):
    P, off, ks, coff, init = _small(d)
    B = len(ks)
    ctx = _ctx(dkm, P, off, ks)
    ctx_b = _ctx(dkm, P, off, ks, algo=dkm.DKM_ALGO_BRUTE)
    C = init.copy()
    flips = 0
    for t in range(5):
        lab_g, sse_g, chg = gpu_assign(dkm, ctx, C)
        lab_b, sse_b, _ = gpu_assign(dkm, ctx_b, C)
        assert np.array_equal(lab_g, lab_b), f"pass {t}: indexed labels differ from brute force"
        assert sse_g == sse_b
        if t == 0:
            assert chg == P.shape[0]
        C_g, cnt_g = gpu_update(dkm, ctx, lab_g, C)
        C_next = np.empty_like(C)
        sse_o = 0.0
        for b in range(B):
            ps, cs = slice(off[b], off[b + 1]), slice(coff[b], coff[b + 1])
            Pb, Cb = P[ps], C[cs].astype(np.float64)
            lab_o, best, second = oracle.assign(Pb, Cb)
            assert lab_g[ps].min() >= 0 and lab_g[ps].max() < ks[b]
            flips += check_labels(lab_g[ps], lab_o, best, second)
            sse_o += best.sum()
            C_o, cnt_o = oracle.update(Pb, lab_g[ps], Cb)
            assert np.array_equal(cnt_g[cs], cnt_o), f"pass {t} cloud {b}: counts differ"
            err = np.abs(C_g[cs].astype(np.float64) - C_o).max()
            assert err <= CENTROID_TOL * extent(Pb), f"pass {t} cloud {b}: centroid error {err:.3g}"
            C_next[cs] = C_o.astype(np.float32)
        assert abs(sse_g - sse_o) <= SSE_RTOL * sse_o
        C = C_next
    assert flips <= 2


def test_batched_run_matches_lockstep_composition(dkm):
    """dkm_run_batched(T) == T x (dkm_assign + dkm_update(NULL)), bit for bit."""
    P, off, ks, coff, init = _small(3, seed=43)
    ctx = _ctx(dkm, P, off, ks, early_stop=0)
    T = 5
    C_r, lab_r, it, sse_r = _run(dkm, ctx, init, T)
    assert np.all(it == T)
    C = init.copy()
    for _ in range(T):
        lab, _, _ = gpu_assign(dkm, ctx, C)
        C, _ = gpu_update(dkm, ctx, None, C)
    assert np.array_equal(C_r, C)
    assert np.array_equal(lab_r, lab)


def test_batched_fit_vs_oracle_per_cloud_early_stop(dkm, oracle):
    """Free-running fit with early stop: each cloud stops on its own."""
    P, off, ks, coff, init = _small(3, seed=45, n_clouds=12)
    B = len(ks)
    C_g = np.empty_like(init)
    lab_g = np.empty(P.shape[0], np.int32)
    it, sse = dkm.dkm_fit_batched(P, off, 3, ks, init, 40, C_g, lab_g,
                                  opts=dkm.dkm_default_options(early_stop=1))
    assert len(set(it.tolist())) > 1, "clouds should converge after different pass counts"
    for b in range(B):
        ps, cs = slice(off[b], off[b + 1]), slice(coff[b], coff[b + 1])
        Pb = P[ps]
        r = oracle.fit(Pb, init[cs].astype(np.float64), 40, early_stop=True)
        Cb = C_g[cs].astype(np.float64)
        assert abs(sse[b] - oracle.sse(Pb, lab_g[ps], Cb)) <= SSE_RTOL * sse[b]
        assert abs(sse[b] - r["sse"]) <= SSE_RTOL * r["sse"]
        agree = np.mean(lab_g[ps] == r["labels"])
        assert agree > 0.995, f"cloud {b}: label agreement {agree}"
        if agree == 1.0:
            assert it[b] == r["iterations"], f"cloud {b}"
            assert np.abs(C_g[cs] - r["centroids"]).max() <= CENTROID_TOL * extent(Pb)


def test_single_cloud_batch_equals_plain_context(dkm):
    """A batch of one cloud is the plain context, bit for bit."""
    w = synth.lidar3d(seed=47, n=40_003, k=90, n_objects=20)
    P = np.ascontiguousarray(w.points.astype(np.float32))
    off = np.array([0, w.n], np.int64)
    ks = np.array([w.k], np.int32)
    ctx1 = _ctx(dkm, P, off, ks, early_stop=0)
    ctx0 = dkm.dkm_create(dev(P), w.n, 3, w.k, dkm.dkm_default_options(early_stop=0))
    C1, lab1, it1, sse1 = _run(dkm, ctx1, w.init, 6)
    torch = torch_cuda()
    C0 = torch.empty(w.k * 3, dtype=torch.float32, device="cuda")
    lab0 = torch.empty(w.n, dtype=torch.int32, device="cuda")
    it0, sse0 = dkm.dkm_run(ctx0, dev(w.init), 6, C0, lab0)
    assert np.array_equal(C1, C0.cpu().numpy().reshape(w.k, 3))
    assert np.array_equal(lab1, lab0.cpu().numpy())
    assert it1[0] == it0 and sse1[0] == sse0


def test_batched_stats_and_plan(dkm):
    P, off, ks, coff, init = _small(3, seed=49)
    ctx = _ctx(dkm, P, off, ks)
    gpu_assign(dkm, ctx, init)
    st = dkm.dkm_last_stats(ctx)
    windows = -(-P.shape[0] // 256)
    assert windows <= st.tiles <= windows + windows // 8 + 3 * len(ks) + 2
    assert st.evals_per_point >= 1.0
    plan = dkm.dkm_get_plan(ctx)
    assert plan.cells >= len(ks)
    dev_bytes, idx_bytes = dkm.dkm_query_memory(ctx)
    assert idx_bytes <= dkm.dkm_default_options().mem_budget_bytes
    assert idx_bytes < dev_bytes


def test_batched_uneven_workload_full_size(dkm, oracle):
    """512 clouds, n_i log-uniform in [2^10, 2^17], k_i = max(8, n_i / 100),
    25 passes, one launch per kernel per pass for all clouds.  Checked at full
    size: labels of pass 25 on 64 sampled points per cloud against the
    oracle's assignment with the same centroids, the update of all points
    against the oracle's update, the SSE of all points, and the graph run
    against the per-pass composition."""
    torch = torch_cuda()
    ws = synth.batched3d(seed=4)
    P, off, ks, coff, init = _batch(ws)
    B = len(ks)
    ctx = _ctx(dkm, P, off, ks, early_stop=0)
    C24, _, it24, _ = _run(dkm, ctx, init, 24)
    assert np.all(it24 == 24)
    C25, lab25, it25, sse25 = _run(dkm, ctx, init, 25)
    assert np.all(it25 == 25)
    lab_g, _, _ = gpu_assign(dkm, ctx, C24)
    assert np.array_equal(lab_g, lab25)
    C_u, cnt_u = gpu_update(dkm, ctx, lab_g, C24)
    rng = np.random.default_rng(4)
    flips = 0
    for b in range(B):
        ps, cs = slice(off[b], off[b + 1]), slice(coff[b], coff[b + 1])
        Pb, Cb = P[ps], C24[cs].astype(np.float64)
        idx = np.sort(rng.choice(Pb.shape[0], size=64, replace=False)).astype(np.int64)
        lab_o, best, second = oracle.assign_subset(Pb, idx, Cb)
        flips += check_labels(lab_g[ps][idx], lab_o, best, second)
        C_o, cnt_o = oracle.update(Pb, lab_g[ps], Cb)
        assert np.array_equal(cnt_u[cs], cnt_o)
        assert np.abs(C_u[cs].astype(np.float64) - C_o).max() <= CENTROID_TOL * extent(Pb)
        s_o = oracle.sse(Pb, lab25[ps], C25[cs].astype(np.float64))
        assert abs(sse25[b] - s_o) <= SSE_RTOL * s_o, f"cloud {b}"
    assert flips <= 2
    # the run's final centroids are the 25th update of the composition
    assert np.array_equal(C25, C_u)


def test_batched_full_size_lockstep(dkm, oracle):
    """The 512-cloud workload at full size (Σn = 14.3M, Σk = 142,788), all 25
    passes in lock-step with the oracle, cloud by cloud (Eq. 1; Algorithm 1's
    refine step): every pass the indexed labels equal the GPU brute force on
    all points; the labels equal the oracle's except at near-ties on a seeded
    sample of 256 points per cloud, and on all points at the first and the
    last pass; the update from the pass's own sums equals the oracle's update
    of the same labels within 1e-5 of each cloud's extent, with equal cluster
    sizes; the pass SSE is within 1e-4 of the oracle's SSE of those labels.
    Then C_{t+1} = the oracle's update, rounded to FP32."""
    ws = synth.batched3d(seed=4)
    P, off, ks, coff, init = _batch(ws)
    B = len(ks)
    ctx = _ctx(dkm, P, off, ks)
    dkm.dkm_set_tuning(ctx, cells_per_centroid=2.0, tile_cut_div=1, row_filter_min=256)
    ctx_b = _ctx(dkm, P, off, ks, algo=dkm.DKM_ALGO_BRUTE)
    rng = np.random.default_rng(44)
    idx = [np.sort(rng.choice(int(off[b + 1] - off[b]), size=256, replace=False)).astype(np.int64)
           for b in range(B)]
    ext = [extent(P[off[b]:off[b + 1]]) for b in range(B)]
    C = init.copy()
    flips = 0
    passes = 25
    for t in range(passes):
        lab_g, sse_g, _ = gpu_assign(dkm, ctx, C)
        lab_b, sse_b, _ = gpu_assign(dkm, ctx_b, C)
        assert np.array_equal(lab_g, lab_b), f"pass {t}: indexed labels differ from brute force"
        C_g, cnt_g = gpu_update(dkm, ctx, None, C)   # the pass's own sums
        full = t == 0 or t == passes - 1
        C_next = np.empty_like(C)
        sse_o = 0.0
        for b in range(B):
            ps, cs = slice(off[b], off[b + 1]), slice(coff[b], coff[b + 1])
            Pb, Cb = P[ps], C[cs].astype(np.float64)
            if full:
                lab_o, best, second = oracle.assign(Pb, Cb)
                flips += check_labels(lab_g[ps], lab_o, best, second)
            else:
                lab_o, best, second = oracle.assign_subset(Pb, idx[b], Cb)
                flips += check_labels(lab_g[ps][idx[b]], lab_o, best, second)
            sse_o += oracle.sse(Pb, lab_g[ps], Cb)
            C_o, cnt_o = oracle.update(Pb, lab_g[ps], Cb)
            assert np.array_equal(cnt_g[cs], cnt_o), f"pass {t} cloud {b}: cluster sizes"
            err = np.abs(C_g[cs].astype(np.float64) - C_o).max()
            assert err <= CENTROID_TOL * ext[b], f"pass {t} cloud {b}: centroid error {err:.3g}"
            C_next[cs] = C_o.astype(np.float32)
        assert abs(sse_g - sse_o) <= SSE_RTOL * sse_o, f"pass {t}: SSE"
        C = C_next
    ctx.close()
    ctx_b.close()
    assert flips <= 50


@pytest.mark.parametrize("setting", [dict(cells_per_centroid=0.5), dict(cells_per_centroid=4.0),
                                     dict(tile_cut_div=1), dict(tile_cut_div=32),
                                     dict(row_filter_min=16), dict(row_filter_min=256),
                                     dict(sort_max=32), dict(sort_max=16),
                                     dict(tile_group=4), dict(tile_group=32),
                                     dict(tile_group=8, sort_max=32), dict(stay_test=1),
                                     dict(stay_test=1, sort_max=32), dict(stay_test=2),
                                     dict(stay_test=2, row_filter_min=16)])
def test_tuning_settings_keep_labels_exact(dkm, oracle, setting):
    """Every index setting labels exactly like brute force, and cloud by
    cloud like the FP64 oracle (near-ties aside); the setting's own update
    sums match the oracle's update of those labels.  The SSE is a sum of
    per-tile fixed-point partials (each tile at its own power-of-two scale),
    so a setting that regroups the tiles moves its last bits: it is compared
    to 1e-6 relative, the labels bit for bit.  Lock-step: both sides continue
    from the oracle's centroids; six passes, so that the bound layer's stay
    test (Section IV-A) has tiles to keep."""
    P, off, ks, coff, init = _small(3, seed=51)
    ctx = _ctx(dkm, P, off, ks)
    ctx_b = _ctx(dkm, P, off, ks, algo=dkm.DKM_ALGO_BRUTE)
    dkm.dkm_set_tuning(ctx, **setting)
    t = dkm.dkm_get_tuning(ctx)
    for k, v in setting.items():
        assert getattr(t, k) == pytest.approx(v)
    C = init.copy()
    flips = 0
    stays = 0
    pstays = 0
    for _ in range(6):
        lab, sse, _ = gpu_assign(dkm, ctx, C)
        lab_b, sse_b, _ = gpu_assign(dkm, ctx_b, C)
        assert np.array_equal(lab, lab_b)
        assert abs(sse - sse_b) <= 1e-6 * sse_b
        st = dkm.dkm_last_stats(ctx)
        stays += st.stayed_tiles
        pstays += st.stayed_points
        C_g, _ = gpu_update(dkm, ctx, None, C)
        C_next = np.empty_like(C)
        for b in range(len(ks)):
            ps, cs = slice(off[b], off[b + 1]), slice(coff[b], coff[b + 1])
            Pb, Cb = P[ps], C[cs].astype(np.float64)
            lo, best, second = oracle.assign(Pb, Cb)
            flips += check_labels(lab[ps], lo, best, second)
            C_o, _ = oracle.update(Pb, lab[ps], Cb)
            err = np.abs(C_g[cs].astype(np.float64) - C_o).max()
            assert err <= CENTROID_TOL * extent(Pb), f"cloud {b}: centroid error {err:.3g}"
            C_next[cs] = C_o.astype(np.float32)
        C = C_next
    assert flips <= 2
    if setting.get("stay_test"):
        assert stays > 0
    if setting.get("stay_test") == 2:
        assert pstays > 0


def test_autotune_choice_cache_and_exactness(dkm):
    P, off, ks, coff, init = _small(3, seed=53, n_clouds=16)
    ctx = _ctx(dkm, P, off, ks)
    lab0, sse0, _ = gpu_assign(dkm, ctx, init)
    t = dkm.dkm_autotune(ctx, dev(init), passes=2, use_cache=False)
    assert t.from_cache == 0 and t.trials >= 10
    assert 0 < t.ms_per_pass <= t.ms_per_pass_before
    assert t.cells_per_centroid in (0.5, 1.0, 2.0, 4.0)
    assert t.tile_cut_div in (1, 2, 4, 8, 16, 32) and t.row_filter_min in (16, 32, 48, 96, 256)
    assert t.sort_max in (0, 16, 32) and t.tile_group in (1, 2, 4, 8, 16)
    assert t.stay_test in (0, 1, 2)
    cur = dkm.dkm_get_tuning(ctx)
    assert (cur.cells_per_centroid, cur.tile_cut_div, cur.row_filter_min) == \
        (t.cells_per_centroid, t.tile_cut_div, t.row_filter_min)
    lab1, sse1, _ = gpu_assign(dkm, ctx, init)
    assert np.array_equal(lab0, lab1) and abs(sse0 - sse1) <= 1e-6 * sse0
    ctx2 = _ctx(dkm, P, off, ks)
    t2 = dkm.dkm_autotune(ctx2, dev(init), passes=2, use_cache=True)
    assert t2.from_cache == 1
    assert (t2.cells_per_centroid, t2.tile_cut_div, t2.row_filter_min) == \
        (t.cells_per_centroid, t.tile_cut_div, t.row_filter_min)


def test_tuning_rejects_bad_values(dkm):
    P, off, ks, coff, init = _small(3, seed=55, n_clouds=3)
    ctx = _ctx(dkm, P, off, ks)
    for kw in (dict(cells_per_centroid=0.0), dict(cells_per_centroid=100.0),
               dict(tile_cut_div=0), dict(row_filter_min=-1), dict(sort_max=33),
               dict(tile_group=0), dict(tile_group=33), dict(stay_test=3)):
        with pytest.raises(dkm.DkmError) as e:
            dkm.dkm_set_tuning(ctx, **kw)
        assert e.value.status == dkm.DKM_EINVAL
    with pytest.raises(dkm.DkmError):
        dkm.dkm_autotune(ctx, dev(init), passes=0)


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("batched", [False, True])
def test_stay_test_gives_the_same_run_bit_for_bit(dkm, oracle, batched, level):
    """The bound layer only skips searches whose outcome it has proved, so a
    run with it equals the run without it in every bit, and near
    convergence some tiles do stay."""
    if batched:
        P, off, ks, coff, init = _small(3, seed=57, n_clouds=6)
    else:
        w = synth.lidar3d(seed=58, n=60_011, k=60, n_objects=20)
        P, init = np.ascontiguousarray(w.points), w.init
        off, ks = np.array([0, w.n], np.int64), np.array([w.k], np.int32)
    out = []
    for stay in (0, level):
        ctx = _ctx(dkm, P, off, ks, early_stop=0)
        dkm.dkm_set_tuning(ctx, stay_test=stay)
        out.append(_run(dkm, ctx, init, 12))
        st = dkm.dkm_last_stats(ctx)
        if stay:
            assert st.stayed_tiles > 0
        else:
            assert st.stayed_tiles == 0
        if stay == 2:
            assert st.stayed_points > 0
    (C0, l0, i0, s0), (C1, l1, i1, s1) = out
    assert np.array_equal(C0, C1) and np.array_equal(l0, l1)
    assert np.array_equal(i0, i1) and np.array_equal(s0, s1)
    # and the bound layer keeps Lloyd's result: after the same run, one more
    # pass with the stay test from the run's final centroids labels every
    # cloud like the oracle (near-ties aside) and updates like the oracle
    ctx = _ctx(dkm, P, off, ks, early_stop=0)
    dkm.dkm_set_tuning(ctx, stay_test=level)
    _run(dkm, ctx, init, 12)
    lab, _, _ = gpu_assign(dkm, ctx, C1)
    C_g, _ = gpu_update(dkm, ctx, None, C1)
    coff = np.zeros(len(ks) + 1, np.int64)
    coff[1:] = np.cumsum(ks)
    flips = 0
    for b in range(len(ks)):
        ps, cs = slice(off[b], off[b + 1]), slice(coff[b], coff[b + 1])
        Pb, Cb = P[ps], C1[cs].astype(np.float64)
        lo, best, second = oracle.assign(Pb, Cb)
        flips += check_labels(lab[ps], lo, best, second)
        C_o, _ = oracle.update(Pb, lab[ps], Cb)
        assert np.abs(C_g[cs].astype(np.float64) - C_o).max() <= CENTROID_TOL * extent(Pb)
    assert flips <= 2
    assert dkm.dkm_last_stats(ctx).stayed_tiles > 0
