"""Parity of the CUDA path with the FP64 oracle (GPU required).

Lock-step protocol: at every iteration both sides receive the same FP32
centroids; the GPU labels must equal the oracle's except at near-ties, the
GPU update of the GPU labels must match the oracle's update of the same
labels within 1e-5 of the bounding-box extent, the pass SSE must match
within 1e-4 relative; then both continue from the oracle's centroids
(rounded to FP32).  The indexed path must equal plain brute-force Lloyd on
the GPU bit for bit (Section II-B: index acceleration returns Lloyd's
result)."""
import numpy as np
import pytest

import oracle as oracle_pkg
from paper_2412_02244_gb300 import synth
from gpu_util import (CENTROID_TOL, SSE_RTOL, check_labels, dev, extent, gpu_assign, gpu_run,
                      gpu_update, make_ctx, replay_free_running, torch_cuda)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dkm():
    torch_cuda()
    from paper_2412_02244_gb300 import build
    build.build()
    from paper_2412_02244_gb300 import dkm as m
    return m


# scaled-down workloads: several blocks of 2048 points and a ragged tail
SMALL = {
    "geo2d-blobs": lambda: synth.geo2d_blobs(seed=11, n=20_011, k=40),
    "geo2d-roads": lambda: synth.geo2d_roads(seed=12, n=60_013, k=120, n_lines=60),
    "lidar3d": lambda: synth.lidar3d(seed=13, n=150_007, k=300, n_objects=40),
    "blobs3d": lambda: synth.batched3d(seed=14, n_clouds=1, log2_lo=14.0, log2_hi=14.01)[0],
}


@pytest.mark.parametrize("name", list(SMALL))
def test_lockstep_against_oracle(dkm, oracle, name):
    w = SMALL[name]()
    pts = w.points
    ext = extent(pts)
    ctx = make_ctx(dkm, pts, w.k)
    ctx_b = make_ctx(dkm, pts, w.k, algo=dkm.DKM_ALGO_BRUTE)
    C = w.init.copy()
    flips = 0
    for t in range(6):
        lab_g, sse_g, chg = gpu_assign(dkm, ctx, C)
        lab_b, sse_b, _ = gpu_assign(dkm, ctx_b, C)
        assert np.array_equal(lab_g, lab_b), f"pass {t}: indexed labels differ from brute force"
        assert sse_g == sse_b
        lab_o, best, second = oracle.assign(pts, C.astype(np.float64))
        flips += check_labels(lab_g, lab_o, best, second)
        assert abs(sse_g - best.sum()) <= SSE_RTOL * best.sum()
        if t == 0:
            assert chg == w.n
        # update of the GPU labels, explicit and reused-sums forms
        C_g, cnt_g = gpu_update(dkm, ctx, lab_g, C)
        gpu_assign(dkm, ctx, C)
        C_g2, cnt_g2 = gpu_update(dkm, ctx, None, C)
        assert np.array_equal(C_g, C_g2) and np.array_equal(cnt_g, cnt_g2)
        C_o, cnt_o = oracle.update(pts, lab_g, C.astype(np.float64))
        assert np.array_equal(cnt_g, cnt_o)
        err = np.abs(C_g.astype(np.float64) - C_o).max()
        assert err <= CENTROID_TOL * ext, f"pass {t}: centroid error {err:.3g} > {CENTROID_TOL * ext:.3g}"
        C = C_o.astype(np.float32)
    assert flips <= max(2, w.n // 10_000)


@pytest.mark.parametrize("name", list(SMALL))
def test_run_matches_lockstep_composition(dkm, name):
    """dkm_run(T) == T x (dkm_assign + dkm_update(NULL)), bit for bit."""
    w = SMALL[name]()
    ctx = make_ctx(dkm, w.points, w.k, early_stop=0)
    T = 5
    C_r, lab_r, it, sse_r = gpu_run(dkm, ctx, w.init, T)
    assert it == T
    C = w.init.copy()
    for _ in range(T):
        lab, _, _ = gpu_assign(dkm, ctx, C)
        C, _ = gpu_update(dkm, ctx, None, C)
    assert np.array_equal(C_r, C)
    assert np.array_equal(lab_r, lab)


@pytest.mark.parametrize("name", ["geo2d-blobs", "lidar3d"])
def test_free_running_fit_vs_oracle(dkm, oracle, name):
    """A free-running fit with early stop, every pass checked against the
    oracle at the GPU's own centroids (near-tie flips only), then against an
    independent oracle fit."""
    w = SMALL[name]()
    replay_free_running(dkm, oracle, w.points, w.k, w.init, 20, 1)


def test_early_stop_iterations_and_fixed_point(dkm, oracle):
    w = synth.geo2d_blobs(seed=21, n=8_000, k=12)
    ctx = make_ctx(dkm, w.points, w.k, early_stop=1)
    C_g, lab_g, it, sse = gpu_run(dkm, ctx, w.init, 100)
    assert 1 <= it < 100
    # a converged labelling is a fixed point of the assignment
    lab2, _, chg = gpu_assign(dkm, ctx, C_g)
    assert np.array_equal(lab2, lab_g)


def test_budget_and_grid_invariance(dkm):
    """Labels do not depend on the index configuration (exactness)."""
    w = SMALL["lidar3d"]()
    ref = None
    for opts in (dict(), dict(mem_budget_bytes=1 << 20), dict(cells_per_centroid=0.05),
                 dict(cells_per_centroid=16.0), dict(algo=1)):
        ctx = make_ctx(dkm, w.points, w.k, **opts)
        lab, sse, _ = gpu_assign(dkm, ctx, w.init)
        if ref is None:
            ref = (lab, sse)
        assert np.array_equal(lab, ref[0]), opts
        assert sse == ref[1], opts


def _oracle_case(dkm, oracle, pts, init, k, iters=4, **opts):
    ctx = make_ctx(dkm, pts, k, early_stop=0, **opts)
    C_g, lab_g, it, sse = gpu_run(dkm, ctx, init, iters)
    r = oracle.fit(pts, init.astype(np.float64), iters, early_stop=False)
    return C_g, lab_g, it, sse, r


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("n,k", [(1, 1), (37, 5), (64, 64), (2048 * 3 + 1, 17), (5000, 1)])
def test_edge_sizes(dkm, oracle, d, n, k):
    rng = np.random.default_rng(n * 10 + d)
    pts = rng.uniform(-5, 5, size=(n, d)).astype(np.float32)
    init = pts[rng.permutation(n)[:k]]
    C_g, lab_g, it, sse, r = _oracle_case(dkm, oracle, pts, init, k)
    assert it == 4
    assert np.array_equal(lab_g, r["labels"])
    assert np.abs(C_g - r["centroids"]).max() <= CENTROID_TOL * max(extent(pts), 1e-30)
    assert abs(sse - r["sse"]) <= SSE_RTOL * max(r["sse"], 1e-30) + 1e-12


def test_identical_points_and_duplicate_centroids(dkm, oracle):
    pts = np.full((3000, 3), 7.25, np.float32)
    init = np.full((4, 3), 7.25, np.float32)
    C_g, lab_g, it, sse, r = _oracle_case(dkm, oracle, pts, init, 4)
    assert np.all(lab_g == 0)                       # every tie goes to index 0
    assert np.array_equal(C_g, init)
    assert sse == 0.0


def test_empty_cluster_keeps_its_centroid(dkm, oracle):
    rng = np.random.default_rng(3)
    pts = rng.normal(0, 1, (4000, 2)).astype(np.float32)
    init = np.concatenate([pts[:5], np.array([[500.0, -500.0]], np.float32)])
    C_g, lab_g, it, sse, r = _oracle_case(dkm, oracle, pts, init, 6)
    assert not np.any(lab_g == 5)
    assert np.array_equal(C_g[5], init[5])
    assert np.array_equal(lab_g, r["labels"])


def test_each_point_its_own_cluster(dkm):
    rng = np.random.default_rng(4)
    pts = rng.uniform(0, 100, (700, 3)).astype(np.float32)
    ctx = make_ctx(dkm, pts, 700)
    lab, sse, _ = gpu_assign(dkm, ctx, pts)
    assert np.array_equal(lab, np.arange(700))
    assert sse == 0.0


def test_grid_overflow_path(dkm, oracle):
    """All centroids in one grid cell: most go to the overflow list."""
    rng = np.random.default_rng(5)
    pts = rng.uniform(0, 1000, (30_000, 2)).astype(np.float32)
    init = (rng.uniform(0, 1, (200, 2)) + 500).astype(np.float32)
    ctx = make_ctx(dkm, pts, 200)
    lab, sse, _ = gpu_assign(dkm, ctx, init)
    st = dkm.dkm_last_stats(ctx)
    assert st.grid_overflow > 0
    lab_o, best, second = oracle.assign(pts, init.astype(np.float64))
    check_labels(lab, lab_o, best, second)
    ctx_b = make_ctx(dkm, pts, 200, algo=1)
    assert np.array_equal(lab, gpu_assign(dkm, ctx_b, init)[0])


def test_candidate_list_overflow_fallback(dkm, oracle):
    """Blocks whose candidate list exceeds the buffer fall back to chunked
    search over all centroids and still return the exact result."""
    rng = np.random.default_rng(6)
    a = rng.normal(0, 1, (4096, 3))
    b = rng.normal(0, 1, (4096, 3)) + np.array([1000.0, 0, 0])
    pts = np.concatenate([a, b]).astype(np.float32)
    ang = rng.uniform(0, 2 * np.pi, 1500)
    ring = np.stack([np.full(1500, 500.0), 300 * np.cos(ang), 300 * np.sin(ang)], 1)
    init = np.concatenate([ring, pts[:2]]).astype(np.float32)
    k = init.shape[0]
    ctx = make_ctx(dkm, pts, k)
    lab, sse, _ = gpu_assign(dkm, ctx, init)
    st = dkm.dkm_last_stats(ctx)
    assert st.fallback_tiles > 0
    lab_o, best, second = oracle.assign(pts, init.astype(np.float64))
    check_labels(lab, lab_o, best, second)
    assert np.array_equal(lab, gpu_assign(dkm, make_ctx(dkm, pts, k, algo=1), init)[0])


def test_large_coordinates_2d(dkm, oracle):
    """Coordinates near 1e5 (the geo workload): difference-form distances."""
    w = synth.geo2d_roads(seed=31, n=40_000, k=80, n_lines=40)
    pts = (w.points + np.float32(5e4)).astype(np.float32)
    init = (w.init + np.float32(5e4)).astype(np.float32)
    ctx = make_ctx(dkm, pts, w.k)
    lab, sse, _ = gpu_assign(dkm, ctx, init)
    lab_o, best, second = oracle.assign(pts, init.astype(np.float64))
    check_labels(lab, lab_o, best, second)
    assert abs(sse - best.sum()) <= SSE_RTOL * best.sum()


def test_max_iter_zero(dkm, oracle):
    w = SMALL["geo2d-blobs"]()
    ctx = make_ctx(dkm, w.points, w.k)
    C, lab, it, sse = gpu_run(dkm, ctx, w.init, 0)
    assert it == 0
    assert np.array_equal(C, w.init)
    lab_o, best, second = oracle.assign(w.points, w.init.astype(np.float64))
    check_labels(lab, lab_o, best, second)


def test_host_buffers_match_device_buffers(dkm):
    """The end-to-end path (numpy in, numpy out) equals the device path."""
    w = SMALL["lidar3d"]()
    n, d, k = w.n, w.d, w.k
    o = dkm.dkm_default_options(early_stop=0)
    C_h = np.empty((k, d), np.float32)
    lab_h = np.empty(n, np.int32)
    it_h, sse_h = dkm.dkm_fit(w.points, n, d, k, w.init, 7, C_h, lab_h, o)
    torch = torch_cuda()
    C_d = torch.empty(k * d, dtype=torch.float32, device="cuda")
    lab_d = torch.empty(n, dtype=torch.int32, device="cuda")
    it_d, sse_d = dkm.dkm_fit(dev(w.points), n, d, k, dev(w.init), 7, C_d, lab_d, o)
    assert it_h == it_d == 7 and sse_h == sse_d
    assert np.array_equal(C_h.ravel(), C_d.cpu().numpy())
    assert np.array_equal(lab_h, lab_d.cpu().numpy())


@pytest.mark.parametrize("early_stop,profile", [(0, 0), (1, 0), (0, 1)])
def test_one_shot_fit_equals_context_run(dkm, early_stop, profile):
    """dkm_fit launches the run's kernels directly instead of capturing a
    graph; its outputs equal a context's dkm_run (graph launch) bit for bit."""
    torch = torch_cuda()
    w = SMALL["geo2d-blobs"]()
    n, d, k = w.n, w.d, w.k
    o = dkm.dkm_default_options(early_stop=early_stop, profile=profile)
    C_f = torch.empty(k * d, dtype=torch.float32, device="cuda")
    lab_f = torch.empty(n, dtype=torch.int32, device="cuda")
    it_f, sse_f = dkm.dkm_fit(dev(w.points), n, d, k, dev(w.init), 20, C_f, lab_f, o)
    ctx = make_ctx(dkm, w.points, k, early_stop=early_stop, profile=profile)
    C_r, lab_r, it_r, sse_r = gpu_run(dkm, ctx, w.init, 20)
    ctx.close()
    assert it_f == it_r and sse_f == sse_r
    assert np.array_equal(C_f.cpu().numpy().reshape(k, d), C_r)
    assert np.array_equal(lab_f.cpu().numpy(), lab_r)


def test_setup_reuse_new_points(dkm, oracle):
    w1 = synth.lidar3d(seed=41, n=50_000, k=64, n_objects=20)
    w2 = synth.lidar3d(seed=42, n=50_000, k=64, n_objects=20)
    ctx = make_ctx(dkm, w1.points, 64)
    dkm.dkm_setup(ctx, dev(w2.points))
    lab, sse, _ = gpu_assign(dkm, ctx, w2.init)
    lab_o, best, second = oracle.assign(w2.points, w2.init.astype(np.float64))
    check_labels(lab, lab_o, best, second)


def test_errors(dkm):
    w = SMALL["geo2d-blobs"]()
    ctx = make_ctx(dkm, w.points, w.k)
    bad = w.init.copy()
    bad[3, 1] = np.nan
    with pytest.raises(dkm.DkmError) as e:
        gpu_assign(dkm, ctx, bad)
    assert e.value.status == dkm.DKM_EINVAL
    # still usable afterwards
    gpu_assign(dkm, ctx, w.init)
    labels = np.zeros(w.n, np.int32)
    labels[17] = w.k        # out of range
    torch = torch_cuda()
    C = dev(w.init).clone()
    with pytest.raises(dkm.DkmError) as e:
        dkm.dkm_update(ctx, dev(labels), C, None)
    assert e.value.status == dkm.DKM_EINVAL
    assert np.array_equal(C.cpu().numpy(), w.init)
    with pytest.raises(dkm.DkmError):
        dkm.dkm_update(make_ctx(dkm, w.points, w.k), None, C, None)   # no preceding assign
    pts = w.points.copy()
    pts[5, 0] = np.inf
    with pytest.raises(dkm.DkmError) as e:
        make_ctx(dkm, pts, w.k)
    assert e.value.status == dkm.DKM_EINVAL


def test_sse_history_non_increasing(dkm):
    """Per-pass SSE (labels against the centroids they were assigned with)
    never increases in Lloyd's algorithm."""
    w = SMALL["geo2d-roads"]()
    ctx = make_ctx(dkm, w.points, w.k)
    C = w.init.copy()
    prev = np.inf
    for _ in range(8):
        lab, sse, _ = gpu_assign(dkm, ctx, C)
        assert sse <= prev * (1 + 1e-6)
        prev = sse
        C, _ = gpu_update(dkm, ctx, None, C)


def test_run_graph_reuse_across_setups(dkm):
    """A run after re-running dkm_setup equals a fresh context bit for bit,
    whether the cached run graph is kept (same points) or rebuilt (new
    points of the same size)."""
    a = synth.lidar3d(seed=71, n=50_003, k=70, n_objects=20)
    b = synth.lidar3d(seed=72, n=50_003, k=70, n_objects=25)
    ctx = make_ctx(dkm, a.points, a.k, early_stop=0)
    first = gpu_run(dkm, ctx, a.init, 7)
    dkm.dkm_setup(ctx, dev(a.points))
    again = gpu_run(dkm, ctx, a.init, 7)
    for x, y in zip(first, again):
        assert np.array_equal(x, y)
    dkm.dkm_setup(ctx, dev(b.points))
    moved = gpu_run(dkm, ctx, b.init, 7)
    fresh = gpu_run(dkm, make_ctx(dkm, b.points, b.k, early_stop=0), b.init, 7)
    for x, y in zip(moved, fresh):
        assert np.array_equal(x, y)


def test_bounded_sort_wait_gives_up_and_the_device_stays_usable(dkm):
    """The radix sort of dkm_setup is the library's one device-side wait
    (decoupled look-back).  Its self-test hands the only CTA of a pass the
    second tile, so the count it waits for is never published: the wait
    must end by itself after about a second and report it, and the device
    must keep working (a full fit afterwards matches the oracle)."""
    sec = dkm.dkm_selftest_wait()
    assert 0.5 < sec < 30.0
    w = synth.lidar3d(seed=73, n=20_011, k=40, n_objects=10)
    lab_o, best, second = oracle_pkg.get().assign(w.points, w.init)
    lab_g, sse_g, _ = gpu_assign(dkm, make_ctx(dkm, w.points, w.k), w.init)
    check_labels(lab_g, lab_o, best, second)


@pytest.mark.parametrize("d", [2, 3])
def test_exact_ties_survive_pruning(dkm, oracle, d):
    """Points and centroids on integer lattices, so every d^2 is exact in
    FP32 and FP64: each point with an odd coordinate is exactly equidistant
    from 2, 4 or 8 centroids, and the centroid order is shuffled, so the
    lowest index is spatially arbitrary; some centroids are duplicated.
    The ball bound and the dominance test must keep every tied centroid
    that the lowest index decides for: labels equal brute force and the
    oracle exactly, with no near-tie allowance."""
    rng = np.random.default_rng(11 + d)
    g = np.arange(0, 48, 2, dtype=np.float32)
    axes = [g, g] if d == 2 else [g, g, g[:6]]
    C = np.stack(np.meshgrid(*axes, indexing="ij"), -1).reshape(-1, d)
    C = np.concatenate([C, C[rng.choice(len(C), 40, replace=False)]])   # duplicates
    C = np.ascontiguousarray(C[rng.permutation(len(C))])
    q = np.arange(0, 47, dtype=np.float32)
    paxes = [q, q] if d == 2 else [q, q, q[:11]]
    P = np.stack(np.meshgrid(*paxes, indexing="ij"), -1).reshape(-1, d)
    P = np.ascontiguousarray(P[rng.permutation(len(P))])
    k = len(C)
    lab_o, best, second = oracle.assign(P, C)
    assert np.count_nonzero(best == second) > len(P) // 4   # many exact ties
    for algo in (dkm.DKM_ALGO_INDEXED, dkm.DKM_ALGO_BRUTE):
        lab_g, _, _ = gpu_assign(dkm, make_ctx(dkm, P, k, algo=algo), C)
        assert np.array_equal(lab_g, lab_o)


@pytest.mark.parametrize("profile,expect", [(1, 4), (10, 2), (20, 1), (50, 1)])
def test_profiled_passes_and_unchanged_results(dkm, profile, expect):
    """opts.profile sets how many passes carry CUDA events (one in each
    period, 5 for profile = 1); profiling never changes a result."""
    w = synth.lidar3d(seed=74, n=40_009, k=60, n_objects=12)
    plain = gpu_run(dkm, make_ctx(dkm, w.points, w.k, early_stop=0), w.init, 20)
    ctx = make_ctx(dkm, w.points, w.k, early_stop=0, profile=profile)
    prof = gpu_run(dkm, ctx, w.init, 20)
    for x, y in zip(plain, prof):
        assert np.array_equal(x, y)
    T = dkm.dkm_last_timings(ctx)
    assert T.passes == expect
    assert T.assign_ms > 0 and T.search_ms > 0 and T.iterations_ms > 0
