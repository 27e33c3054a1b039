"""Helpers for the GPU tests: device copies through torch and thin wrappers
that call the C ABI (via the binding) and bring results back to numpy."""
import numpy as np


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def dev(a, torch=None):
    torch = torch or torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_ctx(dkm, pts, k, **opts):
    o = dkm.dkm_default_options(**opts)
    n, d = pts.shape
    return dkm.dkm_create(dev(pts.astype(np.float32)), n, d, k, o)


def gpu_assign(dkm, ctx, C):
    torch = torch_cuda()
    lab = torch.empty(ctx.n, dtype=torch.int32, device="cuda")
    sse, chg = dkm.dkm_assign(ctx, dev(np.asarray(C, np.float32)), lab)
    return lab.cpu().numpy(), sse, chg


def gpu_update(dkm, ctx, labels, C):
    torch = torch_cuda()
    c = dev(np.asarray(C, np.float32)).clone()
    cnt = torch.empty(ctx.k, dtype=torch.int32, device="cuda")
    dkm.dkm_update(ctx, None if labels is None else dev(labels.astype(np.int32)), c, cnt)
    return c.cpu().numpy(), cnt.cpu().numpy()


def gpu_run(dkm, ctx, init, max_iter):
    torch = torch_cuda()
    C = torch.empty(ctx.k * ctx.d, dtype=torch.float32, device="cuda")
    lab = torch.empty(ctx.n, dtype=torch.int32, device="cuda")
    it, sse = dkm.dkm_run(ctx, dev(np.asarray(init, np.float32)), max_iter, C, lab)
    return C.cpu().numpy().reshape(ctx.k, ctx.d), lab.cpu().numpy(), it, sse


def extent(pts):
    return float(np.max(pts.max(axis=0).astype(np.float64) - pts.min(axis=0)))


# Parity rule: labels identical except near-ties (oracle best/second gap
# below 1e-5 relative); centroids within 1e-5 of the bounding-box extent;
# SSE within 1e-4 relative.
LABEL_GAP = 1e-5
CENTROID_TOL = 1e-5
SSE_RTOL = 1e-4


def check_labels(lab_g, lab_o, best, second):
    from oracle import relative_gap
    bad = lab_g != lab_o
    if not bad.any():
        return 0
    gap = relative_gap(best[bad], second[bad])
    assert np.all(gap < LABEL_GAP), (
        f"{int(bad.sum())} labels differ; {int((gap >= LABEL_GAP).sum())} of them are not "
        f"near-ties (max gap {gap.max():.3g})")
    return int(bad.sum())


def replay_free_running(dkm, oracle, pts, k, init, max_iter, early_stop, **opts):
    """A free-running dkm_run checked against the FP64 oracle pass by pass.

    dkm_run equals the composition of dkm_assign + dkm_update(NULL) bit for
    bit, so the run's trajectory is replayed one pass at a time on a second
    context, and every pass is checked against the oracle at the GPU's own
    centroids: labels equal except near-ties (Eq. 1 argmin), the update of
    those labels within the centroid tolerance (Algorithm 1 refine step).
    The run's final labels and centroids must equal the replay's bit for
    bit.  Then the run is compared with an independent oracle.fit, whose
    centroids stay in FP64 from pass to pass while the GPU's are rounded to
    FP32 (the caller's type): the two trajectories differ by that rounding,
    which near the end of a long run moves more labels than the near-tie
    band of one pass covers (coordinates near 1e5 have an FP32 ulp of
    0.008).  So the final SSE must agree within 1e-4; when the final labels
    agree too, so must the pass count and the centroids.
    Returns (near-tie flips seen, fraction of final labels equal to the
    oracle fit's)."""
    ext = extent(pts)
    ctx = make_ctx(dkm, pts, k, early_stop=early_stop, **opts)
    C_r, lab_r, it_r, sse_r = gpu_run(dkm, ctx, init, max_iter)
    ctx.close()
    ctx2 = make_ctx(dkm, pts, k, early_stop=early_stop, **opts)
    C = np.asarray(init, np.float32).copy()
    flips = 0
    lab = chg = None
    for t in range(it_r):
        lab, sse, chg = gpu_assign(dkm, ctx2, C)
        C64 = C.astype(np.float64)
        lab_o, best, second = oracle.assign(pts, C64)
        flips += check_labels(lab, lab_o, best, second)
        assert abs(sse - best.sum()) <= SSE_RTOL * best.sum(), f"pass {t}: SSE"
        C_next, cnt = gpu_update(dkm, ctx2, None, C)
        C_o, cnt_o = oracle.update(pts, lab, C64)
        assert np.array_equal(cnt, cnt_o), f"pass {t}: cluster sizes"
        err = np.abs(C_next.astype(np.float64) - C_o).max()
        assert err <= CENTROID_TOL * ext, f"pass {t}: centroid error {err:.3g}"
        C = C_next
    ctx2.close()
    assert np.array_equal(C, C_r), "dkm_run's centroids differ from its pass-by-pass replay"
    if it_r > 0:
        assert np.array_equal(lab, lab_r), "dkm_run's labels differ from its replay"
    if early_stop and it_r < max_iter:
        assert chg == 0, "an early-stopped run must end on a pass that changed no label"
    r = oracle.fit(pts, np.asarray(init, np.float64), max_iter, early_stop=bool(early_stop))
    assert abs(sse_r - oracle.sse(pts, lab_r, C_r.astype(np.float64))) <= SSE_RTOL * sse_r
    assert abs(sse_r - r["sse"]) <= SSE_RTOL * r["sse"]
    agree = float(np.mean(lab_r == r["labels"])) if it_r > 0 else 1.0
    if agree == 1.0:
        assert it_r == r["iterations"]
        assert np.abs(C_r.astype(np.float64) - r["centroids"]).max() <= CENTROID_TOL * ext
    return flips, agree
