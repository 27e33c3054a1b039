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
