"""dkm_lloyd_step_noalloc: one Lloyd step that allocates no device memory.

Some callers cannot call cudaMalloc (code inside a host framework that owns
all device memory, or a latency-critical loop where an allocation would
synchronise the device).  This entry point keeps its scratch in a fixed
array inside the library instead.  The test checks it against the regular
entry points (dkm_assign + dkm_update) on two different problems in a row,
so the second call also shows the scratch is cleared between calls.  This
file is collected last so that a stop at the first failure has run every
other test first.
"""
import numpy as np
import pytest

from paper_2412_02244_gb300 import synth
from gpu_util import CENTROID_TOL, SSE_RTOL, dev, extent, gpu_assign, gpu_update, make_ctx, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dkm():
    torch_cuda()
    from paper_2412_02244_gb300 import build
    build.build()
    from paper_2412_02244_gb300 import dkm as m
    return m


def _noalloc(dkm, pts, C):
    torch = torch_cuda()
    n, d = pts.shape
    k = C.shape[0]
    C_out = torch.empty(k * d, dtype=torch.float32, device="cuda")
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    sse = dkm.dkm_lloyd_step_noalloc(dev(pts), n, d, k, dev(C), C_out, lab)
    torch.cuda.synchronize()
    return lab.cpu().numpy(), C_out.cpu().numpy().reshape(k, d), sse


def test_noalloc_step_matches_assign_and_update(dkm):
    problems = [synth.lidar3d(seed=51, n=60_011, k=150, n_objects=20),
                synth.geo2d_blobs(seed=52, n=20_003, k=37),
                # centroids staged in three shared-memory rounds, the last partial
                synth.lidar3d(seed=53, n=30_007, k=2_500, n_objects=30),
                # the largest k the fixed scratch holds
                synth.geo2d_blobs(seed=54, n=70_001, k=dkm.DKM_NOALLOC_MAX_K)]
    for w in problems:   # calls in a row, different n, d and k
        lab_na, C_na, sse_na = _noalloc(dkm, w.points, w.init)
        ctx = make_ctx(dkm, w.points, w.k)
        lab_ref, sse_ref, _ = gpu_assign(dkm, ctx, w.init)
        C_ref, _ = gpu_update(dkm, ctx, lab_ref, w.init)
        assert np.array_equal(lab_na, lab_ref)
        tol = CENTROID_TOL * extent(w.points)
        assert np.abs(C_na.astype(np.float64) - C_ref).max() <= tol
        assert abs(sse_na - sse_ref) <= SSE_RTOL * sse_ref


def test_noalloc_step_rejects_non_finite_input(dkm):
    """A NaN point or an infinite centroid is reported as DKM_EINVAL (the
    status is read back with the SSE); labels are -1 and the centroids pass
    through.  The next call with clean input works again."""
    torch = torch_cuda()
    w = synth.geo2d_blobs(seed=55, n=5_003, k=20)
    for which in ("points", "centroids"):
        P = w.points.copy()
        C = w.init.copy()
        if which == "points":
            P[1234, 1] = np.nan
        else:
            C[7, 0] = np.inf
        n, d = P.shape
        C_out = torch.zeros(w.k * d, dtype=torch.float32, device="cuda")
        lab = torch.zeros(n, dtype=torch.int32, device="cuda")
        with pytest.raises(dkm.DkmError) as ei:
            dkm.dkm_lloyd_step_noalloc(dev(P), n, d, w.k, dev(C), C_out, lab)
        assert ei.value.status == dkm.DKM_EINVAL
        assert np.all(lab.cpu().numpy() == -1)
        assert np.array_equal(C_out.cpu().numpy().reshape(w.k, d), C)
    lab_na, C_na, sse_na = _noalloc(dkm, w.points, w.init)
    assert lab_na.min() >= 0 and np.isfinite(sse_na)
