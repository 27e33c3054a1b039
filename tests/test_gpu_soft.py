"""Differentiable k-means losses on the GPU against the FP64 oracle
(oracle/soft_kmeans.py): loss, per-step centroids, analytic gradients,
FP64 central finite differences, the autograd wrapper, a 64 x 16,384-point
batch shaped like the differentiable workload, and the hard SSE."""
import numpy as np
import pytest

import oracle.soft_kmeans as sk
from paper_2412_02244_gb300 import synth
from gpu_util import check_labels, torch_cuda

pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-4


@pytest.fixture(scope="module")
def dkm():
    torch_cuda()
    from paper_2412_02244_gb300 import build
    build.build()
    from paper_2412_02244_gb300 import dkm as m
    return m


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _batch(clouds, k, seed):
    rng = np.random.default_rng(seed)
    pts = [c.astype(np.float32) for c in clouds]
    init = np.stack([p[rng.permutation(p.shape[0])[:k]] for p in pts]).astype(np.float32)
    off = np.zeros(len(pts) + 1, np.int64)
    off[1:] = np.cumsum([p.shape[0] for p in pts])
    tau = np.array([sk.temperature(p) for p in pts], np.float32)
    return pts, np.concatenate(pts), init, off, tau


def _gpu_soft(dkm, P, init, off, tau, T, dloss=None):
    torch = torch_cuda()
    B, k, d = init.shape
    Pt = torch.from_numpy(P).cuda()
    It = torch.from_numpy(init).cuda()
    ck = torch.empty((T + 1, B, k, d), dtype=torch.float32, device="cuda")
    loss = torch.empty(B, dtype=torch.float64, device="cuda")
    dkm.dkm_soft_forward(Pt, off, B, d, k, It, T, tau, ck, loss)
    dl = np.ones(B) if dloss is None else np.asarray(dloss, np.float64)
    gp = torch.empty_like(Pt)
    gi = torch.empty_like(It)
    dkm.dkm_soft_backward(Pt, off, B, d, k, ck, T, tau, dl, gp, gi)
    return loss.cpu().numpy(), ck.cpu().numpy(), gp.cpu().numpy(), gi.cpu().numpy()


@pytest.mark.parametrize("d", [2, 3])
def test_soft_forward_backward_vs_oracle(dkm, d):
    rng = np.random.default_rng(31 + d)
    clouds = [synth.gaussian_mixture_3d(n, 6, rng)[:, :d] for n in (700, 2048 + 13, 1500)]
    pts, P, init, off, tau = _batch(clouds, 12, 33)
    T = 3
    dl = np.array([1.0, -0.5, 2.0])
    loss, ck, gp, gi = _gpu_soft(dkm, P, init, off, tau, T, dl)
    for b, Pb in enumerate(pts):
        L, Cs = sk.soft_forward(Pb.astype(np.float64), init[b].astype(np.float64), float(tau[b]), T)
        ext = float(np.max(Pb.max(0) - Pb.min(0)))
        assert abs(loss[b] - L) <= 1e-5 * L
        for t in range(T + 1):
            assert np.abs(ck[t, b] - Cs[t]).max() <= 1e-5 * ext
        _, gP, gC = sk.soft_backward(Pb.astype(np.float64), init[b].astype(np.float64),
                                     float(tau[b]), T)
        assert _rel(gp[off[b]:off[b + 1]], dl[b] * gP) <= GRAD_RTOL
        assert _rel(gi[b], dl[b] * gC) <= GRAD_RTOL


def test_soft_backward_vs_finite_differences(dkm):
    """GPU gradient against FP64 central differences of the oracle's loss."""
    rng = np.random.default_rng(41)
    Pb = synth.gaussian_mixture_3d(60, 4, rng)
    pts, P, init, off, tau = _batch([Pb], 4, 42)
    T = 2
    _, _, gp, gi = _gpu_soft(dkm, P, init, off, tau, T)
    P64, C64, t = P.astype(np.float64), init[0].astype(np.float64), float(tau[0])
    h = 1e-6

    def fd(f, X):
        g = np.zeros_like(X)
        for idx in np.ndindex(*X.shape):
            Xp, Xm = X.copy(), X.copy()
            Xp[idx] += h
            Xm[idx] -= h
            g[idx] = (f(Xp) - f(Xm)) / (2 * h)
        return g
    fP = fd(lambda X: sk.soft_forward(X, C64, t, T)[0], P64)
    fC = fd(lambda X: sk.soft_forward(P64, X, t, T)[0], C64)
    assert _rel(gp, fP) <= GRAD_RTOL
    assert _rel(gi[0], fC) <= GRAD_RTOL


def test_soft_autograd_function(dkm):
    torch = torch_cuda()
    from paper_2412_02244_gb300.autograd import SoftKMeansLoss, temperature
    rng = np.random.default_rng(51)
    clouds = [synth.gaussian_mixture_3d(n, 5, rng) for n in (900, 1200)]
    pts, P, init, off, tau = _batch(clouds, 8, 52)
    Pt = torch.from_numpy(P).cuda().requires_grad_(True)
    It = torch.from_numpy(init).cuda().requires_grad_(True)
    offt = torch.from_numpy(off)
    taut = temperature(Pt.detach(), offt)
    assert np.allclose(taut.numpy(), tau, rtol=1e-6)
    w = torch.tensor([0.3, 1.7], dtype=torch.float64, device="cuda")
    loss = SoftKMeansLoss.apply(Pt, It, offt, taut, 4)
    (loss * w).sum().backward()
    for b, Pb in enumerate(pts):
        _, gP, gC = sk.soft_backward(Pb.astype(np.float64), init[b].astype(np.float64),
                                     float(tau[b]), 4)
        assert _rel(Pt.grad[off[b]:off[b + 1]].cpu().numpy(), float(w[b]) * gP) <= GRAD_RTOL
        assert _rel(It.grad[b].cpu().numpy(), float(w[b]) * gC) <= GRAD_RTOL


def test_soft_differentiable_workload_shape(dkm):
    """Clouds of 16,384 points (32-blob mixtures), k = 256, T = 10, the
    temperature at 1% of the squared bbox diagonal; two clouds of the
    64-cloud batch are checked against the oracle's analytic gradient."""
    ws = synth.soft3d(seed=5, n_clouds=64)
    clouds = [w.points for w in ws]
    init = np.stack([w.init for w in ws])
    off = np.zeros(65, np.int64)
    off[1:] = np.cumsum([c.shape[0] for c in clouds])
    tau = np.array([sk.temperature(c) for c in clouds], np.float32)
    P = np.concatenate(clouds)
    loss, ck, gp, gi = _gpu_soft(dkm, P, init, off, tau, 10)
    assert np.all(np.isfinite(loss)) and np.all(np.isfinite(gp)) and np.all(np.isfinite(gi))
    for b in (0, 37):
        Pb = clouds[b].astype(np.float64)
        L, gP, gC = sk.soft_backward(Pb, init[b].astype(np.float64), float(tau[b]), 10)
        assert abs(loss[b] - L) <= 1e-5 * L
        assert _rel(gp[off[b]:off[b + 1]], gP) <= GRAD_RTOL
        assert _rel(gi[b], gC) <= GRAD_RTOL


def test_hard_sse_vs_oracle(dkm, oracle):
    torch = torch_cuda()
    from paper_2412_02244_gb300.autograd import HardSSELoss
    rng = np.random.default_rng(61)
    clouds = [synth.gaussian_mixture_3d(n, 5, rng) for n in (1000, 3000 + 7)]
    pts, P, init, off, tau = _batch(clouds, 9, 62)
    Pt = torch.from_numpy(P).cuda().requires_grad_(True)
    Ct = torch.from_numpy(init).cuda().requires_grad_(True)
    loss = HardSSELoss.apply(Pt, Ct, torch.from_numpy(off))
    w = torch.tensor([2.0, 0.5], dtype=torch.float64, device="cuda")
    (loss * w).sum().backward()
    lab = torch.empty(P.shape[0], dtype=torch.int32, device="cuda")
    dkm.dkm_hard_sse(Pt.detach(), off, 2, 3, 9, Ct.detach(), lab)
    for b, Pb in enumerate(pts):
        L, a, gP, gC = sk.hard_sse_grad(Pb.astype(np.float64), init[b].astype(np.float64))
        lo, best, second = oracle.assign(Pb, init[b].astype(np.float64))
        assert np.array_equal(lab.cpu().numpy()[off[b]:off[b + 1]], lo)
        assert abs(float(loss.detach()[b]) - L) <= 1e-5 * L
        assert _rel(Pt.grad[off[b]:off[b + 1]].cpu().numpy(), float(w[b]) * gP) <= GRAD_RTOL
        assert _rel(Ct.grad[b].cpu().numpy(), float(w[b]) * gC) <= GRAD_RTOL


def test_soft_errors(dkm):
    torch = torch_cuda()
    P = torch.zeros((10, 3), device="cuda")
    ck = torch.empty((2, 2, 2, 3), device="cuda")
    loss = torch.empty(2, dtype=torch.float64, device="cuda")
    init = torch.zeros((2, 2, 3), device="cuda")
    with pytest.raises(dkm.DkmError) as e:     # the second cloud is empty
        dkm.dkm_soft_forward(P, np.array([0, 10, 10], np.int64), 2, 3, 2, init, 1,
                             np.ones(2, np.float32), ck, loss)
    assert e.value.status == dkm.DKM_EINVAL


def test_soft_backward_with_forward_statistics_is_identical(dkm):
    """The backward given the forward's per-step statistics returns exactly
    the gradient it computes without them."""
    torch = torch_cuda()
    rng = np.random.default_rng(81)
    clouds = [synth.gaussian_mixture_3d(n, 6, rng) for n in (900, 2500 + 3)]
    pts, P, init, off, tau = _batch(clouds, 16, 82)
    B, k, d = init.shape
    T = 4
    Pt = torch.from_numpy(P).cuda()
    It = torch.from_numpy(init).cuda()
    ck = torch.empty((T + 1, B, k, d), dtype=torch.float32, device="cuda")
    loss = torch.empty(B, dtype=torch.float64, device="cuda")
    st = torch.empty((T, 2, P.shape[0]), dtype=torch.float32, device="cuda")
    nm = torch.empty((T, B, k), dtype=torch.float32, device="cuda")
    dkm.dkm_soft_forward(Pt, off, B, d, k, It, T, tau, ck, loss, stats=st, norms=nm)
    dl = np.array([0.7, -1.3])
    out = []
    for kw in (dict(), dict(stats=st, norms=nm)):
        gp = torch.empty_like(Pt)
        gi = torch.empty_like(It)
        dkm.dkm_soft_backward(Pt, off, B, d, k, ck, T, tau, dl, gp, gi, **kw)
        out.append((gp.cpu().numpy(), gi.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
    assert np.all(nm.cpu().numpy() > 0)


def test_soft_gradient_passes_through_a_centroid_with_no_weight(dkm):
    """A centroid whose weights all underflow to zero in step 0 keeps its
    position (c^1_B = c^0_B), so dL/dc^0_B must equal dL/dc^1_B.  Built so
    that centroid B has no weight in step 0 but a large one in step 1 (A
    moves away from the small cluster next to B); the GPU's T = 2 gradient
    of c^0_B is checked against the FP64 oracle's T = 1 gradient of c^1_B
    taken from the GPU's own checkpoint c^1."""
    torch = torch_cuda()
    rng = np.random.default_rng(91)
    big = rng.normal(0.0, 0.05, size=(90, 3))
    small = rng.normal(0.0, 0.05, size=(10, 3)) + np.array([10.0, 0.0, 0.0])
    P = np.concatenate([big, small]).astype(np.float32)
    init = np.array([[[10.0, 0.0, 0.0], [19.03, 0.0, 0.0]]], np.float32)   # A, B
    off = np.array([0, P.shape[0]], np.int64)
    tau = np.array([0.5], np.float32)
    B, k, d, T = 1, 2, 3, 2
    Pt = torch.from_numpy(P).cuda()
    It = torch.from_numpy(init).cuda()
    ck = torch.empty((T + 1, B, k, d), dtype=torch.float32, device="cuda")
    loss = torch.empty(B, dtype=torch.float64, device="cuda")
    st = torch.empty((T, 2, P.shape[0]), dtype=torch.float32, device="cuda")
    nm = torch.empty((T, B, k), dtype=torch.float32, device="cuda")
    dkm.dkm_soft_forward(Pt, off, B, d, k, It, T, tau, ck, loss, stats=st, norms=nm)
    nm = nm.cpu().numpy()
    ck = ck.cpu().numpy()
    assert nm[0, 0, 1] == 0.0 and nm[1, 0, 1] > 0.5   # no weight in step 0, some in step 1
    assert np.array_equal(ck[1, 0, 1], init[0, 1])     # B kept its position
    for kw in (dict(), dict(stats=st, norms=torch.from_numpy(nm).cuda())):
        gp = torch.empty_like(Pt)
        gi = torch.empty_like(It)
        dkm.dkm_soft_backward(Pt, off, B, d, k, torch.from_numpy(ck).cuda(), T, tau,
                              np.ones(1), gp, gi, **kw)
        _, _, gC1 = sk.soft_backward(P.astype(np.float64), ck[1, 0].astype(np.float64),
                                     float(tau[0]), 1)
        g = gi.cpu().numpy()[0, 1]
        assert np.linalg.norm(gC1[1]) > 1e-2
        assert _rel(g, gC1[1]) <= GRAD_RTOL


def test_hard_sse_backward_scales_and_checks_labels(dkm):
    """dkm_hard_sse_backward: gradients scale with the upstream gradient of
    each cloud, and a label outside [0, k) is an error."""
    torch = torch_cuda()
    rng = np.random.default_rng(71)
    clouds = [synth.gaussian_mixture_3d(n, 4, rng) for n in (700, 1300)]
    pts, P, init, off, tau = _batch(clouds, 6, 72)
    B, k, d = init.shape
    Pt = torch.from_numpy(P).cuda()
    Ct = torch.from_numpy(init).cuda()
    lab = torch.empty(P.shape[0], dtype=torch.int32, device="cuda")
    loss = torch.empty(B, dtype=torch.float64, device="cuda")
    dkm.dkm_hard_sse(Pt, off, B, d, k, Ct, lab, loss)
    dl = np.array([-0.25, 3.0])
    gp = torch.empty_like(Pt)
    gc = torch.empty_like(Ct)
    dkm.dkm_hard_sse_backward(Pt, off, B, d, k, Ct, lab, dl, gp, gc)
    for b, Pb in enumerate(pts):
        _, _, gP, gC = sk.hard_sse_grad(Pb.astype(np.float64), init[b].astype(np.float64))
        assert _rel(gp.cpu().numpy()[off[b]:off[b + 1]], dl[b] * gP) <= GRAD_RTOL
        assert _rel(gc.cpu().numpy()[b], dl[b] * gC) <= GRAD_RTOL
    bad = lab.clone()
    bad[5] = k
    with pytest.raises(dkm.DkmError) as e:
        dkm.dkm_hard_sse_backward(Pt, off, B, d, k, Ct, bad, dl, gp, gc)
    assert e.value.status == dkm.DKM_EINVAL


@pytest.mark.parametrize("d", [2, 3])
def test_soft_and_hard_with_odd_k_above_one_warp(dkm, oracle, d):
    """k = 101: the column passes give each thread two centroids (j and j +
    64 here), so both packed lanes are live for some threads and only the
    first for others; clouds of 777 and 1,537 points end inside a row-pass
    CTA (512 points) and a column split (512 points).  Soft forward and
    backward and the hard SSE with both gradients against the oracle."""
    torch = torch_cuda()
    rng = np.random.default_rng(71 + d)
    clouds = [synth.gaussian_mixture_3d(n, 7, rng)[:, :d] for n in (777, 1537)]
    k = 101
    pts, P, init, off, tau = _batch(clouds, k, 72)
    T = 2
    dl = np.array([1.5, -0.75])
    loss, ck, gp, gi = _gpu_soft(dkm, P, init, off, tau, T, dl)
    for b, Pb in enumerate(pts):
        P64, C64 = Pb.astype(np.float64), init[b].astype(np.float64)
        L, Cs = sk.soft_forward(P64, C64, float(tau[b]), T)
        ext = float(np.max(Pb.max(0) - Pb.min(0)))
        assert abs(loss[b] - L) <= 1e-5 * L
        for t in range(T + 1):
            assert np.abs(ck[t, b] - Cs[t]).max() <= 1e-5 * ext
        _, gP, gC = sk.soft_backward(P64, C64, float(tau[b]), T)
        assert _rel(gp[off[b]:off[b + 1]], dl[b] * gP) <= GRAD_RTOL
        assert _rel(gi[b], dl[b] * gC) <= GRAD_RTOL
    Pt = torch.from_numpy(P).cuda()
    Ct = torch.from_numpy(init).cuda()
    hl = torch.empty(2, dtype=torch.float64, device="cuda")
    lab = torch.empty(P.shape[0], dtype=torch.int32, device="cuda")
    hp = torch.empty_like(Pt)
    hc = torch.empty_like(Ct)
    dkm.dkm_hard_sse(Pt, off, 2, d, k, Ct, lab, hl, hp, hc)
    for b, Pb in enumerate(pts):
        L, a, gP, gC = sk.hard_sse_grad(Pb.astype(np.float64), init[b].astype(np.float64))
        lo, best, second = oracle.assign(Pb, init[b].astype(np.float64))
        check_labels(lab.cpu().numpy()[off[b]:off[b + 1]], lo, best, second)   # near-ties only
        assert abs(float(hl[b]) - L) <= 1e-5 * L
        assert _rel(hp[off[b]:off[b + 1]].cpu().numpy(), gP) <= GRAD_RTOL
        assert _rel(hc[b].cpu().numpy(), gC) <= GRAD_RTOL
