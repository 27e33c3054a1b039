"""Pins for the FP64 soft / hard k-means loss oracle (oracle/soft_kmeans.py).

  fd          central finite differences of the forward (FP64) against the
              analytic backward, on tiny random clouds, T = 0, 1, 3
  lloyd       tau -> 0: the soft iterations become Lloyd's algorithm, so the
              centroids after T steps equal the (separately pinned) C
              oracle's Lloyd centroids and the loss equals the hard SSE
  uniform     tau -> infinity: every weight is 1/k, so c^1 = mean(P) for all
              centroids and the loss is sum_i ||p_i - mean||^2
  shift       translating points and centroids together changes nothing, so
              the gradients of points and centroids sum to zero
  hard        the hard-SSE gradient against finite differences away from ties
"""
from __future__ import annotations

import numpy as np


def _fd_grad(f, X, h):
    g = np.zeros_like(X)
    it = np.nditer(X, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        Xp = X.copy()
        Xm = X.copy()
        Xp[idx] += h
        Xm[idx] -= h
        g[idx] = (f(Xp) - f(Xm)) / (2 * h)
    return g


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def pin_fd(sk) -> list:
    fails = []
    rng = np.random.default_rng(21)
    for T in (0, 1, 3):
        P = rng.normal(0, 1, (9, 3))
        C0 = P[rng.permutation(9)[:3]] + rng.normal(0, 0.1, (3, 3))
        tau = 0.7
        _, gP, gC = sk.soft_backward(P, C0, tau, T)
        fP = _fd_grad(lambda X: sk.soft_forward(X, C0, tau, T)[0], P, 1e-5)
        fC = _fd_grad(lambda X: sk.soft_forward(P, X, tau, T)[0], C0, 1e-5)
        if _rel(gP, fP) > 1e-6:
            fails.append(f"fd T={T}: dL/dP off by {_rel(gP, fP):.3g}")
        if _rel(gC, fC) > 1e-6:
            fails.append(f"fd T={T}: dL/dC0 off by {_rel(gC, fC):.3g}")
    return fails


def pin_lloyd(sk, oracle) -> list:
    fails = []
    rng = np.random.default_rng(22)
    ctr = np.array([[0, 0, 0], [10, 0, 0], [0, 10, 0], [0, 0, 10]], float)
    P = (ctr[rng.integers(0, 4, 400)] + rng.normal(0, 1, (400, 3))).astype(np.float32)
    C0 = P[rng.permutation(400)[:4]].astype(np.float64)
    for T in (1, 2, 5):
        loss, Cs = sk.soft_forward(P.astype(np.float64), C0, 1e-4, T)
        r = oracle.fit(P, C0, T, early_stop=False)
        if np.abs(Cs[T] - r["centroids"]).max() > 1e-9 * 10:
            fails.append(f"lloyd T={T}: soft centroids differ from Lloyd "
                         f"({np.abs(Cs[T] - r['centroids']).max():.3g})")
        hard, _, _, _ = sk.hard_sse_grad(P, Cs[T])
        if abs(loss - hard) > 1e-9 * hard:
            fails.append(f"lloyd T={T}: soft loss {loss} != hard SSE {hard}")
    return fails


def pin_uniform(sk) -> list:
    fails = []
    rng = np.random.default_rng(23)
    P = rng.normal(0, 1, (50, 3))
    C0 = rng.normal(0, 1, (5, 3))
    loss, Cs = sk.soft_forward(P, C0, 1e12, 1)
    mean = P.mean(axis=0)
    if np.abs(Cs[1] - mean[None, :]).max() > 1e-9:
        fails.append("uniform: c^1 is not the mean of all points")
    want = float(((P - mean) ** 2).sum())
    if abs(loss - want) > 1e-9 * want:
        fails.append(f"uniform: loss {loss} != {want}")
    return fails


def pin_shift(sk) -> list:
    fails = []
    rng = np.random.default_rng(24)
    P = rng.normal(0, 1, (40, 3))
    C0 = P[:4] + 0.05
    for T in (0, 2):
        l0, gP, gC = sk.soft_backward(P, C0, 0.5, T)
        v = np.array([3.0, -2.0, 7.0])
        l1, _, _ = sk.soft_backward(P + v, C0 + v, 0.5, T)
        if abs(l0 - l1) > 1e-9 * abs(l0):
            fails.append(f"shift T={T}: loss changed under translation")
        tot = gP.sum(axis=0) + gC.sum(axis=0)
        if np.abs(tot).max() > 1e-9 * np.abs(gP).sum():
            fails.append(f"shift T={T}: gradients do not sum to zero ({tot})")
    return fails


def pin_hard(sk, oracle) -> list:
    fails = []
    rng = np.random.default_rng(25)
    P = rng.normal(0, 1, (30, 3)).astype(np.float32).astype(np.float64)
    C = rng.normal(0, 1, (4, 3))
    L, a, gP, gC = sk.hard_sse_grad(P, C)
    lab, best, second = oracle.assign(P.astype(np.float32), C)
    if not np.array_equal(a, lab):
        fails.append("hard: labels differ from the C oracle")
    if abs(L - best.sum()) > 1e-12 * L:
        fails.append("hard: loss differs from the C oracle")
    f = lambda X: sk.hard_sse_grad(X, C)[0]
    g = lambda X: sk.hard_sse_grad(P, X)[0]
    if _rel(gP, _fd_grad(f, P, 1e-6)) > 1e-6:
        fails.append("hard: dL/dP off")
    if _rel(gC, _fd_grad(g, C, 1e-6)) > 1e-6:
        fails.append("hard: dL/dC off")
    return fails


def run_soft_pins(sk, oracle) -> list:
    fails = []
    for p in (pin_fd, pin_uniform, pin_shift):
        try:
            fails += p(sk)
        except Exception as exc:
            fails.append(f"{p.__name__}: raised {type(exc).__name__}: {exc}")
    for p in (pin_lloyd, pin_hard):
        try:
            fails += p(sk, oracle)
        except Exception as exc:
            fails.append(f"{p.__name__}: raised {type(exc).__name__}: {exc}")
    return fails
