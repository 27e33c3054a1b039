"""FP64 numpy oracle for the differentiable k-means losses.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper (Dask-means, arXiv 2412.02244) optimises the k-means objective of
Eq. 1 with Lloyd's algorithm; it has no differentiable form.  The
differentiable extension defines two losses of a point cloud P (n x d) and
initial centroids C0 (k x d):

  hard SSE   L_h(P, C) = sum_i min_j ||p_i - c_j||^2            (Eq. 1)
             dL/dp_i = 2 (p_i - c_a(i)),  dL/dc_j = -2 sum_{a(i)=j} (p_i - c_j)
             with a(i) the nearest centroid (lowest index on ties).

  soft k-means, T unrolled iterations at a fixed temperature tau:
             D^t_ij = ||p_i - c^t_j||^2
             w^t_ij = exp(-D^t_ij / tau) / sum_l exp(-D^t_il / tau)
             c^{t+1}_j = sum_i w^t_ij p_i / sum_i w^t_ij          (t < T)
             L_s = sum_i sum_j w^T_ij D^T_ij

The backward below is reverse-mode differentiation written out step by step
(no autodiff library): the loss stage, then each update in reverse order,
recomputing w^t from the stored centroids c^t.  Everything is FP64.
"""
from __future__ import annotations

import numpy as np


def sq_dists(P: np.ndarray, C: np.ndarray) -> np.ndarray:
    """D_ij = ||p_i - c_j||^2 (n x k)."""
    diff = P[:, None, :] - C[None, :, :]
    return (diff * diff).sum(axis=2)


def soft_weights(D: np.ndarray, tau: float) -> np.ndarray:
    """Row softmax of -D / tau, shifted by the row minimum for stability."""
    Z = -(D - D.min(axis=1, keepdims=True)) / tau
    E = np.exp(Z)
    return E / E.sum(axis=1, keepdims=True)


def soft_forward(P, C0, tau: float, T: int):
    """(L_s, [c^0, ..., c^T])."""
    P = np.asarray(P, dtype=np.float64)
    C = np.asarray(C0, dtype=np.float64)
    Cs = [C]
    for _ in range(T):
        W = soft_weights(sq_dists(P, C), tau)
        C = (W.T @ P) / W.sum(axis=0)[:, None]
        Cs.append(C)
    D = sq_dists(P, C)
    W = soft_weights(D, tau)
    return float((W * D).sum()), Cs


def soft_backward(P, C0, tau: float, T: int):
    """(L_s, dL/dP, dL/dC0) with tau held constant."""
    P = np.asarray(P, dtype=np.float64)
    loss, Cs = soft_forward(P, C0, tau, T)
    # loss stage: L = sum_ij w_ij D_ij with w = softmax(-D / tau)
    C = Cs[T]
    D = sq_dists(P, C)
    W = soft_weights(D, tau)
    E = (W * D).sum(axis=1, keepdims=True)
    dD = W * (1.0 - (D - E) / tau)                       # dL/dD_ij
    diff = P[:, None, :] - C[None, :, :]
    gP = 2.0 * (dD[:, :, None] * diff).sum(axis=1)
    gC = -2.0 * (dD[:, :, None] * diff).sum(axis=0)      # dL/dc^T
    # updates, last first: c^{t+1} = (W^t)^T P / N^t with N^t_j = sum_i w^t_ij
    for t in reversed(range(T)):
        Ct, Cn = Cs[t], Cs[t + 1]
        D = sq_dists(P, Ct)
        W = soft_weights(D, tau)
        N = W.sum(axis=0)
        # dL/dw_ij through c^{t+1}_j:  g_ij = gC_j . (p_i - c^{t+1}_j) / N_j
        g = np.einsum("ijd,jd->ij", P[:, None, :] - Cn[None, :, :], gC) / N[None, :]
        # dL/dp_i directly through the weighted sums: sum_j w_ij gC_j / N_j
        gP = gP + (W / N[None, :]) @ gC
        # through the row softmax: dL/dD_ij = -(1/tau) w_ij (g_ij - sum_l w_il g_il)
        rho = (W * g).sum(axis=1, keepdims=True)
        dD = -(W * (g - rho)) / tau
        diff = P[:, None, :] - Ct[None, :, :]
        gP = gP + 2.0 * (dD[:, :, None] * diff).sum(axis=1)
        gC = -2.0 * (dD[:, :, None] * diff).sum(axis=0)  # dL/dc^t
    return loss, gP, gC


def hard_sse_grad(P, C):
    """(L_h, labels, dL/dP, dL/dC) by brute force (lowest index on ties)."""
    P = np.asarray(P, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    D = sq_dists(P, C)
    a = np.argmin(D, axis=1)
    r = P - C[a]
    gP = 2.0 * r
    gC = np.zeros_like(C)
    np.add.at(gC, a, -2.0 * r)
    return float(D[np.arange(P.shape[0]), a].sum()), a.astype(np.int32), gP, gC


def temperature(P, frac: float = 0.01) -> float:
    """tau = frac x squared bounding-box diagonal of the cloud (a constant of
    the loss, computed once from the unperturbed points)."""
    P = np.asarray(P, dtype=np.float64)
    ext = P.max(axis=0) - P.min(axis=0)
    return float(frac * (ext * ext).sum())
