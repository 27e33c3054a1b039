"""Pins for the FP64 oracle: facts fixed by the paper's definitions and by
mathematics, not by the oracle's own code.

``run_pins(oracle)`` returns a list of failure messages (empty = all pins
hold).  It is used twice: on the real oracle (must be empty) and on copies of
the oracle source with a planted mistake (each must fail at least one pin).

Pins
  worked      hand-worked Lloyd passes (tests/golden/worked_examples.json),
              derived from Eq. 1 / Section II-A / Algorithm 1 "Refine centroid"
  vq          nearest-centroid labels and distances against scipy.cluster.vq
              and scipy.spatial.distance.cdist (library routines)
  optimum     brute force over every labelling of tiny inputs: the converged
              Lloyd SSE equals the global minimum of Eq. 1
  invariants  SSE non-increasing, centroid = numpy mean of its points, fixed
              point at convergence, subset assignment = full assignment
  sklearn     scikit-learn's Lloyd on tie-free data (skipped when absent)
"""
from __future__ import annotations

import itertools
import json
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                      "worked_examples.json")


def _close(a, b, tol=1e-12):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return a.shape == b.shape and np.all(np.abs(a - b) <= tol * np.maximum(1.0, np.abs(b)))


def pin_worked(o) -> list:
    fails = []
    with open(GOLDEN) as f:
        ex = json.load(f)["examples"]
    for e in ex:
        pts = np.asarray(e["points"], dtype=np.float32)
        init = np.asarray(e["init"], dtype=np.float64)
        for p_i, ps in enumerate(e["passes"]):
            r = o.fit(pts, init, max_iter=p_i + 1, early_stop=False)
            want_c = np.asarray(ps["centroids_num"], dtype=np.float64) / ps["centroids_den"]
            want_sse = float(Fraction(ps["sse_num"], ps["sse_den"]))
            if list(r["labels"]) != ps["labels"]:
                fails.append(f"worked {e['name']} pass {p_i+1}: labels {list(r['labels'])} != {ps['labels']}")
            if not _close(r["centroids"], want_c):
                fails.append(f"worked {e['name']} pass {p_i+1}: centroids {r['centroids'].tolist()} != {want_c.tolist()}")
            if not _close(r["sse"], want_sse):
                fails.append(f"worked {e['name']} pass {p_i+1}: sse {r['sse']} != {want_sse}")
            if r["iterations"] != p_i + 1:
                fails.append(f"worked {e['name']}: fixed max_iter={p_i+1} ran {r['iterations']} passes")
        if e.get("iterations_early_stop") is not None:
            r = o.fit(pts, init, max_iter=50, early_stop=True)
            if r["iterations"] != e["iterations_early_stop"]:
                fails.append(f"worked {e['name']}: early stop after {r['iterations']} passes, "
                             f"want {e['iterations_early_stop']}")
    return fails


def pin_vq(o) -> list:
    from scipy.cluster.vq import vq
    from scipy.spatial.distance import cdist
    fails = []
    rng = np.random.default_rng(11)
    for d in (1, 2, 3):
        pts = rng.uniform(-50, 50, size=(1500, d)).astype(np.float32)
        C = rng.uniform(-50, 50, size=(37, d))
        lab, b, s = o.assign(pts, C)
        code, dist = vq(pts.astype(np.float64), C)
        D = cdist(pts.astype(np.float64), C, "sqeuclidean")
        part = np.sort(D, axis=1)
        if not np.array_equal(lab, code.astype(np.int32)):
            fails.append(f"vq d={d}: {int((lab != code).sum())} labels differ from scipy vq")
        if not _close(b, dist.astype(np.float64) ** 2, 1e-9):
            fails.append(f"vq d={d}: best squared distance differs from scipy vq")
        if not _close(s, part[:, 1], 1e-9):
            fails.append(f"vq d={d}: second-best squared distance differs from cdist")
        if not np.array_equal(lab, np.argmin(D, axis=1).astype(np.int32)):
            fails.append(f"vq d={d}: labels differ from cdist argmin")
    return fails


def _brute_min_sse(pts: np.ndarray, k: int) -> float:
    best = np.inf
    n = pts.shape[0]
    P = pts.astype(np.float64)
    for lab in itertools.product(range(k), repeat=n):
        lab = np.asarray(lab)
        if len(set(lab.tolist())) < k:
            continue
        s = 0.0
        for j in range(k):
            m = P[lab == j]
            s += float(((m - m.mean(axis=0)) ** 2).sum())
        best = min(best, s)
    return best


def pin_optimum(o) -> list:
    fails = []
    rng = np.random.default_rng(5)
    # well-separated groups: Lloyd from one seed per group reaches the optimum
    cases = [
        (np.concatenate([rng.normal(0, 1, (4, 2)), rng.normal(30, 1, (4, 2))]), 2, [0, 4]),
        (np.concatenate([rng.normal(0, 1, (3, 3)), rng.normal(25, 1, (3, 3)),
                         rng.normal(-25, 1, (3, 3))]), 3, [0, 3, 6]),
    ]
    for pts, k, seeds in cases:
        pts = pts.astype(np.float32)
        r = o.fit(pts, pts[seeds].astype(np.float64), max_iter=50, early_stop=True)
        want = _brute_min_sse(pts, k)
        if not _close(r["sse"], want, 1e-9):
            fails.append(f"optimum n={pts.shape[0]} k={k}: Lloyd SSE {r['sse']} != exhaustive {want}")
    return fails


def pin_invariants(o) -> list:
    fails = []
    rng = np.random.default_rng(7)
    for d in (2, 3):
        pts = (rng.normal(0, 1, (2500, d)) * 5 + rng.integers(0, 6, (2500, 1)) * 20).astype(np.float32)
        C0 = pts[rng.permutation(pts.shape[0])[:12]].astype(np.float64)
        r = o.fit(pts, C0, max_iter=40, early_stop=True)
        h = r["sse_hist"]
        if np.any(np.diff(h) > 1e-9 * np.abs(h[:-1])):
            fails.append(f"invariants d={d}: SSE increased across iterations {h.tolist()}")
        for j in range(C0.shape[0]):
            m = pts[r["labels"] == j].astype(np.float64)
            if m.shape[0] and not _close(r["centroids"][j], m.mean(axis=0), 1e-10):
                fails.append(f"invariants d={d}: centroid {j} is not the mean of its points")
                break
        lab2, _, _ = o.assign(pts, r["centroids"], want_dist=False)
        if r["iterations"] < 40 and not np.array_equal(lab2, r["labels"]):
            fails.append(f"invariants d={d}: converged labels are not a fixed point")
        idx = rng.choice(pts.shape[0], 300, replace=False)
        ls, bs, ss = o.assign_subset(pts, idx, r["centroids"])
        lf, bf, sf = o.assign(pts, r["centroids"])
        if not (np.array_equal(ls, lf[idx]) and _close(bs, bf[idx]) and _close(ss, sf[idx])):
            fails.append(f"invariants d={d}: subset assignment differs from full assignment")
        # the update is a fixed point for its own labels (means do not move)
        C1, cnt = o.update(pts, r["labels"], r["centroids"])
        if int(cnt.sum()) != pts.shape[0]:
            fails.append(f"invariants d={d}: counts sum {int(cnt.sum())} != n")
    return fails


def pin_sklearn(o) -> list:
    try:
        from sklearn.cluster import KMeans
    except Exception:   # not installed on every machine
        return []
    import warnings
    fails = []
    rng = np.random.default_rng(13)
    for d in (2, 3):
        ctr = rng.uniform(0, 100, (8, d))
        pts = (ctr[rng.integers(0, 8, 4000)] + rng.normal(0, 3, (4000, d))).astype(np.float32)
        C0 = pts[rng.permutation(4000)[:8]].astype(np.float64)
        for m in (1, 3, 60):
            r = o.fit(pts, C0, max_iter=m, early_stop=True)
            if np.any(np.bincount(r["labels"], minlength=8) == 0):
                continue   # sklearn relocates empty clusters; the paper's reading keeps them
            with warnings.catch_warnings():
                warnings.simplefilter("ignore")
                km = KMeans(n_clusters=8, init=C0, n_init=1, max_iter=m, tol=0.0,
                            algorithm="lloyd").fit(pts.astype(np.float64))
            if not _close(r["centroids"], km.cluster_centers_, 1e-8):
                fails.append(f"sklearn d={d} max_iter={m}: centroids differ "
                             f"(max {np.abs(r['centroids'] - km.cluster_centers_).max():.3g})")
    return fails


ALL_PINS = [pin_worked, pin_vq, pin_optimum, pin_invariants, pin_sklearn]


def run_pins(o) -> list:
    fails = []
    for p in ALL_PINS:
        try:
            fails += p(o)
        except Exception as exc:   # a crash in a mutant counts as a caught mistake
            fails.append(f"{p.__name__}: raised {type(exc).__name__}: {exc}")
    return fails
