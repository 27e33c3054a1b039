"""FP64 CPU oracle for Lloyd's k-means (Dask-means, arXiv 2412.02244).

TEST INFRASTRUCTURE ONLY.  This package is the checker the CUDA path is
compared against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the product package: it neither imports
``paper_2412_02244_gb300`` nor is imported by it.

Contents
  * ``dkm_oracle.c`` -- brute-force Lloyd in FP64 (Eq. 1, Section II-A,
    Algorithm 1 "Refine centroid"), compiled with gcc into
    ``oracle/_build/libdkm_oracle.so``.
  * ``soft_kmeans.py`` -- FP64 numpy forward and analytic backward of the
    hard-SSE and soft k-means losses (the differentiable extension).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dkm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libdkm_oracle.so")


def build(src: str = _SRC, out: str = _LIB_PATH, openmp: bool = True) -> str:
    """Compile the C oracle with gcc (host code only, portable: no -march)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", out + ".tmp", "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _stale(lib: str, src: str) -> bool:
    return (not os.path.exists(lib)) or os.path.getmtime(lib) < os.path.getmtime(src)


_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


class Oracle:
    """ctypes wrapper around one compiled copy of ``dkm_oracle.c``."""

    def __init__(self, path: Optional[str] = None):
        if path is None:
            if _stale(_LIB_PATH, _SRC):
                build()
            path = _LIB_PATH
        self.path = path
        lib = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        lib.oracle_assign.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, _f64p, ctypes.c_int,
                                      _i32p, vp, vp]
        lib.oracle_assign.restype = None
        lib.oracle_assign_subset.argtypes = [_f32p, ctypes.c_int, _i64p, ctypes.c_int64, _f64p,
                                             ctypes.c_int, _i32p, vp, vp]
        lib.oracle_assign_subset.restype = None
        lib.oracle_update.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, _i32p, ctypes.c_int,
                                      _f64p, _f64p, vp]
        lib.oracle_update.restype = ctypes.c_int
        lib.oracle_sse.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, _i32p, _f64p]
        lib.oracle_sse.restype = ctypes.c_double
        lib.oracle_fit.argtypes = [_f32p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, _f64p,
                                   ctypes.c_int, ctypes.c_int, _f64p, _i32p,
                                   ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                   vp, vp]
        lib.oracle_fit.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        self.lib = lib

    # -- helpers -----------------------------------------------------------
    @staticmethod
    def _pts(points) -> np.ndarray:
        p = np.ascontiguousarray(points, dtype=np.float32)
        if p.ndim != 2:
            raise ValueError("points must be (n, d)")
        return p

    @staticmethod
    def _cent(C, d: int) -> np.ndarray:
        c = np.ascontiguousarray(np.asarray(C, dtype=np.float64).reshape(-1, d))
        return c

    @staticmethod
    def _ptr(a: Optional[np.ndarray]):
        return None if a is None else a.ctypes.data_as(ctypes.c_void_p)

    def num_threads(self) -> int:
        return int(self.lib.oracle_num_threads())

    # -- API ---------------------------------------------------------------
    def assign(self, points, C, want_dist: bool = True):
        """labels, best d^2, second-best d^2 (FP64) for every point."""
        p = self._pts(points)
        n, d = p.shape
        c = self._cent(C, d)
        k = c.shape[0]
        lab = np.empty(n, dtype=np.int32)
        b = np.empty(n, dtype=np.float64) if want_dist else None
        s = np.empty(n, dtype=np.float64) if want_dist else None
        self.lib.oracle_assign(p, n, d, c, k, lab, self._ptr(b), self._ptr(s))
        return lab, b, s

    def assign_subset(self, points, idx, C):
        p = self._pts(points)
        d = p.shape[1]
        ix = np.ascontiguousarray(idx, dtype=np.int64)
        if ix.size and (ix.min() < 0 or ix.max() >= p.shape[0]):
            raise IndexError("subset index out of range")
        c = self._cent(C, d)
        k = c.shape[0]
        m = ix.shape[0]
        lab = np.empty(m, dtype=np.int32)
        b = np.empty(m, dtype=np.float64)
        s = np.empty(m, dtype=np.float64)
        self.lib.oracle_assign_subset(p, d, ix, m, c, k, lab, self._ptr(b), self._ptr(s))
        return lab, b, s

    def update(self, points, labels, C_prev):
        """(C_new FP64, counts int64) -- cluster means, empty keeps C_prev."""
        p = self._pts(points)
        n, d = p.shape
        c = self._cent(C_prev, d)
        k = c.shape[0]
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        if lab.shape != (n,):
            raise ValueError("labels must be (n,)")
        out = np.empty_like(c)
        cnt = np.empty(k, dtype=np.int64)
        rc = self.lib.oracle_update(p, n, d, lab, k, c, out, self._ptr(cnt))
        if rc != 0:
            raise ValueError(f"oracle_update failed ({rc}): label out of range")
        return out, cnt

    def sse(self, points, labels, C) -> float:
        p = self._pts(points)
        n, d = p.shape
        c = self._cent(C, d)
        lab = np.ascontiguousarray(labels, dtype=np.int32)
        if lab.size and (lab.min() < 0 or lab.max() >= c.shape[0]):
            raise ValueError("label out of range")
        return float(self.lib.oracle_sse(p, n, d, lab, c))

    def fit(self, points, C0, max_iter: int, early_stop: bool = True):
        """Lloyd's algorithm.  Returns dict(centroids, labels, iterations,
        sse, sse_hist, changed_hist)."""
        p = self._pts(points)
        n, d = p.shape
        c0 = self._cent(C0, d)
        k = c0.shape[0]
        C = np.empty_like(c0)
        lab = np.empty(n, dtype=np.int32)
        it = ctypes.c_int(0)
        sse = ctypes.c_double(0.0)
        m = max(int(max_iter), 1)
        hist = np.zeros(m, dtype=np.float64)
        chg = np.zeros(m, dtype=np.int64)
        rc = self.lib.oracle_fit(p, n, d, k, c0, int(max_iter), int(bool(early_stop)), C, lab,
                                 ctypes.byref(it), ctypes.byref(sse), self._ptr(hist),
                                 self._ptr(chg))
        if rc != 0:
            raise RuntimeError(f"oracle_fit failed ({rc})")
        iters = it.value
        return dict(centroids=C, labels=lab, iterations=iters, sse=sse.value,
                    sse_hist=hist[:iters].copy(), changed_hist=chg[:iters].copy())


def relative_gap(best: np.ndarray, second: np.ndarray) -> np.ndarray:
    """(d2 - d1) / max(d1, tiny): the near-tie measure of the parity rule.
    Points whose gap is below 1e-5 may legitimately flip label between an
    FP32 and an FP64 evaluation."""
    tiny = np.finfo(np.float64).tiny
    return (second - best) / np.maximum(best, tiny)


_default: Optional[Oracle] = None


def get() -> Oracle:
    """The default oracle (built on first use)."""
    global _default
    if _default is None:
        _default = Oracle()
    return _default


if __name__ == "__main__":  # pragma: no cover
    print(build(), file=sys.stderr)
