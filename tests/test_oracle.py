"""The FP64 oracle against its pins (CPU only), and mutation checks that a
plausible mistake planted in a copy of the oracle source fails a pin."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as oracle_pkg
from oracle_pins import (run_pins, pin_worked, pin_vq, pin_optimum, pin_invariants,
                         pin_sklearn)

SRC = os.path.join(os.path.dirname(oracle_pkg.__file__), "dkm_oracle.c")


@pytest.mark.parametrize("pin", [pin_worked, pin_vq, pin_optimum, pin_invariants, pin_sklearn],
                         ids=lambda p: p.__name__)
def test_oracle_pin(oracle, pin):
    fails = pin(oracle)
    assert not fails, "\n".join(fails)


def test_sklearn_pin_is_active():
    pytest.importorskip("sklearn")


def test_relative_gap():
    g = oracle_pkg.relative_gap(np.array([1.0, 0.0, 4.0]), np.array([1.5, 2.0, 4.0]))
    assert g[0] == pytest.approx(0.5) and g[2] == 0.0 and g[1] > 1e300


def test_update_rejects_bad_label(oracle):
    pts = np.zeros((3, 2), np.float32)
    with pytest.raises(ValueError):
        oracle.update(pts, np.array([0, 5, 0], np.int32), np.zeros((2, 2)))


def test_max_iter_zero_labels_only(oracle):
    pts = np.array([[0, 0], [10, 0]], np.float32)
    C0 = np.array([[1.0, 0.0], [9.0, 0.0]])
    r = oracle.fit(pts, C0, max_iter=0)
    assert r["iterations"] == 0
    assert list(r["labels"]) == [0, 1]
    assert np.array_equal(r["centroids"], C0)
    assert r["sse"] == pytest.approx(2.0)


# (description, original text, planted mistake)
MUTANTS = [
    ("tie goes to the highest index", "if (s < d1) {", "if (s <= d1) {"),
    ("last coordinate dropped from the distance",
     "for (int t = 0; t < d; ++t) {\n        double diff", "for (int t = 0; t < d - 1; ++t) {\n        double diff"),
    ("wrong sign in the difference", "double diff = (double)p[t] - c[t];",
     "double diff = (double)p[t] + c[t];"),
    ("empty cluster reset to the origin", ": C_prev[o];", ": 0.0;"),
    ("transposed coordinate in the cluster sum", "+= (double)pts[i * d + t];",
     "+= (double)pts[i * d + (d - 1 - t)];"),
    ("mean divides by count + 1", "S[o] / (double)cnt[j]", "S[o] / (double)(cnt[j] + 1)"),
    ("second-best distance never updated", "} else if (s < d2) {\n            d2 = s;",
     "} else if (s < d2) {\n            d2 = d2;"),
    ("early stop tolerates one changed label", "if (early_stop && changed == 0) break;",
     "if (early_stop && changed <= 1) break;"),
    ("SSE summed with the wrong centroid index",
     "s += sq_dist(pts + i * d, C + (int64_t)labels[i] * d, d);",
     "s += sq_dist(pts + i * d, C + (int64_t)(labels[i] > 0 ? labels[i] - 1 : 0) * d, d);"),
    ("point index stride mixed up in assignment", "nearest_two(pts + i * d, d, C, k, &a, &d1, &d2);",
     "nearest_two(pts + (i / 2) * d, d, C, k, &a, &d1, &d2);"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(desc, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    tmp = tempfile.mkdtemp(prefix="oracle_mutant_")
    try:
        c = os.path.join(tmp, "m.c")
        with open(c, "w") as f:
            f.write(src.replace(old, new))
        so = os.path.join(tmp, "libm.so")
        oracle_pkg.build(src=c, out=so, openmp=False)
        fails = run_pins(oracle_pkg.Oracle(so))
        assert fails, f"planted mistake '{desc}' passed every pin"
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
