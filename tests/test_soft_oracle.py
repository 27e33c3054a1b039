"""The FP64 soft / hard k-means loss oracle against its pins (CPU), and
planted mistakes in copies of it, each of which must fail a pin."""
import importlib.util
import os
import tempfile

import pytest

import oracle.soft_kmeans as sk
from soft_pins import pin_fd, pin_hard, pin_lloyd, pin_shift, pin_uniform, run_soft_pins

SRC = sk.__file__


@pytest.mark.parametrize("pin", [pin_fd, pin_uniform, pin_shift], ids=lambda p: p.__name__)
def test_soft_pin(pin):
    fails = pin(sk)
    assert not fails, "\n".join(fails)


@pytest.mark.parametrize("pin", [pin_lloyd, pin_hard], ids=lambda p: p.__name__)
def test_soft_pin_against_lloyd_oracle(oracle, pin):
    fails = pin(sk, oracle)
    assert not fails, "\n".join(fails)


MUTANTS = [
    ("softmax row term dropped", "dD = -(W * (g - rho)) / tau", "dD = -(W * g) / tau"),
    ("wrong sign of the softmax derivative", "dD = -(W * (g - rho)) / tau", "dD = (W * (g - rho)) / tau"),
    ("direct weighted-sum term dropped", "gP = gP + (W / N[None, :]) @ gC", "gP = gP"),
    ("loss-stage entropy term dropped", "dD = W * (1.0 - (D - E) / tau)", "dD = W"),
    ("update not normalised by the weight sum", "C = (W.T @ P) / W.sum(axis=0)[:, None]",
     "C = (W.T @ P) / W.shape[0]"),
    ("g_ij measured from the old centroid", "P[:, None, :] - Cn[None, :, :], gC",
     "P[:, None, :] - Ct[None, :, :], gC"),
    ("softmax over points instead of centroids", "E / E.sum(axis=1, keepdims=True)",
     "E / E.sum(axis=0, keepdims=True)"),
    ("hard gradient sign flipped", "np.add.at(gC, a, -2.0 * r)", "np.add.at(gC, a, 2.0 * r)"),
]


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_soft_pin(oracle, desc, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not found once: {old!r}"
    d = tempfile.mkdtemp(prefix="soft_mutant_")
    path = os.path.join(d, "soft_mutant.py")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    spec = importlib.util.spec_from_file_location("soft_mutant", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    assert run_soft_pins(mod, oracle), f"planted mistake '{desc}' passed every pin"
