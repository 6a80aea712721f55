"""bench.py's workload table on the CPU: every single-tensor workload has an
input generator, and the reference arm's oracle step runs each workload's
variant (Algorithm 2 or 3, precision form, Algorithm 4, holistic,
structured test matrix) on a tiny stand-in tensor."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2506_04840_gb300 import inputs as I  # noqa: E402

SINGLE = sorted(k for k, w in bench.WORKLOADS.items() if w.get("kind") is None)


def test_workload_fields():
    for name in SINGLE:
        w = bench.WORKLOADS[name]
        d = len(w["shape"])
        assert len(w["r"]) == d and all(1 <= r < n for r, n in zip(w["r"], w["shape"])), name
        assert w["dtype"] in ("f32", "f64") and w["prec"] in (0, 1), name
        assert w["s"] >= 0 and 0 <= w["q"] <= 32, name
        assert w.get("omega", 0) in (0, 1, 2, 3), name
        if w.get("pve") is not None:
            assert w["st"] and w["q"] >= 1 and w["prec"] == 0, name
    assert bench.DEFAULT_WORKLOAD in SINGLE


@pytest.mark.parametrize("name", SINGLE)
def test_every_workload_has_a_generator(name, monkeypatch):
    """make_input reaches a generator for each name (stubbed: no tensor of
    the full size is built here), with the rank's own seed."""
    calls = []

    def stub(tag):
        def f(*a, **k):
            calls.append((tag, a, k))
            return np.zeros((2, 2, 2), dtype=np.float32)
        return f

    for fn in ("tucker_plus_noise", "inverse_radius", "sparse_rank_one_sum", "superdiagonal",
               "hilbert"):
        monkeypatch.setattr(I, fn, stub(fn))
    bench.make_input(name, rank=1)
    assert len(calls) == 1, name
    tag, a, k = calls[0]
    if "seed" in k:
        assert k["seed"] >= 1000, (name, k)     # rank 1 draws its own content


@pytest.mark.parametrize("name", SINGLE)
def test_oracle_step_runs_each_variant(name):
    w = dict(bench.WORKLOADS[name])
    d = len(w["shape"])
    shape = [14, 12, 10, 9][:d]
    w["shape"] = shape
    w["r"] = [3] * d
    w["s"] = 2
    w["q"] = min(w["q"], 3) if w.get("pve") is None else 4
    A = I.tucker_plus_noise(shape, [4] * d, 3, noise=1e-2, dtype=np.float64)
    re = bench.oracle_step(A, w)
    assert 0.0 <= re < 1.0, (name, re)
