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


def test_config_is_the_same_object_in_both_arms():
    """The driver compares the two arms' config: it names the workload only
    (no measured values), so both arms print the same dict."""
    for name in bench.WORKLOADS:
        cfg = bench.config_of(name)
        assert cfg["workload"] == name and cfg["desc"] == bench.WORKLOADS[name]["desc"]
        assert "l2" in cfg
        assert set(cfg) == {"workload", "desc", "l2"}, name
    assert bench.DEFAULT_WORKLOAD == "invradius1000_bf16power_st"
    assert bench.WORKLOADS[bench.DEFAULT_WORKLOAD]["companion"] == "invradius1000_fp32_st"


def test_oracle_slab_sample_is_a_prefix_of_the_tensor():
    """The oracle's bounded sample of the 1000^3 workloads is the first
    slices of the same tensor (built alone: bitwise the same values), counted
    as that fraction of a tensor."""
    w = dict(bench.WORKLOADS[bench.DEFAULT_WORKLOAD])
    full = I.inverse_radius(96, seed=3)
    w["shape"] = [96, 96, 96]
    w["oracle_slices"] = 20
    frac, As, what = bench.oracle_sample("x", w, full)
    assert frac == pytest.approx(20 / 96)
    assert np.array_equal(As, full[:, :, :20])
    alone = I.inverse_radius(96, seed=3, slices=20)
    assert np.array_equal(alone, As)
    assert "20 of the 96" in what


def test_roofline_is_the_power_pass():
    """The roofline object reports the shifted-power pass against HBM: the
    fused pass when it ran, else the two CUDA-core halves together."""
    def kind(launches=0, ms=0.0, by=0.0, fl=0.0):
        return dict(launches=launches, ms=ms, bytes=by, flops=fl)
    names = ["sketch", "power_w", "power_y", "power_fused", "small_svd", "ttm", "error",
             "convert", "ritz"]
    prof = {"kinds": {k: kind() for k in names}, "kernels": 0}
    prof["kinds"]["small_svd"] = kind(12, 50.0, 1e6)
    prof["kinds"]["power_w"] = kind(3, 6.0, 12e9)
    prof["kinds"]["power_y"] = kind(3, 6.0, 12e9)
    pk = {"hbm_gbs": 6000.0}
    name, roof = bench._roofline(prof, pk, "measured", "x")
    assert name == "power_w+power_y" and roof["bound"] == "hbm"
    assert roof["achieved"] == pytest.approx(4e9 / 4e-3 / 1e9)
    prof["kinds"]["power_fused"] = kind(2, 1.0, 4e9)
    name, roof = bench._roofline(prof, pk, "measured", "x")
    assert name == "power_fused"
    assert roof["achieved"] == pytest.approx(2e9 / 0.5e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / 6000.0)
    assert roof["traffic"] == pytest.approx(bench.NCU_TRAFFIC_RATIO["power_fused"] * 2e9)
    lat = bench._latency(prof, 1, 100.0)
    assert lat["small_svd"]["avg_launch_us"] == pytest.approx(50.0 / 12 * 1e3)
    pp = bench._power_pass(prof, 1, pk)
    assert pp["fp32_two_pass"]["reads_of_x_per_step"] == 2
