"""Pins of the oracle's Gaussian test matrix (CPU only).

Philox4x32-10 is checked against Triton's independent implementation (run
in interpreter mode on the CPU); the hand-written FP32 log / cos / sin are
checked against libm over every input they can receive; the resulting
Gaussians against the normal distribution.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import omega as om

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_matches_triton_reference_implementation():
    pytest.importorskip("triton")
    rng = np.random.default_rng(7)
    cases = [[0, 0, 0, 0, 0],
             [0xFFFFFFFFFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF]]
    for _ in range(6):
        cases.append([int(rng.integers(0, 2**63))] + [int(x) for x in rng.integers(0, 2**32, 4)])
    env = dict(os.environ, TRITON_INTERPRET="1")
    out = subprocess.run([sys.executable, os.path.join(HERE, "_philox_triton.py")],
                         input=json.dumps(cases), capture_output=True, text=True, env=env,
                         timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    want = json.loads(out.stdout)
    for case, w in zip(cases, want):
        seed, c0, c1, c2, c3 = case
        got = [int(x) for x in om.philox4x32_10(c0, c1, c2, c3, seed)]
        assert got == w, (case, got, w)


def test_log_u1_within_3_ulp_everywhere():
    wa = (np.arange(0, 2**23, dtype=np.uint32) << np.uint32(9))
    got = om.log_u1(wa).astype(np.float64)
    u1 = (2.0 * (wa >> np.uint32(9)).astype(np.float64) + 1.0) * 2.0**-24
    ref = np.log(u1)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(got - ref) / ulp) <= 3.0
    assert np.all(got < 0)


def test_cos_sin_within_2e7_everywhere():
    wb = (np.arange(0, 2**24, dtype=np.uint32) << np.uint32(8))
    c, s = om.cos_sin_2pi(wb)
    ang = 2.0 * np.pi * (wb >> np.uint32(8)).astype(np.float64) / 2.0**24
    assert np.max(np.abs(c - np.cos(ang))) <= 2e-7
    assert np.max(np.abs(s - np.sin(ang))) <= 2e-7
    # octant boundaries hit the exact values
    assert c[0] == 1.0 and s[0] == 0.0
    assert c[2**22] == 0.0 or abs(c[2**22]) < 1e-7


def test_gaussian_distribution():
    stats = pytest.importorskip("scipy.stats")
    z = om.omega_rows(0, 0, 250_000, 8, seed=0).ravel().astype(np.float64)
    assert abs(z.mean()) < 5e-3
    assert abs(z.std() - 1.0) < 5e-3
    ks = stats.kstest(z, "norm")
    assert ks.pvalue > 1e-3
    # fourth moment of N(0,1) is 3
    assert abs(np.mean(z**4) - 3.0) < 0.05


def test_streams_are_counter_based_and_independent():
    full = om.omega_rows(2, 0, 1000, 13, seed=11, tag=3)
    part = om.omega_rows(2, 400, 200, 13, seed=11, tag=3)
    assert np.array_equal(full[400:600], part)
    # a wider l keeps the first columns (column groups of four are independent)
    wide = om.omega_rows(2, 0, 1000, 20, seed=11, tag=3)
    assert np.array_equal(wide[:, :13], full)
    other_mode = om.omega_rows(1, 0, 1000, 13, seed=11, tag=3)
    other_tag = om.omega_rows(2, 0, 1000, 13, seed=11, tag=4)
    other_seed = om.omega_rows(2, 0, 1000, 13, seed=12, tag=3)
    for o in (other_mode, other_tag, other_seed):
        c = np.corrcoef(full.ravel(), o.ravel())[0, 1]
        assert abs(c) < 0.02
    # columns are uncorrelated
    C = np.corrcoef(om.omega_rows(0, 0, 20000, 8, seed=0).T)
    assert np.max(np.abs(C - np.eye(8))) < 0.05


def test_empty_shapes():
    assert om.omega_rows(0, 0, 0, 5).shape == (0, 5)
    assert om.omega_rows(0, 0, 3, 0).shape == (3, 0)
