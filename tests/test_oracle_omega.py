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


# ---- structured test matrices (Section 5.5) --------------------------------

def test_uniform_map_is_exact_symmetric_and_fills_the_interval():
    """Every 24-bit word prefix maps to its own odd multiple of 2^-24 in
    (-1, 1), monotone, with u(complement) = -u: the map covers the interval
    evenly, so a wrong shift, offset or scale shows up here."""
    top = np.arange(1 << 24, dtype=np.uint64)
    w = (top << np.uint64(8)).astype(np.uint32)
    u = om.uniform_from_word(w).astype(np.float64)
    num = u * 2.0 ** 24
    assert np.array_equal(num, np.round(num)) and np.all(np.abs(num) % 2 == 1)
    assert np.all(np.diff(u) == 2.0 ** -23)
    assert u[0] == -1.0 + 2.0 ** -24 and u[-1] == 1.0 - 2.0 ** -24
    comp = om.uniform_from_word((w ^ np.uint32(0xFFFFFF00)).astype(np.uint32)).astype(np.float64)
    assert np.array_equal(comp, -u)
    # the low 8 bits do not matter
    assert np.array_equal(om.uniform_from_word(w | np.uint32(0xFF)).astype(np.float64), u)


def test_uniform_matrix_distribution_and_words():
    from scipy import stats
    U = om.uniform_rows(1, 5, 20000, 7, seed=11, tag=3)
    x = U.astype(np.float64).ravel()
    assert np.all(np.abs(x) < 1.0)
    assert abs(x.mean()) < 4 * np.sqrt(1 / 3 / x.size)
    assert abs(x.var() - 1 / 3) < 0.01
    assert stats.kstest(x, "uniform", args=(-1, 2)).pvalue > 1e-3
    # entry (j, c) is word c mod 4 of the Gaussian entry's counter
    j = np.arange(5, 20005, dtype=np.uint64)
    ws = om.philox4x32_10(j, j >> np.uint64(32), np.uint64(1), np.uint64(1 | (3 << 8)), 11)
    assert np.array_equal(U[:, 6], om.uniform_from_word(ws[2]))
    # columns are uncorrelated
    C = np.corrcoef(U.T.astype(np.float64))
    assert np.abs(C - np.eye(7)).max() < 0.05


@pytest.mark.parametrize("kind", [om.OMEGA_KR_GAUSS, om.OMEGA_KR_UNIFORM])
def test_khatri_rao_rows_follow_the_unfolding_column_order(kind):
    """Brute force on a small order-4 shape: Omega_k(j, c) is the product of
    the factors' entries at the per-mode indices of unfolding column j
    (mixed radix, lowest mode fastest), for every k."""
    shape = (3, 4, 2, 5)
    l = 6
    for k in range(4):
        Om = om.omega_matrix(kind, shape, k, l, seed=9, tag=2)
        others = [m for m in range(4) if m != k]
        F = {m: om.kr_factor(k, m, shape[m], l, kind == om.OMEGA_KR_GAUSS, seed=9, tag=2)
             for m in others}
        assert Om.shape == (int(np.prod([shape[m] for m in others])), l)
        for j in range(Om.shape[0]):
            rest, idx = j, {}
            for m in others:
                idx[m] = rest % shape[m]
                rest //= shape[m]
            for c in range(l):
                want = 1.0
                for m in others:
                    want *= float(F[m][idx[m], c])
                assert Om[j, c] == pytest.approx(want, rel=1e-15, abs=0.0)


@pytest.mark.parametrize("kind", list(om.OMEGA_KINDS))
def test_sketch_equals_the_unfolding_product_by_another_route(kind):
    """Y = X_(k) Omega_k against a contraction that never forms the
    unfolding: for the dense kinds, Omega's rows placed back on the tensor's
    index grid; for the Khatri-Rao kinds, one factor contracted per mode
    (einsum with the column index c shared)."""
    from oracle import tucker as T
    rng = np.random.default_rng(4)
    shape = (5, 3, 4)
    X = rng.standard_normal(shape)
    l = 5
    letters = "abc"
    for k in range(3):
        Y = T.sketch(X, k, l, seed=3, tag=1, kind=kind)
        others = [m for m in range(3) if m != k]
        if kind in (om.OMEGA_KR_GAUSS, om.OMEGA_KR_UNIFORM):
            Fs = [om.kr_factor(k, m, shape[m], l, kind == om.OMEGA_KR_GAUSS, seed=3,
                               tag=1).astype(np.float64) for m in others]
            spec = letters + "," + ",".join(letters[m] + "z" for m in others) + \
                "->" + letters[k] + "z"
            Y2 = np.einsum(spec, X, *Fs)
        else:
            cols = shape[others[0]] * shape[others[1]]
            rows = (om.omega_rows if kind == om.OMEGA_GAUSS else om.uniform_rows)(
                k, 0, cols, l, seed=3, tag=1).astype(np.float64)
            # row j = i_lo + n_lo * i_hi of the unfolding's columns
            W = rows.reshape(shape[others[1]], shape[others[0]], l)   # [i_hi, i_lo, c]
            Y2 = np.zeros((shape[k], l))
            for i_lo in range(shape[others[0]]):
                for i_hi in range(shape[others[1]]):
                    sl = [slice(None)] * 3
                    sl[others[0]], sl[others[1]] = i_lo, i_hi
                    Y2 += np.outer(X[tuple(sl)], W[i_hi, i_lo])
        assert np.allclose(Y, Y2, rtol=1e-12, atol=1e-12), (kind, k)


def test_khatri_rao_factors_are_distinct_draws():
    """Each (mode k, factor m) pair has its own stream, and the factor
    entries have the stated distributions."""
    from scipy import stats
    a = om.kr_factor(0, 1, 3000, 8, True, seed=5)
    b = om.kr_factor(2, 1, 3000, 8, True, seed=5)
    c = om.kr_factor(0, 2, 3000, 8, True, seed=5)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    assert stats.kstest(a.astype(np.float64).ravel(), "norm").pvalue > 1e-3
    u = om.kr_factor(0, 1, 3000, 8, False, seed=5).astype(np.float64).ravel()
    assert np.all(np.abs(u) < 1) and stats.kstest(u, "uniform", args=(-1, 2)).pvalue > 1e-3
    # not the dense matrix's draws
    assert not np.array_equal(a[:, :4], om.omega_rows(0, 0, 3000, 4, seed=5))
