"""Structured test matrices (Section 5.5): dense uniform and Khatri-Rao
products of Gaussian or uniform factors, through the C ABI, against the
oracle's definitions.

* Omega itself: bit-exact against the oracle's FP64 values rounded to
  FP32 (both take the Khatri-Rao product in FP64 with the same rounding
  sequence, exact for two factors).
* Whole decompositions: the tolerances of the Gaussian parity tests
  (|RE_gpu - RE_oracle| <= 1e-6 for FP32, 1e-12 for FP64; factors
  orthonormal; sines of the separated leading block).
"""
import numpy as np
import pytest

from oracle import omega as om
from oracle import tucker as T
from paper_2506_04840_gb300 import api
from paper_2506_04840_gb300 import inputs as I

from gpu_helpers import run_hosvd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KINDS = {api.TK_OMEGA_GAUSS: om.OMEGA_GAUSS, api.TK_OMEGA_UNIFORM: om.OMEGA_UNIFORM,
         api.TK_OMEGA_KR_GAUSS: om.OMEGA_KR_GAUSS, api.TK_OMEGA_KR_UNIFORM: om.OMEGA_KR_UNIFORM}


@pytest.mark.parametrize("kind", list(KINDS))
@pytest.mark.parametrize("shape,l,seed,tag", [
    ((7, 5, 6), 9, 0, 0),
    ((33, 1, 20), 13, (1 << 40) + 7, 5),
    ((3, 4, 5, 2), 6, 3, (1 << 24) - 1),
    ((2, 3, 2, 3, 2), 128, 11, 2),
])
def test_omega_matrix_matches_definition(lib, kind, shape, l, seed, tag):
    for k in range(len(shape)):
        cols = int(np.prod([n for m, n in enumerate(shape) if m != k]))
        out = torch.empty(cols * l, dtype=torch.float32, device="cuda")
        api.tucker_debug_omega_matrix(kind, list(shape), k, l, seed, tag, out)
        got = out.cpu().numpy().reshape((cols, l), order="F").astype(np.float64)
        want = om.omega_matrix(KINDS[kind], shape, k, l, seed=seed, tag=tag)
        assert np.array_equal(got.astype(np.float32).view(np.uint32),
                              want.astype(np.float32).view(np.uint32)), k


CASES = [
    # shape, ranks, s, q, seed of the input
    ((40, 36, 30), (6, 5, 4), 5, 2, 11),
    ((21, 18, 15, 12), (4, 3, 3, 2), 3, 1, 12),
    ((64, 20, 131), (10, 7, 12), 10, 1, 13),
    ((40, 36, 30), (6, 5, 4), 5, 0, 15),       # q = 0: the sketch alone
]


def _check_factors(Us_g, Us_w, stats_w, dtype):
    for k, (Ug, Uw) in enumerate(zip(Us_g, Us_w)):
        r = Uw.shape[1]
        Ug = np.asarray(Ug, dtype=np.float64)
        assert np.abs(Ug.T @ Ug - np.eye(r)).max() <= (1e-13 if dtype == np.float64 else 1e-6)
        sig = np.asarray(stats_w[k]["sigma"])
        if not stats_w[k]["alpha"]:
            sig = sig ** 2
        j = T.separated_block(sig, r)
        if j > 0:
            tol = 1e-9 if dtype == np.float64 else (1e-5 if stats_w[k]["alpha"] else 1e-4)
            assert T.principal_sines(Ug[:, :j], Uw[:, :j]).max() <= tol, k


@pytest.mark.parametrize("kind", [api.TK_OMEGA_UNIFORM, api.TK_OMEGA_KR_GAUSS,
                                  api.TK_OMEGA_KR_UNIFORM])
@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("st", [True, False])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_structured_hosvd_matches_oracle(lib, kind, case, st, dtype):
    """FP32 ST-HOSVD runs on the rotated (mode-major) layout, where the
    structured Omega is written in the layout's column order; T-HOSVD and
    FP64 on the strided natural layout."""
    shape, r, s, q, seed = case
    A = I.tucker_plus_noise(shape, [min(x + 2, n - 1) for x, n in zip(r, shape)], seed,
                            noise=1e-3, decay=0.85, dtype=dtype)
    f = T.rsthosvd if st else T.rthosvd
    Gw, Uw, sw = f(A, list(r), s, q, omega=KINDS[kind])
    G, Us, info = run_hosvd(A, list(r), s, q, st=st, omega=kind, workspace=True)
    re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= (1e-12 if dtype == np.float64 else 1e-6), (re_g, re_w)
    _check_factors(Us, Uw, sw, dtype)


def test_structured_kinds_on_tensor_C_full_size(lib):
    """Section 5.5's setting at the paper's size: tensor C (600^3, slow
    decay), r = 20, s = 10, q = 1, FP32 ST-HOSVD.  Each kind's error equals
    the oracle's (stored by tests/golden/make_structured_omega_C600.py)
    within the FP32 tolerance, lies above the closed-form optimum, and the
    kinds are comparable: within 2% of the Gaussian sketch's error."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                     "structured_omega_C600.json")))
    A = I.superdiagonal(600, "slow", seed=11, dtype=np.float32)
    v = I.superdiagonal_values(600, "slow")
    opt = float(np.sqrt(np.sum(v[20:] ** 2) / np.sum(v ** 2)))
    res = {}
    for kind, name in KINDS.items():
        G, Us, _ = run_hosvd(A, [20, 20, 20], 10, 1, omega=kind, stats=False)
        res[name] = T.rel_error(A, G, Us)
        assert abs(res[name] - g["re"][name]) <= 1e-6, (name, res[name], g["re"][name])
        assert res[name] >= opt * (1 - 1e-6), (name, res[name], opt)
    for name, re in res.items():
        assert re <= 1.02 * res[om.OMEGA_GAUSS], (name, re, res)
