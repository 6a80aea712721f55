"""Degenerate and extreme cases of Algorithms 2 and 3 through the C ABI,
against the FP64 oracle at the parity tolerances of test_gpu_parity:

* the smallest and largest tensor orders: a matrix (d = 2, where both
  algorithms reduce to a shifted randomized range finder per side) and
  d = TK_MAX_D = 8;
* rank one with no oversampling (l = 1): the svd of a single column, and
  the shift rule acting on Sigma(1, 1);
* the largest power count, q = TK_MAX_Q = 32;
* r_k = n_k - 1 with l clamped at n_k, and l clamped by the columns of an
  unfolding that earlier modes have shrunk.
Empty tensors and ranks outside 1 <= r_k < n_k are rejected on the host
before any launch (test_abi).
"""
import numpy as np
import pytest

from oracle import tucker as T
from paper_2506_04840_gb300 import api
from paper_2506_04840_gb300 import inputs as I

from gpu_helpers import run_hosvd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [
    # shape, ranks, s, q, seed of the input
    ((300, 200), (12, 12), 6, 2, 21),                        # d = 2
    ((4, 3, 4, 3, 3, 4, 3, 3), (2,) * 8, 1, 1, 22),          # d = TK_MAX_D
    ((30, 25, 20), (1, 1, 1), 0, 2, 23),                     # l = 1
    ((24, 20, 16), (5, 4, 3), 4, api.TK_MAX_Q, 24),          # q = TK_MAX_Q
    ((12, 40, 3), (11, 2, 2), 3, 1, 25),                     # l = n_k; l = columns
]


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


@pytest.mark.parametrize("case", CASES, ids=["d2", "d8", "l1", "qmax", "clamped"])
@pytest.mark.parametrize("st", [True, False], ids=["st", "t"])
@pytest.mark.parametrize("dtype", [np.float64, np.float32], ids=["f64", "f32"])
def test_edge_cases_match_oracle(lib, case, st, dtype):
    shape, r, s, q, seed = case
    A = I.tucker_plus_noise(shape, [min(x + 1, n - 1) for x, n in zip(r, shape)], seed,
                            noise=1e-3, decay=0.8, dtype=dtype)
    f = T.rsthosvd if st else T.rthosvd
    Gw, Uw, sw = f(A, list(r), s, q)
    G, Us, info = run_hosvd(A, list(r), s, q, st=st)
    assert info["l"] == [x["l"] for x in sw]
    re_w = T.rel_error(A, Gw, Uw)
    re_g = T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= (1e-12 if dtype == np.float64 else 1e-6), (re_g, re_w)
    for k, (Ug, Uk) in enumerate(zip(Us, Uw)):
        Ug = np.asarray(Ug, dtype=np.float64)
        orth = np.abs(Ug.T @ Ug - np.eye(r[k])).max()
        assert orth <= (1e-13 if dtype == np.float64 else 1e-6), (k, orth)
        j = T.separated_block(np.asarray(sw[k]["sigma"]), r[k])
        if j > 0:
            sines = T.principal_sines(Ug[:, :j], Uk[:, :j]).max()
            assert sines <= (1e-9 if dtype == np.float64 else 1e-5), (k, j, sines)
    # the core is the projection of A on the returned factors
    Gchk = A.astype(np.float64)
    for k in range(A.ndim):
        Gchk = T.mode_product(Gchk, Us[k].T.astype(np.float64), k)
    assert _rel(G, Gchk) <= (1e-12 if dtype == np.float64 else 1e-5)
