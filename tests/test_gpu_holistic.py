"""Holistic variants (Algorithms A.2 and B.1) through the C ABI against
the oracle's ``holistic``.

* |RE_gpu - RE_oracle| <= 1e-6 for FP32 and 1e-12 for FP64; factors
  orthonormal; the core is the projection of A on the returned factors.
* Factor subspaces: V_k comes from the eigenvectors of B_(k) B_(k)^T, with
  B carrying the rounding of the input's arithmetic (FP32: a few
  contractions, ~100 u relative).  To first order (Davis-Kahan) the
  leading j columns then turn by at most ~100 u / g_j, g_j = (sigma_j^2 -
  sigma_{j+1}^2) / sigma_1^2 on the oracle's singular values of that
  unfolding; the check takes the largest j <= r_k with g_j >= 1e-3 and
  that bound (u = 2^-24 for FP32, 2^-53 for FP64, at least 1e-12).
"""
import numpy as np
import pytest

from oracle import tucker as T
from paper_2506_04840_gb300 import api
from paper_2506_04840_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def run_holistic(A, r, s, q, st, shift=api.TK_SHIFT_PAPER, omega=api.TK_OMEGA_GAUSS,
                 workspace=False):
    d, dims = A.ndim, list(A.shape)
    dt = np.float64 if A.dtype == np.float64 else np.float32
    tdt = torch.float64 if dt == np.float64 else torch.float32
    Ad = api.to_device(A, dt)
    core = torch.full((int(np.prod(r)),), float("nan"), dtype=tdt, device="cuda")
    U = [torch.full((dims[k] * r[k],), float("nan"), dtype=tdt, device="cuda") for k in range(d)]
    opts = api.make_opts(d, q, s, shift=shift, omega=omega)
    if workspace:
        nb = api.tucker_holistic_workspace_size(Ad, dims, r, opts, st)
        ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
        opts = api.make_opts(d, q, s, shift=shift, omega=omega, workspace=ws)
    info = api.tucker_holistic(Ad, dims, r, opts, st, core, U, stats=True)
    torch.cuda.synchronize()
    G = api.from_device(core, r)
    Us = [api.from_device(U[k], [dims[k], r[k]]) for k in range(d)]
    return G, Us, info


CASES = [
    # shape, ranks, s, q, seed of the input
    ((40, 36, 30), (6, 5, 4), 5, 2, 11),
    ((21, 18, 15, 12), (4, 3, 3, 2), 3, 1, 12),
    ((64, 20, 131), (10, 7, 12), 10, 1, 13),
    ((33, 33, 33), (28, 8, 8), 6, 2, 14),      # l_1 clamped at n_1: Q_1 square
    ((40, 36, 30), (6, 5, 4), 5, 0, 15),       # q = 0
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("st", [1, 0])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("shift", [api.TK_SHIFT_PAPER, api.TK_SHIFT_NONE])
def test_holistic_matches_oracle(lib, case, st, dtype, shift):
    shape, r, s, q, seed = case
    A = I.tucker_plus_noise(shape, [min(x + 2, n - 1) for x, n in zip(r, shape)], seed,
                            noise=1e-3, decay=0.85, dtype=dtype)
    rule = T.SHIFT_PAPER if shift == api.TK_SHIFT_PAPER else T.SHIFT_NONE
    Gw, Uw, sw = T.holistic(A, list(r), s, q, rule=rule, st=bool(st))
    G, Us, info = run_holistic(A, list(r), s, q, st, shift=shift, workspace=(seed % 2 == 0))
    assert info["l"] == [x["l"] for x in sw]
    re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= (1e-12 if dtype == np.float64 else 1e-6), (re_g, re_w)
    Gm = A.astype(np.float64)
    for k in range(A.ndim):
        Ug = np.asarray(Us[k], dtype=np.float64)
        assert np.abs(Ug.T @ Ug - np.eye(r[k])).max() <= (1e-12 if dtype == np.float64 else 1e-6)
        Gm = T.mode_product(Gm, Ug.T, k)
        sig = np.asarray(sw[k]["sigma_small"], dtype=np.float64)
        j = T.separated_block(sig, r[k], gap=1e-3)
        if j:
            g = (sig[j - 1] ** 2 - sig[j] ** 2) / sig[0] ** 2
            u = 2.0 ** -53 if dtype == np.float64 else 2.0 ** -24
            tol = max(100 * u / g, 1e-12)
            assert T.principal_sines(Ug[:, :j], Uw[k][:, :j]).max() <= tol, (k, j, g)
    scale = np.abs(A).max()
    assert np.abs(G - Gm).max() <= (1e-12 if dtype == np.float64 else 1e-5) * scale


def test_holistic_structured_omega_and_full_size(lib):
    """Algorithm B.1 on the 400^3 FP32 Tucker workload (r = 20, s = 10,
    q = 2) against the oracle, with the Gaussian and a Khatri-Rao test
    matrix."""
    A = I.tucker_plus_noise([400, 400, 400], [20, 20, 20], seed=2, noise=1e-4, decay=0.8,
                            dtype=np.float32)
    for omega, name in ((api.TK_OMEGA_GAUSS, "gauss"), (api.TK_OMEGA_KR_GAUSS, "kr_gauss")):
        Gw, Uw, _ = T.holistic(A.astype(np.float64), [20] * 3, 10, 2, omega=name)
        G, Us, _ = run_holistic(A, [20] * 3, 10, 2, 1, omega=omega)
        re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
        assert abs(re_g - re_w) <= 1e-6, (name, re_g, re_w)
