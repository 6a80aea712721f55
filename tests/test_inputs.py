"""The seeded input recipes (CPU only).

The benchmark and parity workloads are synthetic; these tests check that
the generators make what their recipes state: the closed-form entries of
the Hilbert-type and inverse-radius tensors, the noise levels, the Haar
factors' orthonormality, the closed-form spectra of Section 5.1's tensor C,
the sparsity and weights of tensor B, the constraints on batch instances
and serving requests, and bitwise reproducibility from the seed.
"""
import math

import numpy as np
import pytest

from paper_2506_04840_gb300 import inputs as I


def _unfold(X, k):
    return np.moveaxis(X, k, 0).reshape(X.shape[k], -1)


def test_hilbert_entries():
    A = I.hilbert([4, 3, 5])
    assert A.flags["F_CONTIGUOUS"]
    for i, j, k in [(1, 1, 1), (4, 3, 5), (2, 3, 1)]:
        assert A[i - 1, j - 1, k - 1] == 1.0 / (i + j + k - 2)
    B = I.hilbert([3, 2, 2, 2])
    assert B[2, 1, 1, 1] == 1.0 / (3 + 2 + 2 + 2 - 3)


def test_inverse_radius_entries_and_noise_level():
    n = 40
    A = I.inverse_radius(n, seed=3, noise=0.0, dtype=np.float64)
    i = np.arange(1, n + 1, dtype=np.float64)
    A0 = 1.0 / np.sqrt(i[:, None, None] ** 2 + i[None, :, None] ** 2 + i[None, None, :] ** 2)
    assert np.array_equal(A, A0)
    An = I.inverse_radius(n, seed=3, noise=1e-2, dtype=np.float64)
    E = An - A0
    want = 1e-2 * np.linalg.norm(A0) / math.sqrt(n ** 3)
    assert abs(E.std() / want - 1.0) < 0.01
    assert abs(E.mean()) < 4 * want / math.sqrt(n ** 3)
    # the first slices alone are the same bits as the whole tensor's
    S = I.inverse_radius(n, seed=3, noise=1e-2, dtype=np.float32, slices=7)
    W = I.inverse_radius(n, seed=3, noise=1e-2, dtype=np.float32)
    assert np.array_equal(S, W[:, :, :7])


def test_haar_factors_are_orthonormal_and_sign_normalised():
    rng = np.random.default_rng(0)
    U = I.haar(rng, 50, 7)
    assert np.abs(U.T @ U - np.eye(7)).max() < 1e-13
    # U = Q diag(sign(diag R)) for the QR of the same Gaussian draw
    Z = np.random.default_rng(0).standard_normal((50, 7))
    Q, R = np.linalg.qr(Z)
    assert np.allclose(U, Q * np.sign(np.diag(R)), rtol=0, atol=1e-14)
    assert np.allclose(U.T @ Z, np.triu(U.T @ Z), atol=1e-12)      # U^T Z = |R|-signed R
    assert np.all(np.diag(U.T @ Z) > 0)


def test_tucker_plus_noise_ranks_and_noise_modes():
    shape, ranks = [20, 18, 16], [4, 3, 2]
    X = I.tucker_plus_noise(shape, ranks, seed=7, noise=0.0, dtype=np.float64)
    for k in range(3):
        s = np.linalg.svd(_unfold(X, k), compute_uv=False)
        assert s[ranks[k]] < 1e-12 * s[0]            # exact multilinear rank
    Y = I.tucker_plus_noise(shape, ranks, seed=7, noise=1e-3, noise_mode="relative",
                            dtype=np.float64)
    assert abs(np.linalg.norm(Y - X) / np.linalg.norm(X) - 1e-3) < 1e-12
    Z1 = I.tucker_plus_noise(shape, ranks, seed=7, noise=1e-3, dtype=np.float32)
    Z2 = I.tucker_plus_noise(shape, ranks, seed=7, noise=1e-3, dtype=np.float32)
    assert np.array_equal(Z1, Z2)


@pytest.mark.parametrize("kind", ["slow", "fast", "sshape"])
def test_tensor_C_unfoldings_have_the_stated_spectrum(kind):
    """Section 5.1's tensor C = tendiag(v) x orthogonal factors: every
    unfolding's singular values are v (sorted), the closed form behind the
    printed errors of Table 5.3."""
    n = 30
    A = I.superdiagonal(n, kind, seed=14)
    v = np.sort(I.superdiagonal_values(n, kind))[::-1]
    for k in range(3):
        s = np.linalg.svd(_unfold(A, k), compute_uv=False)
        assert np.allclose(s, v, rtol=1e-10, atol=1e-14)


def test_tensor_B_sparsity_and_weights():
    n = 40
    A = I.sparse_rank_one_sum(n, seed=12)
    assert A.shape == (n, n, n) and A.min() >= 0.0
    # each term's vectors have ceil(0.05 n) nonzeros: a single term's support
    # is a nnz^3 block, so the tensor has at most n nnz^3 nonzeros
    nnz = math.ceil(0.05 * n)
    assert np.count_nonzero(A) <= n * nnz ** 3
    # the first 50 terms carry the factor gamma = 1000 (with n <= 50 every
    # term does; the same draws are made for any gamma)
    B = I.sparse_rank_one_sum(n, seed=12, gamma=1.0)
    assert np.allclose(A, 1000.0 * B, rtol=1e-12, atol=0)


def test_batch_specs_follow_the_recipe():
    specs = I.batch_specs(400, seed=4)
    orders = [len(s) for s, _, _ in specs]
    assert set(orders) == {3, 4}
    assert abs(orders.count(3) / len(orders) - 0.5) < 0.1
    for shape, ranks, _ in specs:
        assert all(32 <= n <= 160 for n in shape)
        assert all(1 <= r < n for r, n in zip(ranks, shape))
        assert all(r <= 16 for r in ranks)
        for m, r in enumerate(ranks):
            assert r <= np.prod([ranks[x] for x in range(len(ranks)) if x != m])
    assert I.batch_specs(5, seed=4) == specs[:5]


def test_serving_requests_follow_the_recipe():
    reqs = I.serving_requests(4000, seed=5)
    t = np.array([r["arrival"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(gaps.mean() * 200.0 - 1.0) < 0.05          # Poisson at 200 / s
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05     # exponential gaps
    sides = {64, 128, 256, 512, 768}
    for r in reqs:
        assert set(r["shape"]) <= sides
        assert r["q"] in (1, 2, 3) and r["kind"] in ("hilbert", "tucker")
        for m, rk in enumerate(r["ranks"]):
            assert 1 <= rk < r["shape"][m] and rk <= 40
            assert rk <= np.prod([r["ranks"][x] for x in range(3) if x != m])
    kinds = [r["kind"] for r in reqs]
    assert abs(kinds.count("hilbert") / len(kinds) - 0.5) < 0.05
