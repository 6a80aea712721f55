"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances (stated once, used throughout):
* Omega: bit-exact.
* FP64 tensors: contraction error <= 1e-12 on the same scale, core <= 1e-12,
  |RE_gpu - RE_oracle| <= 1e-12, principal-angle sines <= 1e-9.
* FP32 tensors: error of a single contraction <= 1e-6 relative to
  || |X_(k)| |B| ||_F (the forward-error scale of a floating-point product),
  |RE_gpu - RE_oracle| <= 1e-6, sines <= 1e-5 on the well-separated leading
  block of each factor (gap (s_j^2 - s_{j+1}^2)/s_1^2 >= 1e-5 in the
  oracle's final Sigma), orthonormality ||U^T U - I||_max <= 1e-6.
"""
import numpy as np
import pytest

from oracle import omega as om
from oracle import tucker as T
from paper_2506_04840_gb300 import api
from paper_2506_04840_gb300 import inputs as I

from gpu_helpers import gpu_error, run_hosvd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def _sketch_err(got, X, k, l, seed, tag):
    """||Y_gpu - Y_oracle|| / || |X_(k)| |Omega| ||: the forward-error scale of
    a floating-point product (stable under cancellation in Y itself)."""
    Xk = T.unfold(np.asarray(X, dtype=np.float64), k)
    Om = om.omega_rows(k, 0, Xk.shape[1], l, seed=seed, tag=tag).astype(np.float64)
    want = Xk @ Om
    scale = np.linalg.norm(np.abs(Xk) @ np.abs(Om))
    return np.linalg.norm(got - want) / max(scale, 1e-300)


@pytest.mark.parametrize("k,row0,rows,l,seed,tag", [
    (0, 0, 1000, 60, 0, 0),
    (1, 12345, 777, 7, 0, 3),
    (2, (1 << 32) - 300, 600, 13, (1 << 40) + 3, 5),     # row index crosses 2^32
    (7, 5, 33, 1, 0xFFFFFFFFFFFFFFFF, (1 << 24) - 1),
    (3, 0, 257, 128, 99, 0),
])
def test_omega_is_bit_exact(lib, k, row0, rows, l, seed, tag):
    out = torch.empty(rows * l, dtype=torch.float32, device="cuda")
    api.tucker_debug_omega(k, row0, rows, l, seed, tag, out)
    got = out.cpu().numpy().reshape((rows, l), order="F")
    want = om.omega_rows(k, row0, rows, l, seed=seed, tag=tag)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


SHAPES = [(37, 29, 23), (9, 11, 7, 13), (130, 3, 70), (1, 40, 33)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_sketch_all_modes(lib, shape, dtype):
    rng = np.random.default_rng(1)
    A = np.asfortranarray(rng.standard_normal(shape).astype(dtype))
    Ad = api.to_device(A, dtype)
    for k in range(len(shape)):
        cols = int(np.prod(shape)) // shape[k]
        for l in sorted({1, min(5, cols), min(17, cols)}):
            Y = torch.empty(shape[k] * l, dtype=torch.float64, device="cuda")
            api.tucker_sketch(Ad, list(shape), k, l, 0, 2, Y)
            got = Y.cpu().numpy().reshape((shape[k], l), order="F")
            tol = 1e-12 if dtype == np.float64 else 1e-6
            assert _sketch_err(got, A, k, l, 0, 2) <= tol, (k, l)


def test_sketch_reads_bfloat16(lib):
    rng = np.random.default_rng(2)
    shape = (50, 41, 30)
    A = np.asfortranarray(rng.standard_normal(shape).astype(np.float32))
    Ad = api.to_device(A, np.float32)
    Ab = torch.empty(Ad.numel(), dtype=torch.int16, device="cuda")
    api.tucker_to_bf16(Ad, Ab)
    # the shadow is the oracle's round-to-nearest-even bfloat16
    bits = Ab.cpu().numpy().view(np.uint16).astype(np.uint32) << 16
    assert np.array_equal(bits.view(np.float32).astype(np.float64),
                          T.round_bf16(A).ravel(order="F"))
    for k in range(3):
        Y = torch.empty(shape[k] * 9, dtype=torch.float64, device="cuda")
        api.tucker_sketch(Ab, list(shape), k, 9, 0, 0, Y)
        got = Y.cpu().numpy().reshape((shape[k], 9), order="F")
        assert _sketch_err(got, T.round_bf16(A), k, 9, 0, 0) <= 1e-6


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("rule", [api.TK_SHIFT_PAPER, api.TK_SHIFT_NONE])
def test_shifted_power_steps(lib, dtype, rule):
    A = I.tucker_plus_noise([90, 70, 50], [8, 8, 8], seed=3, noise=1e-2, decay=0.9, dtype=dtype)
    k, l, q = 1, 14, 3
    orule = T.SHIFT_PAPER if rule == api.TK_SHIFT_PAPER else T.SHIFT_NONE
    Q0, _ = T.svd_econ(T.sketch(A, k, l))
    Qw, Sw, aw, _, _ = T.shifted_power(A, k, Q0, 0.0, q, orule)
    Ad = api.to_device(A, dtype)
    Qd = api.to_device(Q0, np.float64)
    sig = torch.zeros(l, dtype=torch.float64, device="cuda")
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
    api.tucker_shifted_power(Ad, list(A.shape), k, l, q, rule, Qd, sig, alpha)
    Qg = Qd.cpu().numpy().reshape((A.shape[k], l), order="F")
    Sg = sig.cpu().numpy()
    tol = 1e-12 if dtype == np.float64 else 1e-6
    j = T.separated_block(Sw, l)
    assert j >= 8
    assert np.max(np.abs(Sg[:j] - Sw[:j]) / Sw[:j]) <= (1e-10 if dtype == np.float64 else 1e-5)
    assert T.principal_sines(Qg[:, :j], Qw[:, :j]).max() <= (1e-9 if dtype == np.float64 else 1e-5)
    assert np.abs(Qg.T @ Qg - np.eye(l)).max() <= max(tol, 1e-13)
    if rule == api.TK_SHIFT_NONE:
        assert alpha.item() == 0.0
    else:
        assert abs(alpha.item() - aw) <= 1e-3 * max(abs(aw), 1e-30) + 1e-6 * Sw[0]


def _check_factors(Us_g, Us_w, stats_w, dtype):
    for k, (Ug, Uw) in enumerate(zip(Us_g, Us_w)):
        r = Uw.shape[1]
        Ug = np.asarray(Ug, dtype=np.float64)      # check in FP64, not in the data's FP32
        orth = np.abs(Ug.T @ Ug - np.eye(r)).max()
        assert orth <= (1e-13 if dtype == np.float64 else 1e-6), (k, orth)
        sig = np.asarray(stats_w[k]["sigma"])
        if not stats_w[k]["alpha"]:
            # q = 0: Sigma is sigma(A Omega), linear in A; square it so the gap
            # test sees the same scale as the power steps' sigma(A A^T Q)
            sig = sig ** 2
        j = T.separated_block(sig, r)
        if j > 0:
            s = T.principal_sines(Ug[:, :j], Uw[:, :j]).max()
            # sketch-only factors (q = 0) are not contracted by any power
            # step, so upstream FP32 differences reach them at first order
            tol = 1e-9 if dtype == np.float64 else (1e-5 if stats_w[k]["alpha"] else 1e-4)
            assert s <= tol, (k, j, s)


CASES = [
    # shape, ranks, s, q, seed of the input
    ((40, 36, 30), (6, 5, 4), 5, 2, 11),
    ((21, 18, 15, 12), (4, 3, 3, 2), 3, 1, 12),
    ((64, 20, 131), (10, 7, 12), 10, 3, 13),
    ((33, 33, 33), (32, 8, 8), 4, 2, 14),      # r = n - 1, l clamped at n
    ((40, 36, 30), (6, 5, 4), 5, 0, 15),       # q = 0: sketch only
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("st", [True, False])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_hosvd_matches_oracle(lib, case, st, dtype):
    shape, r, s, q, seed = case
    A = I.tucker_plus_noise(shape, [min(x + 2, n - 1) for x, n in zip(r, shape)], seed,
                            noise=1e-3, decay=0.85, dtype=dtype)
    f = T.rsthosvd if st else T.rthosvd
    Gw, Uw, sw = f(A, list(r), s, q)
    G, Us, info = run_hosvd(A, list(r), s, q, st=st)
    re_w = T.rel_error(A, Gw, Uw)
    re_g = T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= (1e-12 if dtype == np.float64 else 1e-6), (re_g, re_w)
    assert info["l"] == [x["l"] for x in sw]
    _check_factors(Us, Uw, sw, dtype)
    # core is A x_k U_k^T of the returned factors
    Gchk = A.astype(np.float64)
    for k in range(A.ndim) if not st else [0, 1, 2, 3][:A.ndim]:
        Gchk = T.mode_product(Gchk, Us[k].T.astype(np.float64), k)
    assert _rel(G, Gchk) <= (1e-12 if dtype == np.float64 else 1e-5)
    # shift history on the well-resolved modes matches the oracle
    if dtype == np.float64:
        for k in range(A.ndim):
            for t in range(q):
                aw = sw[k]["alpha"][t]
                assert abs(info["alpha"][k][t] - aw) <= 1e-8 * max(aw, 1e-300) + 1e-14


@pytest.mark.parametrize("rule", [api.TK_SHIFT_PAPER, api.TK_SHIFT_NONE])
def test_shift_rules_and_order(lib, rule):
    A = I.tucker_plus_noise([48, 40, 32], [6, 6, 6], 21, noise=1e-2, dtype=np.float64)
    orule = T.SHIFT_PAPER if rule == api.TK_SHIFT_PAPER else T.SHIFT_NONE
    order = [2, 0, 1]
    Gw, Uw, sw = T.rsthosvd(A, [5, 5, 5], 4, 3, rule=orule, order=order)
    G, Us, info = run_hosvd(A, [5, 5, 5], 4, 3, shift=rule, order=order)
    assert abs(T.rel_error(A, G, Us) - T.rel_error(A, Gw, Uw)) <= 1e-12
    assert info["order"] == order
    _check_factors(Us, Uw, sw, np.float64)


def test_config_hilbert_100_fp64_thosvd(lib):
    A = I.hilbert([100, 100, 100])
    Gw, Uw, sw = T.rthosvd(A, [10, 10, 10], 5, 1)
    G, Us, info = run_hosvd(A, [10, 10, 10], 5, 1, st=False)
    re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= 1e-12
    _check_factors(Us, Uw, sw, np.float64)
    assert abs(gpu_error(A, G, Us) - re_g) <= 1e-12


@pytest.mark.slow
def test_config_tucker_400_fp32_sthosvd(lib):
    A = I.tucker_plus_noise([400, 400, 400], [20, 20, 20], seed=2, noise=1e-4, decay=0.8,
                            dtype=np.float32)
    Gw, Uw, sw = T.rsthosvd(A, [20, 20, 20], 10, 2)
    G, Us, info = run_hosvd(A, [20, 20, 20], 10, 2)
    re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= 1e-6
    _check_factors(Us, Uw, sw, np.float32)
    assert abs(gpu_error(A, G, Us) - re_g) <= 1e-6


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_error_kernel(lib, dtype):
    rng = np.random.default_rng(5)
    A = np.asfortranarray(rng.standard_normal((23, 31, 19, 5)).astype(dtype))
    r = [4, 6, 3, 2]
    G = np.asfortranarray(rng.standard_normal(r).astype(dtype))
    Us = [np.linalg.qr(rng.standard_normal((n, k)))[0].astype(dtype) for n, k in zip(A.shape, r)]
    want = T.rel_error(A, G, Us)
    got = gpu_error(A, G, Us)
    assert abs(got - want) <= (1e-13 if dtype == np.float64 else 1e-6)
    # exact reconstruction gives zero
    Ax = np.asfortranarray(T.reconstruct(G, Us).astype(dtype))
    assert gpu_error(Ax, G, Us) <= (1e-14 if dtype == np.float64 else 1e-6)


def test_workspace_and_determinism(lib):
    A = I.tucker_plus_noise([70, 50, 40], [6, 6, 6], 31, noise=1e-3, dtype=np.float32)
    G1, U1, _ = run_hosvd(A, [5, 5, 5], 5, 2)
    G2, U2, _ = run_hosvd(A, [5, 5, 5], 5, 2, workspace=True)
    G3, U3, _ = run_hosvd(A, [5, 5, 5], 5, 2, stats=False)
    assert np.array_equal(G1, G2) and np.array_equal(G1, G3)
    for a, b, c in zip(U1, U2, U3):
        assert np.array_equal(a, b) and np.array_equal(a, c)


def test_thosvd_concurrent_modes_workspace_and_determinism(lib):
    """Algorithm 2 factors its modes concurrently (one stream each, one
    workspace set each): a caller workspace of tucker_workspace_size bytes
    and the internal allocation give bitwise the same results, run after
    run, and the precision form too."""
    A = I.tucker_plus_noise([70, 50, 40], [6, 6, 6], 33, noise=1e-3, dtype=np.float32)
    for prec in (api.TK_PREC_PLAIN, api.TK_PREC_BF16_POWER):
        G1, U1, _ = run_hosvd(A, [5, 5, 5], 5, 3, st=False, prec=prec)
        G2, U2, _ = run_hosvd(A, [5, 5, 5], 5, 3, st=False, prec=prec, workspace=True)
        G3, U3, _ = run_hosvd(A, [5, 5, 5], 5, 3, st=False, prec=prec, stats=False)
        assert np.array_equal(G1, G2) and np.array_equal(G1, G3)
        for a, b, c in zip(U1, U2, U3):
            assert np.array_equal(a, b) and np.array_equal(a, c)


def test_rank_exceeding_columns_is_rejected(lib):
    # mode 1 has 2*2 = 4 columns: l_1 = min(5 + 1, 6, 4) = 4 < r_1 = 5
    A = np.asfortranarray(np.ones((6, 2, 2), dtype=np.float32))
    with pytest.raises(api.TuckerError) as e:
        run_hosvd(A, [5, 1, 1], 1, 1)
    assert e.value.status == api.TK_EINVAL


def test_bf16_form_accuracy(lib):
    A = I.tucker_plus_noise([120, 110, 100], [12, 12, 12], 41, noise=1e-4, decay=0.85,
                            dtype=np.float32)
    r = [10, 10, 10]
    G, Us, _ = run_hosvd(A, r, 6, 3)
    Gb, Ub, _ = run_hosvd(A, r, 6, 3, prec=api.TK_PREC_BF16_POWER)
    re, reb = T.rel_error(A, G, Us), T.rel_error(A, Gb, Ub)
    assert reb <= 1.01 * re
    Gw, Uw, _ = T.rsthosvd(A, r, 6, 3, bf16_power=True)
    assert abs(reb - T.rel_error(A, Gw, Uw)) <= 1e-6


def _inverse_radius(shape, seed, noise):
    idx = np.indices(shape, dtype=np.float64) + 1.0
    A0 = 1.0 / np.sqrt((idx ** 2).sum(axis=0))
    rng = np.random.default_rng(seed)
    E = rng.standard_normal(shape) * noise * np.linalg.norm(A0.ravel()) / np.sqrt(A0.size)
    return np.asfortranarray((A0 + E).astype(np.float32))


@pytest.mark.parametrize("prec", [api.TK_PREC_PLAIN, api.TK_PREC_BF16_POWER])
def test_long_mode_matches_oracle(lib, prec):
    """A 1000-row mode with l = 60: the two-level TSQR svd path, and in the
    precision form the cluster-pair tensor-core pass, against the oracle."""
    A = _inverse_radius((1000, 60, 48), 3, 1e-6)
    r = [50, 20, 20]
    bf = prec == api.TK_PREC_BF16_POWER
    Gw, Uw, sw = T.rsthosvd(A, r, 10, 3, bf16_power=bf)
    G, Us, info = run_hosvd(A, r, 10, 3, prec=prec)
    re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= 1e-6, (re_g, re_w)
    # FP32 arithmetic costs a few percent of the error here; in the precision
    # form the FP32 step must also resolve the weak directions the bfloat16
    # steps left mixed with the leading ones (without the Ritz rotation of W
    # the error is several times the oracle's)
    assert re_g <= 1.04 * re_w, (re_g, re_w)
    if not bf:
        _check_factors(Us, Uw, sw, np.float32)


def test_precision_form_strided_layout_matches_oracle(lib):
    """Precision form with the modes taken in the order (2, 0, 1): the
    products, and the Ritz rotation of W before the FP32 step, walk the
    (P, l, S) layout with P > 1."""
    A = _inverse_radius((90, 70, 110), 5, 1e-6)
    r, order = [12, 10, 14], [2, 0, 1]
    Gw, Uw, _ = T.rsthosvd(A, r, 8, 3, order=order, bf16_power=True)
    G, Us, _ = run_hosvd(A, r, 8, 3, prec=api.TK_PREC_BF16_POWER, order=order)
    re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= 1e-2 * re_w + 1e-7, (re_g, re_w)
    for U in Us:
        assert np.abs(U.T.astype(np.float64) @ U - np.eye(U.shape[1])).max() <= 1e-5


def _run_pve(A, r, s, qmax, tol, stats=True, st_form=True):
    import torch
    d, dims = A.ndim, list(A.shape)
    Ad = api.to_device(A, np.float32)
    core = torch.empty(int(np.prod(r)), dtype=torch.float32, device="cuda")
    U = [torch.empty(dims[k] * r[k], dtype=torch.float32, device="cuda") for k in range(d)]
    opts = api.make_opts(d, qmax, s)
    fn = api.tucker_rsthosvd_pve if st_form else api.tucker_rthosvd_pve
    qs, st = fn(Ad, dims, r, opts, tol, core, U, stats=stats)
    torch.cuda.synchronize()
    G = api.from_device(core, r)
    Us = [api.from_device(U[k], [dims[k], r[k]]) for k in range(d)]
    return G, Us, qs, st


def test_pve_limits_equal_algorithm3_bitwise(lib):
    """Algorithm 4 with tol -> infinity is Algorithm 3 with q = 1, with tol = 0
    Algorithm 3 with q = q_max: bitwise the same results as tucker_rsthosvd."""
    A = I.tucker_plus_noise([70, 50, 40], [6, 6, 6], 31, noise=1e-3, dtype=np.float32)
    r, s, qmax = [5, 5, 5], 5, 4
    for tol, q in ((1e300, 1), (0.0, qmax)):
        G, Us, qs, _ = _run_pve(A, r, s, qmax, tol, stats=False)
        Gr, Ur, _ = run_hosvd(A, r, s, q, stats=False)
        assert qs == [q] * 3
        assert np.array_equal(G, Gr)
        for a, b in zip(Us, Ur):
            assert np.array_equal(a, b)


def test_pve_matches_oracle(lib):
    """A slowly decaying spectrum (Tucker 20^3 core, decay 0.97, 1% noise),
    r = 8, tol = 0.1, q_max = 10, where every mode runs 3 power steps: the
    per-mode power counts equal the oracle's (the stopping test is at least
    10% away from its threshold at every step, far outside FP32 noise) and
    the error matches."""
    A = I.tucker_plus_noise([60, 56, 48], [20, 20, 20], 7, noise=1e-2, decay=0.97,
                            noise_mode="relative", dtype=np.float32)
    r, s, qmax, tol = [8, 8, 8], 5, 10, 0.1
    Gw, Uw, qw, stw = T.rsthosvd_pve(A.astype(np.float64), r, s, qmax, tol)
    assert max(qw) >= 3
    # the oracle's decisions are not borderline
    for k in range(3):
        hist = stw[k]["sigma_hist"]
        prev = np.zeros_like(hist[0])
        for sig in hist:
            dmax = np.max(np.abs(sig[:r[k]] - prev[:r[k]]))
            thr = tol * sig[T.pve_threshold_index(r[k], len(sig))]
            assert abs(dmax - thr) > 0.1 * thr, (k, dmax, thr)
            prev = sig
    G, Us, qs, st = _run_pve(A, r, s, qmax, tol)
    assert qs == qw, (qs, qw)
    re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= 1e-6, (re_g, re_w)


def test_pve_full_size_tensor_C_reaches_the_optimum(lib):
    """The PVE workload at full size: tensor C of Section 5.1 (600^3, slow
    decay v_i = 1/i^2), r = 20, s = 10, tol = 0.5, q_max = 10.  The error is
    within 1% of the closed-form optimum sqrt(sum_{i>20} v_i^2 / sum v_i^2)
    (the paper prints 5.98e-3 for this case).  The first mode's count equals
    the oracle's: its test sits 45% below the threshold, far outside FP32
    noise.  The later modes' unfoldings have rank exactly 20 after the first
    truncation, so sigma(r+1) is rounding noise there and their counts are
    only checked to lie in [2, q_max]."""
    A = I.superdiagonal(600, "slow", seed=11, dtype=np.float32)
    v = I.superdiagonal_values(600, "slow")
    opt = float(np.sqrt(np.sum(v[20:] ** 2) / np.sum(v ** 2)))
    r, s, qmax, tol = [20, 20, 20], 10, 10, 0.5
    G, Us, qs, _ = _run_pve(A, r, s, qmax, tol, stats=False)
    re = T.rel_error(A, G, Us)
    assert opt * (1 - 1e-6) <= re <= 1.01 * opt, (re, opt, qs)
    assert all(2 <= q <= qmax for q in qs), qs
    _, _, qw, _ = T.rsthosvd_pve(A.astype(np.float64), r, s, qmax, tol)
    assert qs[0] == qw[0], (qs, qw)


def _robust_decisions(ratios, c=10.0):
    """Whether a mode's stopping decisions survive FP32 rounding.  ratios[t]
    is the oracle's max_i |sigma_t(i) - sigma_hat(i)| / threshold at step
    t+1; the first is ~sigma_1 / threshold.  The FP32 estimates carry
    errors of ~c u sigma_1 (u = 2^-24, backward-stable svd of Y), i.e. ~c u
    ratios[0] in units of the threshold, so a later decision is robust when
    its distance from 1 exceeds that."""
    u = 2.0 ** -24
    return all(abs(x - 1.0) > c * u * ratios[0] for x in ratios[1:])


def test_pve_full_size_tensor_B_counts_and_error(lib):
    """Algorithm 4 on tensor B of Section 5.1 at full size (600^3, r = 20,
    s = 10, tol = 0.5, q_max = 10), against the oracle's run stored by
    tests/golden/make_pve_tensor_B600.py: equal counts on every mode whose
    decisions are robust to FP32 rounding (modes 1 and 2; after two
    truncations mode 3's sigma(r+1) is ~1e-7 sigma_1, at the FP32 noise of
    the estimates, and its count is only checked to lie in [2, q_max]);
    RE within 1e-6 of the oracle's."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                     "pve_tensor_B600.json")))
    robust = [_robust_decisions(rk) for rk in g["test_ratios"]]
    assert robust[:2] == [True, True]
    A = I.sparse_rank_one_sum(600, g["seed"], dtype=np.float32)
    G, Us, qs, _ = _run_pve(A, g["r"], g["s"], g["q_max"], g["tol"], stats=False)
    for k in range(3):
        if robust[k]:
            assert qs[k] == g["q"][k], (k, qs, g["q"])
        assert 2 <= qs[k] <= g["q_max"], qs
    re = T.rel_error(A, G, Us)
    assert abs(re - g["re"]) <= 1e-6, (re, g["re"])


def test_thosvd_pve_limits_equal_algorithm2_bitwise(lib):
    """Algorithm 2 with the PVE counts: tol -> infinity is Algorithm 2 with
    q = 1 and tol = 0 with q = q_max, bitwise against tucker_rthosvd."""
    A = I.tucker_plus_noise([70, 50, 40], [6, 6, 6], 31, noise=1e-3, dtype=np.float32)
    r, s, qmax = [5, 5, 5], 5, 4
    for tol, q in ((1e300, 1), (0.0, qmax)):
        G, Us, qs, _ = _run_pve(A, r, s, qmax, tol, stats=False, st_form=False)
        Gr, Ur, _ = run_hosvd(A, r, s, q, st=False, stats=False)
        assert qs == [q] * 3
        assert np.array_equal(G, Gr)
        for a, b in zip(Us, Ur):
            assert np.array_equal(a, b)


def test_thosvd_pve_full_size_tensor_C_counts(lib):
    """Algorithm 2 with the PVE counts on tensor C at 600^3 (r = 20, s = 10,
    tol = 0.5, q_max = 10): every mode reads A, whose unfoldings all have
    the spectrum v^2 (sigma(r+1) ~ 5e-6 sigma_1); the counts agree with the
    oracle's on every mode whose decisions are robust to FP32 rounding
    (_robust_decisions; at least two of the three here) and lie in
    [2, q_max] on the others; RE within 1e-6."""
    A = I.superdiagonal(600, "slow", seed=11, dtype=np.float32)
    r, s, qmax, tol = [20, 20, 20], 10, 10, 0.5
    Gw, Uw, qw, stw = T.rthosvd_pve(A.astype(np.float64), r, s, qmax, tol)
    robust = []
    for k in range(3):
        prev = np.zeros_like(stw[k]["sigma_hist"][0])
        ratios = []
        for sig in stw[k]["sigma_hist"]:
            thr = tol * sig[T.pve_threshold_index(r[k], len(sig))]
            ratios.append(np.max(np.abs(sig[:r[k]] - prev[:r[k]])) / thr)
            prev = sig
        robust.append(_robust_decisions(ratios))
    assert sum(robust) >= 2, robust
    G, Us, qs, _ = _run_pve(A, r, s, qmax, tol, stats=False, st_form=False)
    for k in range(3):
        if robust[k]:
            assert qs[k] == qw[k], (k, qs, qw)
        assert 2 <= qs[k] <= qmax, qs
    re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= 1e-6, (re_g, re_w)


@pytest.mark.parametrize("shape,r,s", [
    ((1024, 40, 30), (20, 8, 8), 10),      # n = 1024: the last row of the long-mode svd
    ((600, 24, 20), (16, 6, 6), 16),       # l = 32, the widest it takes
    ((513, 12, 10), (1, 3, 3), 0),         # one row past the 512-row kernel, l = 1
])
def test_long_mode_register_svd_matches_oracle(lib, shape, r, s):
    """Modes of 513..1024 rows with l <= 32 take the one-CTA register svd
    with eight row chunks per lane: the first mode's factor against
    Algorithm 3's with the tolerances of test_hosvd_matches_oracle, and
    |RE_gpu - RE_oracle| <= 1e-6 for the whole decomposition (the later,
    short modes see the first factor's FP32 rounding through the shrink,
    at first order)."""
    A = I.tucker_plus_noise(list(shape), [min(x + 2, n - 1) for x, n in zip(r, shape)], 41,
                            noise=1e-3, decay=0.85, dtype=np.float32)
    Gw, Uw, sw = T.rsthosvd(A, list(r), s, 2)
    G, Us, info = run_hosvd(A, list(r), s, 2)
    re_w, re_g = T.rel_error(A, Gw, Uw), T.rel_error(A, G, Us)
    assert abs(re_g - re_w) <= 1e-6, (re_g, re_w)
    _check_factors(Us[:1], Uw[:1], sw[:1], np.float32)
    for U in Us[1:]:
        U = np.asarray(U, dtype=np.float64)
        assert np.abs(U.T @ U - np.eye(U.shape[1])).max() <= 1e-6


def test_descending_processing_order_matches_explicit_order(lib):
    """order[0] = TK_ORDER_DESCENDING processes the modes by non-increasing
    n_k (Section 3.2): bitwise the explicit permutation, reported in the
    stats, and the oracle's Algorithm 3 in that order; a shape already in
    that order keeps the natural (rotated-layout) path."""
    A = I.tucker_plus_noise([30, 44, 52], [7, 7, 7], 5, noise=1e-3, decay=0.85,
                            dtype=np.float32)
    r, s, q = [5, 5, 5], 4, 2
    G, Us, info = run_hosvd(A, r, s, q, order="descending")
    Ge, Ue, _ = run_hosvd(A, r, s, q, order=[2, 1, 0])
    assert info["order"][:3] == [2, 1, 0]
    assert np.array_equal(G, Ge) and all(np.array_equal(a, b) for a, b in zip(Us, Ue))
    Gw, Uw, _ = T.rsthosvd(A, r, s, q, order=T.descending_order(A.shape))
    assert abs(T.rel_error(A, G, Us) - T.rel_error(A, Gw, Uw)) <= 1e-6
    B = np.asfortranarray(np.transpose(A, (2, 1, 0)))     # 52 x 44 x 30
    G1, U1, i1 = run_hosvd(B, r, s, q, order="descending")
    G2, U2, _ = run_hosvd(B, r, s, q)
    assert i1["order"][:3] == [0, 1, 2]
    assert np.array_equal(G1, G2) and all(np.array_equal(a, b) for a, b in zip(U1, U2))
