"""Batched problems (one launch per step kind over a work list, optionally
under a CUDA graph).

Every item's job blocks run the single-problem kernels' bodies with the same
block decomposition, so a batch must reproduce tucker_rsthosvd +
tucker_error on each item BITWISE, whatever the batch holds; and, through
them, the oracle (Algorithm 3 in FP64) within the FP32 path's tolerances.
"""
import numpy as np
import pytest

from oracle import tucker as T
from paper_2506_04840_gb300 import api
from paper_2506_04840_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _alloc(A, r, dtype):
    dims = list(A.shape)
    core = torch.full((int(np.prod(r)),), float("nan"), dtype=dtype, device="cuda")
    U = [torch.full((dims[k] * r[k],), float("nan"), dtype=dtype, device="cuda")
         for k in range(A.ndim)]
    rel = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    return core, U, rel


def _single(A, r, s, q, tag, rule=api.TK_SHIFT_PAPER, order=None):
    dt = torch.float64 if A.dtype == np.float64 else torch.float32
    Ad = api.to_device(A)
    core, U, rel = _alloc(A, r, dt)
    opts = api.make_opts(A.ndim, q, s, seed=0, tag=tag, shift=rule, order=order)
    api.tucker_rsthosvd(Ad, list(A.shape), r, opts, core, U)
    api.tucker_error(Ad, list(A.shape), core, r, U, rel)
    torch.cuda.synchronize()
    return core.cpu(), [u.cpu() for u in U], rel.cpu()


def _instances(count, seed, dtype=np.float32):
    out = []
    for i, (A, r) in enumerate(I.batch_instances(count, seed, lo=6, hi=36, rank_lo=2, rank_hi=6,
                                                 dtype=dtype)):
        out.append((A, r, 3, [0, 1, 2][i % 3]))
    return out


def _items(insts, order=None):
    dt = torch.float64 if insts[0][0].dtype == np.float64 else torch.float32
    keep, items = [], []
    for i, (A, r, s, q) in enumerate(insts):
        Ad = api.to_device(A)
        core, U, rel = _alloc(A, r, dt)
        keep.append((Ad, core, U, rel))
        items.append(api.make_item(Ad, list(A.shape), r, s, q, core, U, rel, seed=0, tag=i,
                                   order=order))
    return keep, items


def _run_batch(insts, use_graph, rule=api.TK_SHIFT_PAPER, runs=1, order=None):
    keep, items = _items(insts, order)
    h = api.tucker_batch_create(items, rule, use_graph)
    try:
        outs = []
        for _ in range(runs):
            api.tucker_batch_run(h)
            status, per = api.tucker_batch_wait(h, len(items))
            assert status == api.TK_OK and per == [0] * len(items)
            outs.append([(c.cpu().clone(), [u.cpu().clone() for u in U], rel.cpu().clone())
                         for (_, c, U, rel) in keep])
        launches, nbytes = api.tucker_batch_info(h)
    finally:
        api.tucker_batch_destroy(h)
    return outs, launches


def _same(a, b):
    ca, Ua, ra = a
    cb, Ub, rb = b
    return (torch.equal(ca, cb) and all(torch.equal(x, y) for x, y in zip(Ua, Ub))
            and torch.equal(ra, rb))


@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_equals_single_calls_bitwise(lib, use_graph):
    insts = _instances(14, seed=41)
    outs, launches = _run_batch(insts, use_graph, runs=2)
    assert _same_all(outs[0], outs[1])          # a replayed run is identical
    for i, (A, r, s, q) in enumerate(insts):
        assert _same(outs[0][i], _single(A, r, s, q, tag=i)), i
    # one launch per (schedule slot, position, step kind, tile class): far
    # fewer than the ~40 launches each item's own calls make
    assert launches < 14 * 8


def _same_all(xs, ys):
    return all(_same(a, b) for a, b in zip(xs, ys))


def test_batch_fp64_and_no_shift_bitwise(lib):
    insts = _instances(6, seed=5, dtype=np.float64)
    outs, _ = _run_batch(insts, True, rule=api.TK_SHIFT_NONE)
    for i, (A, r, s, q) in enumerate(insts):
        assert _same(outs[0][i], _single(A, r, s, q, tag=i, rule=api.TK_SHIFT_NONE)), i


def test_batch_matches_oracle(lib):
    """Each item against Algorithm 3 in FP64 on the same tensor and the same
    Omega (tag = item index): RE within 1e-6, factors orthonormal to 1e-6,
    leading separated subspaces within 1e-5."""
    insts = _instances(9, seed=77)
    outs, _ = _run_batch(insts, True)
    for i, (A, r, s, q) in enumerate(insts):
        core, U, rel = outs[0][i]
        G, Us, st = T.rsthosvd(A.astype(np.float64), r, [s] * A.ndim, q, seed=0, tag=i)
        re_o = T.rel_error(A.astype(np.float64), G, Us)
        assert abs(rel.item() - re_o) <= 1e-6, (i, rel.item(), re_o)
        for k in range(A.ndim):
            Ug = U[k].double().numpy().reshape((A.shape[k], r[k]), order="F")
            assert np.abs(Ug.T @ Ug - np.eye(r[k])).max() <= 1e-6
            sig = np.asarray(st[k]["sigma"])
            if q == 0:
                sig = sig ** 2      # sigma(A Omega) is linear in A: compare squared gaps
            j = T.separated_block(sig, r[k])
            if j:
                tol = 1e-5 if q else 1e-4   # sketch-only factors see FP32 noise at first order
                assert T.principal_sines(Ug[:, :j], Us[k][:, :j]).max() <= tol, (i, k)


def test_batch_many_items_share_the_grid(lib):
    """More job blocks than resident CTAs: the persistent grid strides over
    the work list; results still bitwise equal to the single calls."""
    insts = []
    for i, (A, r) in enumerate(I.batch_instances(40, seed=9, lo=20, hi=48, rank_lo=3,
                                                 rank_hi=8)):
        insts.append((A, r, 4, 2))
    outs, _ = _run_batch(insts, True)
    for i in (0, 7, 19, 39):
        A, r, s, q = insts[i]
        assert _same(outs[0][i], _single(A, r, s, q, tag=i)), i


def test_batch_row_split_products_bitwise(lib):
    """Items whose later modes have few columns and long rows: the FP32
    mode-major products split their rows over several CTAs (partials summed
    in a fixed order), in the batch exactly as in the single calls."""
    insts = []
    for i, shape in enumerate([(300, 40, 20), (256, 180, 30), (200, 150, 9, 12)]):
        r = [min(8, n - 1) for n in shape]
        A = I.tucker_plus_noise(list(shape), r, 50 + i, noise=1e-3, noise_mode="relative",
                                dtype=np.float32)
        insts.append((A, r, 4, 2))
    outs, _ = _run_batch(insts, True)
    for i, (A, r, s, q) in enumerate(insts):
        assert _same(outs[0][i], _single(A, r, s, q, tag=i)), i


def test_batch_long_mode_register_svd_bitwise(lib):
    """Items whose first mode has 600 or 1000 rows with l <= 32: the batch
    runs the long-mode register svd body, bitwise as the single calls."""
    insts = []
    for i, shape in enumerate([(600, 30, 20), (1000, 24, 16), (700, 20, 18)]):
        r = [12, 5, 4]
        A = I.tucker_plus_noise(list(shape), [14, 6, 5], 60 + i, noise=1e-3,
                                noise_mode="relative", dtype=np.float32)
        insts.append((A, r, 6, 2))
    outs, _ = _run_batch(insts, True)
    for i, (A, r, s, q) in enumerate(insts):
        assert _same(outs[0][i], _single(A, r, s, q, tag=i)), i


def _tucker_items(cases, seed0, dtype, s, q):
    insts = []
    for i, (shape, r) in enumerate(cases):
        core_r = [min(rk + 4, n - 1) for rk, n in zip(r, shape)]
        A = I.tucker_plus_noise(list(shape), core_r, seed0 + i, noise=1e-3,
                                noise_mode="relative", dtype=dtype)
        insts.append((A, r, s, q))
    return insts


def test_batch_tsqr_svd_bitwise(lib):
    """Items whose first mode is too long for a one-CTA svd: the batch runs
    the two-level TSQR chain (leaf QR, root QR + svd + shift update, leaf Q,
    sign) as four work-list launches, bitwise as the single calls.  Cases:
    register-resident leaves with 4 columns per warp (n = 1000, l = 60, two
    leaves) and 2 (n = 2000, l = 30, four leaves), and the shared-memory
    chain of an FP32 mode with l = 70 > 64; a one-CTA item shares the
    launches."""
    cases = [((1000, 60, 48), [50, 10, 8]), ((2000, 40, 30), [20, 8, 6]),
             ((600, 80, 72), [60, 10, 8]), ((40, 30, 20), [6, 5, 4])]
    insts = _tucker_items(cases, 80, np.float32, 10, 2)
    outs, _ = _run_batch(insts, True)
    for i, (A, r, s, q) in enumerate(insts):
        assert _same(outs[0][i], _single(A, r, s, q, tag=i)), i


def test_batch_fp64_tsqr_and_wide_one_cta_svd_bitwise(lib):
    """FP64 items: a 1000-row first mode takes the shared-memory TSQR chain,
    and a 300-row mode with l = 18 the one-CTA svd at 1024 threads (n l >=
    4096); q = 0 runs the sketch's svd only, q = 1 the power step's."""
    cases = [((1000, 300, 8), [20, 8, 4]), ((1000, 40, 30), [20, 8, 6])]
    for q in (0, 1):
        insts = _tucker_items(cases, 90, np.float64, 10, q)
        outs, _ = _run_batch(insts, True)
        for i, (A, r, s, qq) in enumerate(insts):
            assert _same(outs[0][i], _single(A, r, s, qq, tag=i)), (q, i)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_batch_descending_order_bitwise(lib, dtype):
    """Section 3.2's processing order (modes by non-increasing n_k) in a
    batch: unsorted shapes take strided views of the middle modes (no
    rotated layout), sorted ones keep the natural order; every item bitwise
    as the single call with the same order."""
    cases = [((30, 60, 45), [5, 7, 6]), ((20, 16, 36, 24), [4, 5, 6, 4]),
             ((50, 40, 30), [6, 5, 4]), ((24, 70, 18), [5, 8, 4])]
    insts = _tucker_items(cases, 100, dtype, 5, 2)
    outs, _ = _run_batch(insts, True, order="descending")
    for i, (A, r, s, q) in enumerate(insts):
        assert _same(outs[0][i], _single(A, r, s, q, tag=i, order="descending")), i


def test_tuned_split_counts_keep_batch_equal_to_single_calls(lib):
    """The split-K autotuner: tucker_tune_batch times the batch under each
    candidate scale of the heuristic split counts and stores the fastest
    candidate's counts per shape class.  With tuning on, the batch and the
    single calls read the same table, so every item stays bitwise equal to
    its single call; the stored choice is never slower than the heuristic
    in the tuner's own timing."""
    insts = _instances(14, seed=43)
    keep, items = _items(insts)
    api.tucker_tune_clear()
    try:
        best, base, shift = api.tucker_tune_batch(items)
        assert 0.0 < best <= base, (best, base)
        assert -1 <= shift <= 4
        assert api.tucker_tune_entries() > 0
        api.tucker_tune_enable(True)
        outs, _ = _run_batch(insts, True)
        for i, (A, r, s, q) in enumerate(insts):
            assert _same(outs[0][i], _single(A, r, s, q, tag=i)), i
    finally:
        api.tucker_tune_enable(False)
        api.tucker_tune_clear()
