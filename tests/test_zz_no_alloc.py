"""tucker_sketch_noalloc: the sketch without device allocation, for callers
that cannot let the library allocate device memory (fixed memory budgets,
host applications that own the allocator).  Checked through the C ABI
against tucker_sketch on two calls in a row, at the contraction tolerance the
parity tests use (1e-6 of || |A_(k)| |Omega| || for FP32, 1e-12 for FP64).

Collected last on purpose: it runs after every other test in a stop-at-first-
failure run, and it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_2506_04840_gb300 import api

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(lib):
    fn = lib.tucker_sketch_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.POINTER(api.tk_tensor), ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                   ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p]
    return fn


def _scale(Ad, dims, k, l, seed, tag, dtype):
    """|| |A_(k)| |Omega_k| ||_F computed on the device in FP64."""
    d = len(dims)
    X = Ad.double().reshape(list(reversed(dims))).permute(*reversed(range(d)))  # (n_1..n_d)
    perm = [k] + [m for m in range(d) if m != k]
    Xk = X.permute(*perm).permute(0, *reversed(range(1, d))).reshape(dims[k], -1)
    rows = Xk.shape[1]
    om = torch.empty(rows * l, dtype=torch.float32, device="cuda")
    api.tucker_debug_omega(k, 0, rows, l, seed, tag, om)
    Om = om.double().reshape(l, rows).t()
    return float(torch.linalg.norm(Xk.abs() @ Om.abs()))


def _run_twice(lib, dtype, calls, bf16=False):
    fn = _noalloc(lib)
    rng = np.random.default_rng(17)
    for shape, k, l, seed, tag in calls:
        A = np.asfortranarray(rng.standard_normal(shape).astype(np.float32 if bf16 else dtype))
        Ad = api.to_device(A, np.float32 if bf16 else dtype)
        if bf16:
            Ad = Ad.to(torch.bfloat16)
        desc = api.tensor_desc(Ad, list(shape))
        Y_ref = torch.empty(shape[k] * l, dtype=torch.float64, device="cuda")
        api.tucker_sketch(Ad, list(shape), k, l, seed, tag, Y_ref)
        Y = torch.full((shape[k] * l,), float("nan"), dtype=torch.float64, device="cuda")
        st = fn(ctypes.byref(desc), k, l, seed, tag, ctypes.c_void_p(Y.data_ptr()),
                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert st == api.TK_OK, api.tucker_status_string(st)
        torch.cuda.synchronize()
        tol = 1e-12 if dtype == np.float64 else 1e-6
        err = float(torch.linalg.norm(Y - Y_ref))
        assert np.isfinite(err)
        assert err <= tol * _scale(Ad.float() if bf16 else Ad, list(shape), k, l, seed, tag,
                                   dtype)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_noalloc_sketch_matches_sketch_twice(lib, dtype):
    _run_twice(lib, dtype, [((300, 40, 50), 0, 60, 5, 1),   # a large part of the scratch
                            ((23, 31, 17), 1, 9, 0, 2)])     # smaller, stale data left behind


def test_noalloc_sketch_bfloat16_tensor(lib):
    # a bfloat16 tensor takes the strided kernel with FP32 partials
    _run_twice(lib, np.float32, [((64, 33, 20), 1, 40, 3, 4), ((50, 21, 30), 2, 17, 3, 5)],
               bf16=True)


def test_noalloc_sketch_with_fewer_splits_than_the_plain_call(lib):
    # mode 0 of an FP32 tensor with 8000 rows and l = 60: each split's partial
    # block is 8000 x 64 x 4 B = 2 MiB, so the scratch holds 4 of the ~15
    # splits tucker_sketch uses, and the FP32 register-tiled kernel runs with
    # a reduced split count; then a small call reuses the scratch
    _run_twice(lib, np.float32, [((8000, 40, 50), 0, 60, 9, 6), ((30, 20, 10), 0, 12, 9, 7)])


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    fn = _noalloc(lib)
    shape = (40000, 2, 1)                          # 40000 * 64 * 4 B > 8 MiB
    Ad = torch.zeros(int(np.prod(shape)), dtype=torch.float32, device="cuda")
    desc = api.tensor_desc(Ad, list(shape))
    Y = torch.zeros(shape[0] * 64, dtype=torch.float64, device="cuda")
    st = fn(ctypes.byref(desc), 0, 64, 0, 0, ctypes.c_void_p(Y.data_ptr()), None)
    assert st == api.TK_EWORKSPACE
