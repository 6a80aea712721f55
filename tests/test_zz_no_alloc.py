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


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_noalloc_sketch_matches_sketch_twice(lib, dtype):
    fn = _noalloc(lib)
    rng = np.random.default_rng(17)
    calls = [((300, 40, 50), 0, 60, 5, 1),   # first call uses a large part of the scratch
             ((23, 31, 17), 1, 9, 0, 2)]      # second call: smaller, stale data left behind
    for shape, k, l, seed, tag in calls:
        A = np.asfortranarray(rng.standard_normal(shape).astype(dtype))
        Ad = api.to_device(A, dtype)
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
        assert err <= tol * _scale(Ad, list(shape), k, l, seed, tag, dtype)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    fn = _noalloc(lib)
    shape = (40000, 2, 1)                          # 40000 * 64 * 4 B > 8 MiB
    Ad = torch.zeros(int(np.prod(shape)), dtype=torch.float32, device="cuda")
    desc = api.tensor_desc(Ad, list(shape))
    Y = torch.zeros(shape[0] * 64, dtype=torch.float64, device="cuda")
    st = fn(ctypes.byref(desc), 0, 64, 0, 0, ctypes.c_void_p(Y.data_ptr()), None)
    assert st == api.TK_EWORKSPACE
