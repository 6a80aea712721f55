"""The tcgen05 kind::tf32 behaviour the FP32 tensor-core contractions rely
on, checked on the GPU through tucker_debug_tf32_mma (one 128 x 64 x 32
product, four K = 8 instructions accumulating in tensor memory):

* FP32 operand bits below TF32 precision are dropped (truncation), so an
  operand x used as it stands acts as x_hi = x with its low 13 mantissa bits
  cleared, and x - x_hi is exactly the remainder the 3xTF32 split adds;
* products accumulate in FP32 rounded toward zero, within one instruction
  and between instructions (so accumulation chains are kept short and their
  partials summed in FP64 where a result needs full FP32 accuracy);
* A read from tensor memory gives the same product as A from shared memory.
Then a power step whose W = X^T Q runs in 3xTF32 on the tensor cores,
against FP64."""
import numpy as np
import pytest

from paper_2506_04840_gb300 import api

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _trunc(x):
    return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32)


def _inputs():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((128, 32)).astype(np.float32)
    B = rng.standard_normal((32, 64)).astype(np.float32)
    A[0:4] = 0
    A[0, 0], A[0, 8] = 1.0, 1.5 * 2.0 ** -24          # addend in the next instruction
    A[1, 0], A[1, 1] = 1.0, 1.5 * 2.0 ** -24          # addend in the same instruction
    A[2, 0], A[2, 8], A[2, 16], A[2, 24] = 1.0, 0.75 * 2.0 ** -24, 0.75 * 2.0 ** -24, 0.75 * 2.0 ** -24
    A[3, 0], A[3, 8] = -1.0, -1.5 * 2.0 ** -24
    B[:, 32:] = 1.0
    return A, B


@pytest.mark.parametrize("mode", [0, 1])
def test_tf32_operands_truncate_and_accumulation_rounds_toward_zero(lib, mode):
    A, B = _inputs()
    D = torch.full((128, 64), float("nan"), dtype=torch.float32, device="cuda")
    api.tucker_debug_tf32_mma(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), D, mode)
    D = D.cpu().numpy().astype(np.float64)
    ref = _trunc(A).astype(np.float64) @ _trunc(B).astype(np.float64)
    rows = slice(4, 128)
    scale = np.abs(ref[rows, :32]).max()
    # the truncated-operand model to FP32 accumulation accuracy; rounding the
    # operands to nearest instead would be ~1e-3 off
    assert np.abs(D[rows, :32] - ref[rows, :32]).max() <= 1e-6 * scale
    # 1 + 1.5 2^-24 rounds to nearest as 1 + 2^-23, toward zero as 1
    assert D[0, 40] == 1.0 and D[1, 40] == 1.0 and D[2, 40] == 1.0 and D[3, 40] == -1.0


def test_tf32_a_from_tensor_memory_equals_shared_memory(lib):
    A, B = _inputs()
    out = []
    for mode in (0, 1):
        D = torch.empty((128, 64), dtype=torch.float32, device="cuda")
        api.tucker_debug_tf32_mma(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), D, mode)
        out.append(D.cpu().numpy())
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("shape,l", [((1000, 1500), 60), ((256, 300), 17), ((36, 700), 32),
                                     ((1000, 1), 1)])
def test_tensor_core_power_step_matches_fp64(lib, shape, l):
    """One shifted power step (alpha = 0) on an FP32 matrix through
    tucker_shifted_power, whose W = X^T Q runs on the tensor cores for these
    shapes (rows a multiple of 4, l <= 64, ragged column tiles): the singular
    values of X (X^T Q) against FP64.  Tolerance from the arithmetic: W's
    accumulator takes 3 n/8 truncating (round toward zero) FP32 additions per
    entry, each off by less than one ulp toward zero; their sum acts as a
    relative shrink of W of order (3 n/8) u / 2 (~1e-5 at n = 1000, u =
    2^-24), so the singular values are checked to 5e-5 of the largest."""
    n, cols = shape
    rng = np.random.default_rng(11)
    X = rng.standard_normal((n, cols)).astype(np.float32)
    Q, _ = np.linalg.qr(rng.standard_normal((n, l)))
    Xd = api.to_device(X, np.float32)
    Qd = api.to_device(Q, np.float64)
    sig = torch.zeros(l, dtype=torch.float64, device="cuda")
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
    api.tucker_shifted_power(Xd, [n, cols], 0, l, 1, api.TK_SHIFT_NONE, Qd, sig, alpha)
    torch.cuda.synchronize()
    X64 = X.astype(np.float64)
    s_ref = np.linalg.svd(X64 @ (X64.T @ Q), compute_uv=False)
    s_gpu = sig.cpu().numpy()
    assert np.all(np.abs(s_gpu - s_ref) <= 5e-5 * s_ref[0]), np.abs(s_gpu - s_ref).max() / s_ref[0]
