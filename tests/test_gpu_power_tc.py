"""The fused bfloat16 power step on tcgen05 (mode-major tensors, n % 8 == 0).

It computes Y = X_(k)(X_(k)^T Q) from a bfloat16 tensor with bfloat16
operands (Q and the intermediate W are rounded to bfloat16, products
accumulate in FP32).  Against the FP64 oracle on the same bfloat16 tensor the
error of Y is bounded by a few bfloat16 roundings (2^-9 relative) of
||X||^2 ||Q||, so:
* singular values after the step agree to 1e-2 sigma_1;
* the leading subspace agrees to 5e-2 where it is separated by a gap of at
  least 0.3 sigma_1 (a wrong operand layout gives sines near 1);
* repeated calls are bitwise identical (fixed reduction order).
"""
import numpy as np
import pytest

from oracle import tucker as T
from paper_2506_04840_gb300 import api
from paper_2506_04840_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _bf16_device(A):
    Ad = api.to_device(A, np.float32)
    Ab = torch.empty(Ad.numel(), dtype=torch.int16, device="cuda")
    api.tucker_to_bf16(Ad, Ab)
    return Ab


@pytest.mark.parametrize("shape,rank,l", [
    ((1000, 40, 50), 8, 60),      # the 1000-row mode, two c-parts, ragged column count
    ((400, 30, 30), 8, 30),       # one c-part
    ((136, 37, 11), 6, 16),       # ragged 128-row tile, small l
    ((256, 64, 33), 8, 70),       # three c-parts
    ((520, 33, 29), 6, 20),       # cluster pair, odd tile count, ragged second half
    ((768, 50, 21), 8, 64),       # cluster pair, full 64-wide Q
])
@pytest.mark.parametrize("rule", [api.TK_SHIFT_NONE, api.TK_SHIFT_PAPER])
def test_fused_bf16_power_step(lib, shape, rank, l, rule):
    A = I.tucker_plus_noise(list(shape), [rank] * 3, seed=sum(shape), noise=1e-3, decay=0.9,
                            dtype=np.float32)
    Ab = T.round_bf16(A)
    k, q = 0, 2
    orule = T.SHIFT_PAPER if rule == api.TK_SHIFT_PAPER else T.SHIFT_NONE
    Q0, _ = T.svd_econ(T.sketch(Ab, k, l))
    Qw, Sw, aw, _, _ = T.shifted_power(Ab, k, Q0, 0.0, q, orule)
    Abd = _bf16_device(A)
    outs = []
    for _ in range(2):
        Qd = api.to_device(Q0, np.float64)
        sig = torch.zeros(l, dtype=torch.float64, device="cuda")
        alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
        api.tucker_shifted_power(Abd, list(shape), k, l, q, rule, Qd, sig, alpha)
        outs.append((Qd.cpu().numpy().reshape((shape[0], l), order="F"), sig.cpu().numpy(),
                     alpha.item()))
    (Qg, Sg, ag), (Qg2, Sg2, ag2) = outs
    assert np.array_equal(Qg, Qg2) and np.array_equal(Sg, Sg2) and ag == ag2
    assert np.max(np.abs(Sg - Sw)) <= 1e-2 * Sw[0]
    gaps = (Sw[:-1] - Sw[1:]) / Sw[0]
    j = int(np.argmax(gaps[:rank] >= 0.3)) + 1 if np.any(gaps[:rank] >= 0.3) else 0
    j = max([i + 1 for i in range(rank) if gaps[i] >= 0.3] or [0])
    if j:
        assert T.principal_sines(Qg[:, :j], Qw[:, :j]).max() <= 5e-2
    assert np.abs(Qg.T @ Qg - np.eye(l)).max() <= 1e-5


def test_fused_pass_is_used_and_timed(lib):
    """The bfloat16 power step on a mode-major tensor launches the fused kernel."""
    shape, l = (512, 64, 40), 32
    A = I.tucker_plus_noise(list(shape), [6] * 3, seed=3, noise=1e-3, dtype=np.float32)
    Abd = _bf16_device(A)
    Q0, _ = T.svd_econ(T.sketch(T.round_bf16(A), 0, l))
    Qd = api.to_device(Q0, np.float64)
    sig = torch.zeros(l, dtype=torch.float64, device="cuda")
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
    api.tucker_profile_enable(True)
    api.tucker_shifted_power(Abd, list(shape), 0, l, 1, api.TK_SHIFT_PAPER, Qd, sig, alpha)
    prof = api.tucker_profile_read()
    api.tucker_profile_enable(False)
    assert prof["kinds"]["power_fused"]["launches"] == 1
    assert prof["kinds"]["power_w"]["launches"] == 0


@pytest.mark.parametrize("shape,l", [((1000, 60, 48), 60), ((1000, 40, 50), 60),
                                     ((768, 50, 21), 64), ((520, 33, 29), 20)])
def test_fused_step_matches_rounded_emulation(lib, shape, l):
    """One fused step against its exact emulation: Y = X (bf16(X^T bf16(Q)))
    in FP64 on the bfloat16 tensor, so only the FP32 accumulation order
    differs: singular values to 1e-4 relative, every direction with
    sigma > 1e-3 sigma_1 to sines 1e-3."""
    A = I.tucker_plus_noise(list(shape), [8] * 3, seed=sum(shape) + 1, noise=1e-2, decay=0.9,
                            dtype=np.float32)
    Ab = T.round_bf16(A)
    Q0, _ = T.svd_econ(T.sketch(Ab, 0, l))
    Xk = T.unfold(Ab, 0)
    W = T.round_bf16(Xk.T @ T.round_bf16(Q0))
    Qw, Sw = T.svd_econ(Xk @ W)
    Abd = _bf16_device(A)
    Qd = api.to_device(Q0, np.float64)
    sig = torch.zeros(l, dtype=torch.float64, device="cuda")
    alpha = torch.zeros(1, dtype=torch.float64, device="cuda")
    api.tucker_shifted_power(Abd, list(shape), 0, l, 1, api.TK_SHIFT_NONE, Qd, sig, alpha)
    Sg = sig.cpu().numpy()
    Qg = Qd.cpu().numpy().reshape((shape[0], l), order="F")
    assert np.max(np.abs(Sg - Sw) / Sw[0]) <= 1e-4, np.max(np.abs(Sg - Sw) / Sw[0])
    j = int(np.sum(Sw > 1e-3 * Sw[0]))
    assert T.principal_sines(Qg[:, :j], Qw[:, :j]).max() <= 1e-3
