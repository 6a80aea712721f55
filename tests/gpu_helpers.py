"""Helpers for the GPU parity tests: run the CUDA library through the C ABI
on numpy inputs and bring the results back (layout and marshalling only)."""
import numpy as np

from paper_2506_04840_gb300 import api


def run_hosvd(A, r, s, q, st=True, seed=0, tag=0, shift=api.TK_SHIFT_PAPER,
              prec=api.TK_PREC_PLAIN, order=None, stats=True, workspace=False,
              omega=api.TK_OMEGA_GAUSS):
    import torch
    d = A.ndim
    dims = list(A.shape)
    dt = np.float64 if A.dtype == np.float64 else np.float32
    tdt = torch.float64 if dt == np.float64 else torch.float32
    Ad = api.to_device(A, dt)
    core = torch.empty(int(np.prod(r)), dtype=tdt, device="cuda")
    U = [torch.empty(dims[k] * r[k], dtype=tdt, device="cuda") for k in range(d)]
    ws = None
    opts = api.make_opts(d, q, s, seed=seed, tag=tag, shift=shift, prec=prec, order=order,
                         omega=omega)
    if workspace:
        nbytes = api.tucker_workspace_size(Ad, dims, r, opts, 1 if st else 0)
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        opts = api.make_opts(d, q, s, seed=seed, tag=tag, shift=shift, prec=prec, order=order,
                             workspace=ws, omega=omega)
    fn = api.tucker_rsthosvd if st else api.tucker_rthosvd
    info = fn(Ad, dims, r, opts, core, U, stats=stats)
    torch.cuda.synchronize()
    G = api.from_device(core, r)
    Us = [api.from_device(U[k], [dims[k], r[k]]) for k in range(d)]
    return G, Us, info


def gpu_error(A, G, Us):
    import torch
    dt = np.float64 if A.dtype == np.float64 else np.float32
    Ad = api.to_device(A, dt)
    Gd = api.to_device(G, dt)
    Ud = [api.to_device(U, dt) for U in Us]
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    api.tucker_error(Ad, list(A.shape), Gd, list(G.shape), Ud, out)
    torch.cuda.synchronize()
    return float(out.item())
