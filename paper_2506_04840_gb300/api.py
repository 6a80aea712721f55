"""Thin Python binding of the C ABI in ``include/tucker.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA
library.  Device buffers are torch CUDA tensors used as plain memory; a
tensor's data is the column-major (i_1 fastest) flattening of the
n_1 x ... x n_d array and its sizes are passed explicitly.  Functions carry
the C names; each raises ``TuckerError`` on a non-OK status.  There is no
fallback: if ``libtucker.so`` cannot be loaded, ``load`` raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

TK_MAX_D = 8
TK_MAX_Q = 32
TK_MAX_L = 128

TK_OK, TK_EINVAL, TK_ENOMEM, TK_ECUDA, TK_EBREAKDOWN, TK_ETIMEOUT, TK_ENOTIMPL, TK_EWORKSPACE = range(8)
TK_F64, TK_F32, TK_BF16 = 0, 1, 2
TK_SHIFT_PAPER, TK_SHIFT_NONE = 0, 1
TK_PREC_PLAIN, TK_PREC_BF16_POWER = 0, 1
TK_OMEGA_GAUSS, TK_OMEGA_UNIFORM, TK_OMEGA_KR_GAUSS, TK_OMEGA_KR_UNIFORM = 0, 1, 2, 3
TK_ORDER_DESCENDING = -2   # make_opts(order="descending"): modes by non-increasing n_k

c_int, c_int64, c_uint64, c_uint32, c_double = (ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                                 ctypes.c_uint32, ctypes.c_double)
c_void_p, c_size_t = ctypes.c_void_p, ctypes.c_size_t


class tk_tensor(ctypes.Structure):
    _fields_ = [("d", c_int), ("n", c_int64 * TK_MAX_D), ("dtype", c_int), ("data", c_void_p)]


class tk_opts(ctypes.Structure):
    _fields_ = [("q", c_int), ("s", c_int * TK_MAX_D), ("seed", c_uint64), ("tag", c_uint32),
                ("shift", c_int), ("prec", c_int), ("order", c_int * TK_MAX_D),
                ("workspace", c_void_p), ("workspace_bytes", c_size_t), ("omega", c_int)]


class tk_stats(ctypes.Structure):
    _fields_ = [("d", c_int), ("q", c_int), ("l", c_int * TK_MAX_D), ("order", c_int * TK_MAX_D),
                ("alpha", (c_double * TK_MAX_Q) * TK_MAX_D),
                ("sigma_l", (c_double * TK_MAX_Q) * TK_MAX_D),
                ("sigma", (c_double * TK_MAX_L) * TK_MAX_D)]


TK_K_NAMES = ["sketch", "power_w", "power_y", "power_fused", "small_svd", "ttm", "error",
              "convert", "ritz"]


class tk_profile(ctypes.Structure):
    _fields_ = [("launches", c_int64 * len(TK_K_NAMES)), ("ms", c_double * len(TK_K_NAMES)),
                ("bytes", c_double * len(TK_K_NAMES)), ("flops", c_double * len(TK_K_NAMES)),
                ("kernels", c_int64)]


class tk_item(ctypes.Structure):
    _fields_ = [("A", tk_tensor), ("r", c_int * TK_MAX_D), ("s", c_int * TK_MAX_D), ("q", c_int),
                ("seed", c_uint64), ("tag", c_uint32), ("core", c_void_p),
                ("U", c_void_p * TK_MAX_D), ("rel_err", c_void_p), ("order", c_int)]


class tk_server_opts(ctypes.Structure):
    _fields_ = [("pool_bytes", c_size_t), ("max_active", c_int), ("rule", c_int)]


class tk_completion(ctypes.Structure):
    _fields_ = [("id", c_uint64), ("status", c_int), ("submit_s", c_double),
                ("admit_s", c_double), ("done_s", c_double)]


class TuckerError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__("%s: %s" % (what, _LIB.tucker_status_string(status).decode()
                                     if _LIB is not None else status))


_LIB = None

# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "tucker_status_string": (ctypes.c_char_p, [c_int]),
    "tucker_workspace_size": (c_size_t, [ctypes.POINTER(tk_tensor), ctypes.POINTER(c_int),
                                         ctypes.POINTER(tk_opts), c_int]),
    "tucker_debug_omega_matrix": (c_int, [c_int, c_int, ctypes.POINTER(c_int64), c_int, c_int,
                                          c_uint64, c_uint32, c_void_p, c_void_p]),
    "tucker_debug_omega": (c_int, [c_int, c_int64, c_int64, c_int, c_uint64, c_uint32, c_void_p,
                                   c_void_p]),
    "tucker_debug_tf32_mma": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "tucker_sketch": (c_int, [ctypes.POINTER(tk_tensor), c_int, c_int, c_uint64, c_uint32,
                              c_void_p, c_void_p]),
    "tucker_shifted_power": (c_int, [ctypes.POINTER(tk_tensor), c_int, c_int, c_int, c_int,
                                     c_void_p, c_void_p, c_void_p, c_void_p]),
    "tucker_rthosvd": (c_int, [ctypes.POINTER(tk_tensor), ctypes.POINTER(c_int),
                               ctypes.POINTER(tk_opts), c_void_p, ctypes.POINTER(c_void_p),
                               ctypes.POINTER(tk_stats), c_void_p]),
    "tucker_rsthosvd": (c_int, [ctypes.POINTER(tk_tensor), ctypes.POINTER(c_int),
                                ctypes.POINTER(tk_opts), c_void_p, ctypes.POINTER(c_void_p),
                                ctypes.POINTER(tk_stats), c_void_p]),
    "tucker_rsthosvd_pve": (c_int, [ctypes.POINTER(tk_tensor), ctypes.POINTER(c_int),
                                    ctypes.POINTER(tk_opts), c_double, c_void_p,
                                    ctypes.POINTER(c_void_p), ctypes.POINTER(c_int),
                                    ctypes.POINTER(tk_stats), c_void_p]),
    "tucker_holistic": (c_int, [ctypes.POINTER(tk_tensor), ctypes.POINTER(c_int),
                                ctypes.POINTER(tk_opts), c_int, c_void_p, ctypes.POINTER(c_void_p),
                                ctypes.POINTER(tk_stats), c_void_p]),
    "tucker_holistic_workspace_size": (c_size_t, [ctypes.POINTER(tk_tensor), ctypes.POINTER(c_int),
                                                  ctypes.POINTER(tk_opts), c_int]),
    "tucker_rthosvd_pve": (c_int, [ctypes.POINTER(tk_tensor), ctypes.POINTER(c_int),
                                   ctypes.POINTER(tk_opts), c_double, c_void_p,
                                   ctypes.POINTER(c_void_p), ctypes.POINTER(c_int),
                                   ctypes.POINTER(tk_stats), c_void_p]),
    "tucker_error": (c_int, [ctypes.POINTER(tk_tensor), c_void_p, ctypes.POINTER(c_int),
                             ctypes.POINTER(c_void_p), c_void_p, c_void_p]),
    "tucker_to_bf16": (c_int, [c_void_p, c_int64, c_void_p, c_void_p]),
    "tucker_batch_create": (c_int, [ctypes.POINTER(tk_item), c_int, c_int, c_int,
                                    ctypes.POINTER(c_void_p)]),
    "tucker_batch_run": (c_int, [c_void_p, c_void_p]),
    "tucker_batch_wait": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "tucker_batch_info": (c_int, [c_void_p, ctypes.POINTER(c_int64), ctypes.POINTER(c_size_t)]),
    "tucker_batch_destroy": (c_int, [c_void_p]),
    "tucker_batch_rsthosvd": (c_int, [ctypes.POINTER(tk_item), c_int, c_int, c_void_p]),
    "tucker_server_create": (c_int, [ctypes.POINTER(tk_server_opts), ctypes.POINTER(c_void_p)]),
    "tucker_server_submit": (c_int, [c_void_p, ctypes.POINTER(tk_item),
                                     ctypes.POINTER(c_uint64)]),
    "tucker_server_poll": (c_int, [c_void_p, ctypes.POINTER(tk_completion), c_int]),
    "tucker_server_drain": (c_int, [c_void_p, c_double]),
    "tucker_server_clock": (c_double, [c_void_p]),
    "tucker_server_destroy": (c_int, [c_void_p]),
    "tucker_tune_enable": (c_int, [c_int]),
    "tucker_tune_clear": (c_int, []),
    "tucker_tune_entries": (c_int, [ctypes.POINTER(c_int)]),
    "tucker_tune_save": (c_int, [ctypes.c_char_p]),
    "tucker_tune_load": (c_int, [ctypes.c_char_p]),
    "tucker_tune_batch": (c_int, [ctypes.POINTER(tk_item), c_int, c_int, c_void_p,
                                  ctypes.POINTER(c_double), ctypes.POINTER(c_double),
                                  ctypes.POINTER(c_int)]),
    "tucker_profile_enable": (c_int, [c_int]),
    "tucker_profile_read": (c_int, [ctypes.POINTER(tk_profile)]),
}


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libtucker.so (building it in-tree first if needed)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError("libtucker.so is missing; run paper_2506_04840_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _check(status, what):
    if status != TK_OK:
        raise TuckerError(status, what)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(int(t.data_ptr()))


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dtype_code(t):
    import torch
    if t.dtype == torch.float64:
        return TK_F64
    if t.dtype == torch.float32:
        return TK_F32
    if t.dtype in (torch.bfloat16, torch.int16, torch.uint16):
        return TK_BF16
    raise TypeError("unsupported dtype %s" % t.dtype)


def tensor_desc(data, dims, dtype=None):
    """tk_tensor for a device buffer holding the column-major data."""
    t = tk_tensor()
    t.d = len(dims)
    for k, n in enumerate(dims):
        t.n[k] = int(n)
    t.dtype = _dtype_code(data) if dtype is None else dtype
    t.data = int(data.data_ptr())
    return t


def make_opts(d, q, s, seed=0, tag=0, shift=TK_SHIFT_PAPER, prec=TK_PREC_PLAIN, order=None,
              workspace=None, omega=TK_OMEGA_GAUSS):
    o = tk_opts()
    o.q = int(q)
    svals = [s] * d if np.isscalar(s) else list(s)
    for k in range(d):
        o.s[k] = int(svals[k])
    o.seed = int(seed)
    o.tag = int(tag)
    o.shift = int(shift)
    o.prec = int(prec)
    o.omega = int(omega)
    if order is None:
        o.order[0] = -1
    elif isinstance(order, str):
        if order != "descending":
            raise ValueError(order)
        o.order[0] = TK_ORDER_DESCENDING
    else:
        for k, m in enumerate(order):
            o.order[k] = int(m)
    if workspace is not None:
        o.workspace = int(workspace.data_ptr())
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def _ranks(r):
    arr = (c_int * len(r))()
    for k, x in enumerate(r):
        arr[k] = int(x)
    return arr


def _ptr_array(ts):
    arr = (c_void_p * len(ts))()
    for k, t in enumerate(ts):
        arr[k] = int(t.data_ptr())
    return arr


def tucker_status_string(status):
    return load().tucker_status_string(int(status)).decode()


def tucker_workspace_size(A, dims, r, opts, st):
    desc = tensor_desc(A, dims)
    return int(load().tucker_workspace_size(ctypes.byref(desc), _ranks(r), ctypes.byref(opts),
                                            int(st)))


def tucker_debug_omega(k, row0, rows, l, seed, tag, out, stream=None):
    _check(load().tucker_debug_omega(k, row0, rows, l, seed, tag, _ptr(out), _stream(stream)),
           "tucker_debug_omega")


def tucker_debug_omega_matrix(kind, dims, k, l, seed, tag, out, stream=None):
    n = (c_int64 * len(dims))(*[int(x) for x in dims])
    _check(load().tucker_debug_omega_matrix(int(kind), len(dims), n, k, l, seed, tag, _ptr(out),
                                            _stream(stream)), "tucker_debug_omega_matrix")


def tucker_sketch(A, dims, k, l, seed, tag, Y, stream=None):
    desc = tensor_desc(A, dims)
    _check(load().tucker_sketch(ctypes.byref(desc), k, l, seed, tag, _ptr(Y), _stream(stream)),
           "tucker_sketch")


def tucker_shifted_power(A, dims, k, l, q, rule, Q, sigma, alpha, stream=None):
    desc = tensor_desc(A, dims)
    _check(load().tucker_shifted_power(ctypes.byref(desc), k, l, q, rule, _ptr(Q), _ptr(sigma),
                                       _ptr(alpha), _stream(stream)), "tucker_shifted_power")


def _stats_dict(st):
    d = st.d
    return dict(l=[st.l[k] for k in range(d)], order=[st.order[k] for k in range(d)],
                alpha=[[st.alpha[k][t] for t in range(st.q)] for k in range(d)],
                sigma_l=[[st.sigma_l[k][t] for t in range(st.q)] for k in range(d)],
                sigma=[[st.sigma[k][i] for i in range(st.l[k])] for k in range(d)])


def _hosvd(fn, A, dims, r, opts, core, U, stats, stream):
    desc = tensor_desc(A, dims)
    st = tk_stats() if stats else None
    _check(getattr(load(), fn)(ctypes.byref(desc), _ranks(r), ctypes.byref(opts), _ptr(core),
                               _ptr_array(U), ctypes.byref(st) if st is not None else None,
                               _stream(stream)), fn)
    return _stats_dict(st) if st is not None else None


def tucker_rthosvd(A, dims, r, opts, core, U, stats=False, stream=None):
    return _hosvd("tucker_rthosvd", A, dims, r, opts, core, U, stats, stream)


def tucker_rsthosvd(A, dims, r, opts, core, U, stats=False, stream=None):
    return _hosvd("tucker_rsthosvd", A, dims, r, opts, core, U, stats, stream)


def _pve(name, A, dims, r, opts, tol, core, U, stats, stream):
    desc = tensor_desc(A, dims)
    st = tk_stats() if stats else None
    qs = (c_int * len(dims))()
    _check(getattr(load(), name)(ctypes.byref(desc), _ranks(r), ctypes.byref(opts), float(tol),
                                 _ptr(core), _ptr_array(U), qs,
                                 ctypes.byref(st) if st is not None else None, _stream(stream)),
           name)
    return [int(x) for x in qs], (_stats_dict(st) if st is not None else None)


def tucker_rsthosvd_pve(A, dims, r, opts, tol, core, U, stats=False, stream=None):
    """Algorithm 4 (opts.q = q_max).  Returns (q_k list, stats dict or None)."""
    return _pve("tucker_rsthosvd_pve", A, dims, r, opts, tol, core, U, stats, stream)


def tucker_rthosvd_pve(A, dims, r, opts, tol, core, U, stats=False, stream=None):
    """Algorithm 2 with Algorithm 4's counts.  Returns (q_k list, stats or None)."""
    return _pve("tucker_rthosvd_pve", A, dims, r, opts, tol, core, U, stats, stream)


def tucker_holistic(A, dims, r, opts, st, core, U, stats=False, stream=None):
    """Algorithms A.2 / B.1 (holistic range finding, then ST-HOSVD of the
    small tensor).  Returns the stats dict or None."""
    desc = tensor_desc(A, dims)
    s = tk_stats() if stats else None
    _check(load().tucker_holistic(ctypes.byref(desc), _ranks(r), ctypes.byref(opts), int(st),
                                  _ptr(core), _ptr_array(U),
                                  ctypes.byref(s) if s is not None else None, _stream(stream)),
           "tucker_holistic")
    return _stats_dict(s) if s is not None else None


def tucker_holistic_workspace_size(A, dims, r, opts, st):
    desc = tensor_desc(A, dims)
    return int(load().tucker_holistic_workspace_size(ctypes.byref(desc), _ranks(r),
                                                     ctypes.byref(opts), int(st)))


def tucker_error(A, dims, core, r, U, rel_err, stream=None):
    desc = tensor_desc(A, dims)
    _check(load().tucker_error(ctypes.byref(desc), _ptr(core), _ranks(r), _ptr_array(U),
                               _ptr(rel_err), _stream(stream)), "tucker_error")


def tucker_debug_tf32_mma(A, B, D, mode, stream=None):
    _check(load().tucker_debug_tf32_mma(_ptr(A), _ptr(B), _ptr(D), int(mode), _stream(stream)),
           "tucker_debug_tf32_mma")


def tucker_to_bf16(x, out, stream=None):
    _check(load().tucker_to_bf16(_ptr(x), int(x.numel()), _ptr(out), _stream(stream)),
           "tucker_to_bf16")


def make_item(A, dims, r, s, q, core, U, rel_err=None, seed=0, tag=0, order=None):
    """tk_item for one problem of a batch or one serving request (order:
    None = natural, "descending" = Section 3.2's order)."""
    it = tk_item()
    it.A = tensor_desc(A, dims)
    d = len(dims)
    svals = [s] * d if np.isscalar(s) else list(s)
    for k in range(d):
        it.r[k] = int(r[k])
        it.s[k] = int(svals[k])
        it.U[k] = int(U[k].data_ptr())
    it.q = int(q)
    it.seed = int(seed)
    it.tag = int(tag)
    it.core = int(core.data_ptr())
    it.rel_err = None if rel_err is None else int(rel_err.data_ptr())
    if order is None:
        it.order = 0
    elif order == "descending":
        it.order = TK_ORDER_DESCENDING
    else:
        raise ValueError(order)
    return it


def _items(items):
    arr = (tk_item * len(items))()
    for i, it in enumerate(items):
        arr[i] = it
    return arr


def tucker_batch_create(items, rule=TK_SHIFT_PAPER, use_graph=True):
    h = c_void_p()
    _check(load().tucker_batch_create(_items(items), len(items), int(rule), 1 if use_graph else 0,
                                      ctypes.byref(h)), "tucker_batch_create")
    return h


def tucker_tune_enable(on=True):
    _check(load().tucker_tune_enable(1 if on else 0), "tucker_tune_enable")


def tucker_tune_clear():
    _check(load().tucker_tune_clear(), "tucker_tune_clear")


def tucker_tune_entries():
    n = c_int()
    _check(load().tucker_tune_entries(ctypes.byref(n)), "tucker_tune_entries")
    return int(n.value)


def tucker_tune_save(path):
    _check(load().tucker_tune_save(str(path).encode()), "tucker_tune_save")


def tucker_tune_load(path):
    """Returns the status (TK_EINVAL for a missing or malformed file)."""
    return load().tucker_tune_load(str(path).encode())


def tucker_tune_batch(items, rule=TK_SHIFT_PAPER, stream=None):
    """Returns (best ms, heuristic ms, best shift)."""
    b, h, sh = c_double(), c_double(), c_int()
    _check(load().tucker_tune_batch(_items(items), len(items), int(rule), _stream(stream),
                                    ctypes.byref(b), ctypes.byref(h), ctypes.byref(sh)),
           "tucker_tune_batch")
    return float(b.value), float(h.value), int(sh.value)


def tucker_batch_run(h, stream=None):
    _check(load().tucker_batch_run(h, _stream(stream)), "tucker_batch_run")


def tucker_batch_wait(h, count):
    st = (c_int * count)()
    status = load().tucker_batch_wait(h, st)
    return status, [int(x) for x in st]


def tucker_batch_info(h):
    n, b = c_int64(), c_size_t()
    _check(load().tucker_batch_info(h, ctypes.byref(n), ctypes.byref(b)), "tucker_batch_info")
    return int(n.value), int(b.value)


def tucker_batch_destroy(h):
    _check(load().tucker_batch_destroy(h), "tucker_batch_destroy")


def tucker_batch_rsthosvd(items, rule=TK_SHIFT_PAPER, stream=None):
    _check(load().tucker_batch_rsthosvd(_items(items), len(items), int(rule), _stream(stream)),
           "tucker_batch_rsthosvd")


def tucker_server_create(pool_bytes=0, max_active=0, rule=TK_SHIFT_PAPER):
    o = tk_server_opts()
    o.pool_bytes = int(pool_bytes)
    o.max_active = int(max_active)
    o.rule = int(rule)
    h = c_void_p()
    _check(load().tucker_server_create(ctypes.byref(o), ctypes.byref(h)), "tucker_server_create")
    return h


def tucker_server_submit(h, item):
    rid = c_uint64()
    _check(load().tucker_server_submit(h, ctypes.byref(item), ctypes.byref(rid)),
           "tucker_server_submit")
    return int(rid.value)


def tucker_server_poll(h, max_n=256):
    arr = (tk_completion * max_n)()
    n = load().tucker_server_poll(h, arr, max_n)
    return [dict(id=int(c.id), status=int(c.status), submit_s=c.submit_s, admit_s=c.admit_s,
                 done_s=c.done_s) for c in arr[:n]]


def tucker_server_drain(h, timeout_s=60.0):
    _check(load().tucker_server_drain(h, float(timeout_s)), "tucker_server_drain")


def tucker_server_clock(h):
    return float(load().tucker_server_clock(h))


def tucker_server_destroy(h):
    _check(load().tucker_server_destroy(h), "tucker_server_destroy")


def tucker_profile_enable(on):
    _check(load().tucker_profile_enable(1 if on else 0), "tucker_profile_enable")


def tucker_profile_read():
    p = tk_profile()
    _check(load().tucker_profile_read(ctypes.byref(p)), "tucker_profile_read")
    kinds = {}
    for i, name in enumerate(TK_K_NAMES):
        kinds[name] = dict(launches=int(p.launches[i]), ms=float(p.ms[i]),
                           bytes=float(p.bytes[i]), flops=float(p.flops[i]))
    return dict(kinds=kinds, kernels=int(p.kernels))


# ---- host helpers (layout only) --------------------------------------------
def to_device(arr, dtype=None, device="cuda"):
    """Upload a numpy array as its column-major flattening."""
    import torch
    a = np.asarray(arr)
    if dtype is not None:
        a = a.astype(dtype)
    flat = np.ascontiguousarray(a.ravel(order="F"))
    return torch.from_numpy(flat).to(device)


def from_device(t, dims):
    """Download a column-major device buffer as a numpy array of shape dims."""
    return t.detach().cpu().numpy().reshape(tuple(dims), order="F")
