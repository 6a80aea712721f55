"""The C-ABI library builds, loads and exports every declared symbol; the
ctypes structures match the C header; host-side argument validation
rejects bad calls before any launch (CPU only, no kernel runs)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_2506_04840_gb300 import api

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^\s*[\w\s\*]*?\b(tucker_\w+)\s*\(", txt, re.M))
    return names


def test_library_exports_every_declared_symbol():
    lib = api.load()
    declared = _declared()
    assert "tucker_rsthosvd" in declared and len(declared) >= 9
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(api.SIGNATURES) | {"tucker_server_create"} | declared


def test_ctypes_structs_match_header():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "tucker.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(tk_tensor), sizeof(tk_opts), sizeof(tk_stats),
         offsetof(tk_opts, seed), offsetof(tk_opts, workspace), offsetof(tk_stats, sigma));
  printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(tk_item), offsetof(tk_item, q),
         offsetof(tk_item, core), offsetof(tk_item, rel_err), offsetof(tk_item, order),
         sizeof(tk_server_opts), sizeof(tk_completion), offsetof(tk_completion, done_s));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    want = [ctypes.sizeof(api.tk_tensor), ctypes.sizeof(api.tk_opts), ctypes.sizeof(api.tk_stats),
            api.tk_opts.seed.offset, api.tk_opts.workspace.offset, api.tk_stats.sigma.offset,
            ctypes.sizeof(api.tk_item), api.tk_item.q.offset, api.tk_item.core.offset,
            api.tk_item.rel_err.offset, api.tk_item.order.offset,
            ctypes.sizeof(api.tk_server_opts),
            ctypes.sizeof(api.tk_completion), api.tk_completion.done_s.offset]
    assert [int(x) for x in out] == want


def test_status_strings():
    lib = api.load()
    for s in range(8):
        assert lib.tucker_status_string(s).decode().startswith("TK_")


def _fake_tensor(dims, dtype=api.TK_F32):
    t = api.tk_tensor()
    t.d = len(dims)
    for k, n in enumerate(dims):
        t.n[k] = n
    t.dtype = dtype
    t.data = 0x1000          # never dereferenced: validation fails first
    return t


def test_argument_validation_before_launch():
    lib = api.load()
    o = api.make_opts(3, 2, 5)
    U = (ctypes.c_void_p * 3)(0x2000, 0x2000, 0x2000)
    A = _fake_tensor([10, 10, 10])
    bad_ranks = [(10, 2, 2), (0, 2, 2), (2, 2, 11)]        # r_k < n_k and r_k >= 1
    for r in bad_ranks:
        rr = (ctypes.c_int * 3)(*r)
        for fn in (lib.tucker_rsthosvd, lib.tucker_rthosvd):
            assert fn(ctypes.byref(A), rr, ctypes.byref(o), ctypes.c_void_p(0x3000), U, None,
                      None) == api.TK_EINVAL
    rr = (ctypes.c_int * 3)(2, 2, 2)
    # q out of range, tag too wide, bad order, BF16 form on FP64 data
    for field, val in (("q", -1), ("q", api.TK_MAX_Q + 1), ("tag", 1 << 24), ("shift", 7)):
        oo = api.make_opts(3, 2, 5)
        setattr(oo, field, val)
        assert lib.tucker_rsthosvd(ctypes.byref(A), rr, ctypes.byref(oo), ctypes.c_void_p(0x3000),
                                   U, None, None) == api.TK_EINVAL
    oo = api.make_opts(3, 2, 5, order=[0, 0, 1])
    assert lib.tucker_rsthosvd(ctypes.byref(A), rr, ctypes.byref(oo), ctypes.c_void_p(0x3000), U,
                               None, None) == api.TK_EINVAL
    oo = api.make_opts(3, 2, 5, prec=api.TK_PREC_BF16_POWER)
    A64 = _fake_tensor([10, 10, 10], api.TK_F64)
    assert lib.tucker_rsthosvd(ctypes.byref(A64), rr, ctypes.byref(oo), ctypes.c_void_p(0x3000),
                               U, None, None) == api.TK_EINVAL
    # null outputs
    assert lib.tucker_rsthosvd(ctypes.byref(A), rr, ctypes.byref(o), None, U, None,
                               None) == api.TK_EINVAL
    # sketch / power / error argument checks
    assert lib.tucker_sketch(ctypes.byref(A), 3, 4, 0, 0, ctypes.c_void_p(0x3000),
                             None) == api.TK_EINVAL
    assert lib.tucker_sketch(ctypes.byref(A), 0, api.TK_MAX_L + 1, 0, 0, ctypes.c_void_p(0x3000),
                             None) == api.TK_EINVAL
    assert lib.tucker_shifted_power(ctypes.byref(A), 0, 11, 1, 0, ctypes.c_void_p(0x3000),
                                    ctypes.c_void_p(0x3000), ctypes.c_void_p(0x3000),
                                    None) == api.TK_EINVAL
    assert lib.tucker_debug_omega(0, -1, 4, 4, 0, 0, ctypes.c_void_p(0x3000),
                                  None) == api.TK_EINVAL
    assert lib.tucker_to_bf16(None, 5, None, None) == api.TK_EINVAL
    # test matrix kinds: an unknown kind, and the debug writer's checks
    oo = api.make_opts(3, 2, 5, omega=7)
    assert lib.tucker_rsthosvd(ctypes.byref(A), rr, ctypes.byref(oo), ctypes.c_void_p(0x3000),
                               U, None, None) == api.TK_EINVAL
    n3 = (ctypes.c_int64 * 3)(10, 10, 10)
    for args in ((4, 3, n3, 0, 4), (api.TK_OMEGA_KR_GAUSS, 3, n3, 3, 4),
                 (api.TK_OMEGA_UNIFORM, 3, n3, 0, 0),
                 (api.TK_OMEGA_UNIFORM, 3, n3, 0, api.TK_MAX_L + 1),
                 (api.TK_OMEGA_UNIFORM, 0, n3, 0, 4),
                 (api.TK_OMEGA_UNIFORM, 3, (ctypes.c_int64 * 3)(10, 0, 10), 0, 4)):
        assert lib.tucker_debug_omega_matrix(*args, 0, 0, ctypes.c_void_p(0x3000),
                                             None) == api.TK_EINVAL, args
    assert lib.tucker_debug_omega_matrix(api.TK_OMEGA_UNIFORM, 3, n3, 0, 4, 0, 1 << 24,
                                         ctypes.c_void_p(0x3000), None) == api.TK_EINVAL
    # holistic variants: plain precision, r_k < n_k, outputs present
    for oo, rk in ((api.make_opts(3, 2, 5, prec=api.TK_PREC_BF16_POWER), rr),
                   (api.make_opts(3, 2, 5), (ctypes.c_int * 3)(5, 10, 5)),
                   (api.make_opts(3, 2, -1), rr)):
        assert lib.tucker_holistic(ctypes.byref(A), rk, ctypes.byref(oo), 1,
                                   ctypes.c_void_p(0x3000), U, None, None) == api.TK_EINVAL
    assert lib.tucker_holistic(ctypes.byref(A), rr, ctypes.byref(o), 1, None, U, None,
                               None) == api.TK_EINVAL
    # Algorithm 4: tol >= 0, q_max >= 1, plain precision only
    for tol, oo in ((-1.0, api.make_opts(3, 2, 5)), (0.5, api.make_opts(3, 0, 5)),
                    (0.5, api.make_opts(3, 2, 5, prec=api.TK_PREC_BF16_POWER))):
        for name in ("tucker_rsthosvd_pve", "tucker_rthosvd_pve"):
            assert getattr(lib, name)(ctypes.byref(A), rr, ctypes.byref(oo), tol,
                                      ctypes.c_void_p(0x3000), U, None, None,
                                      None) == api.TK_EINVAL
    bad = _fake_tensor([10, 0, 10])
    assert lib.tucker_error(ctypes.byref(bad), ctypes.c_void_p(0x3000), rr, U,
                            ctypes.c_void_p(0x3000), None) == api.TK_EINVAL


def test_workspace_size_is_host_only_and_monotone():
    lib = api.load()
    rr = (ctypes.c_int * 3)(5, 5, 5)
    small = lib.tucker_workspace_size(ctypes.byref(_fake_tensor([40, 40, 40])), rr,
                                      ctypes.byref(api.make_opts(3, 2, 5)), 1)
    big = lib.tucker_workspace_size(ctypes.byref(_fake_tensor([80, 80, 80])), rr,
                                    ctypes.byref(api.make_opts(3, 2, 5)), 1)
    assert 0 < small < big
    bf = lib.tucker_workspace_size(ctypes.byref(_fake_tensor([80, 80, 80])), rr,
                                   ctypes.byref(api.make_opts(3, 3, 5,
                                                              prec=api.TK_PREC_BF16_POWER)), 1)
    assert bf > big            # the bfloat16 shadow
    # Section 3.2's order is a valid request
    assert lib.tucker_workspace_size(ctypes.byref(_fake_tensor([40, 60, 80])), rr,
                                     ctypes.byref(api.make_opts(3, 2, 5, order="descending")),
                                     1) > 0
    # a stored test matrix needs W even without power steps; Khatri-Rao
    # factors add their scratch
    t = _fake_tensor([80, 80, 80])
    ws = {kind: lib.tucker_workspace_size(ctypes.byref(t), rr,
                                          ctypes.byref(api.make_opts(3, 0, 5, omega=kind)), 1)
          for kind in range(4)}
    assert ws[api.TK_OMEGA_UNIFORM] > ws[api.TK_OMEGA_GAUSS]
    assert ws[api.TK_OMEGA_KR_GAUSS] == ws[api.TK_OMEGA_KR_UNIFORM] > ws[api.TK_OMEGA_UNIFORM]
    # the holistic range finder keeps l_k columns: more than the plain call
    o2 = api.make_opts(3, 2, 5)
    for st in (0, 1):
        hw = lib.tucker_holistic_workspace_size(ctypes.byref(t), rr, ctypes.byref(o2), st)
        assert hw > lib.tucker_workspace_size(ctypes.byref(t), rr, ctypes.byref(o2), st) > 0
    assert lib.tucker_holistic_workspace_size(ctypes.byref(t), rr,
                                              ctypes.byref(api.make_opts(3, 2, -1)), 1) == 0
    bad = (ctypes.c_int * 3)(80, 5, 5)
    assert lib.tucker_workspace_size(ctypes.byref(_fake_tensor([80, 80, 80])), bad,
                                     ctypes.byref(api.make_opts(3, 2, 5)), 1) == 0


def test_batch_validation_before_allocation():
    """A batch with an invalid item is rejected on the host (nothing is
    allocated or launched): rank >= size, mixed dtypes, bad shift rule, an
    unknown processing order."""
    lib = api.load()

    def item(dims, r, dtype=api.TK_F32):
        it = api.tk_item()
        it.A = _fake_tensor(dims, dtype)
        for k in range(len(dims)):
            it.r[k] = r[k]
            it.s[k] = 2
            it.U[k] = 0x2000
        it.q = 1
        it.core = 0x3000
        return it

    h = ctypes.c_void_p()
    good = item([10, 9, 8], [3, 3, 3])
    bad_rank = item([10, 9, 8], [3, 9, 3])
    other = item([10, 9, 8], [3, 3, 3], api.TK_F64)
    bad_order = item([10, 9, 8], [3, 3, 3])
    bad_order.order = 1
    for items, rule in (([good, bad_rank], 0), ([good, other], 0), ([good], 7),
                        ([good, bad_order], 0)):
        arr = (api.tk_item * len(items))(*items)
        assert lib.tucker_batch_create(arr, len(items), rule, 0, ctypes.byref(h)) == api.TK_EINVAL
        assert not h.value
    assert lib.tucker_batch_create(None, 0, 0, 0, ctypes.byref(h)) == api.TK_EINVAL
