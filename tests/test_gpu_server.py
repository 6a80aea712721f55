"""Serving loop: continuous batching of Tucker requests.

Requests that arrive while others run are admitted as memory and slots free
up and share ticks (one batched launch per step kind) with them.  A
request's blocks do the single-problem work in the same order, so its
result is bitwise the same alone, in any mix, and as a direct
tucker_rsthosvd + tucker_error call.
"""
import numpy as np
import pytest

from paper_2506_04840_gb300 import api
from paper_2506_04840_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


class Req:
    def __init__(self, A, r, s, q, tag):
        self.A, self.r, self.s, self.q, self.tag = A, r, s, q, tag
        self.Ad = api.to_device(A)
        dt = self.Ad.dtype
        self.core = torch.full((int(np.prod(r)),), float("nan"), dtype=dt, device="cuda")
        self.U = [torch.full((A.shape[k] * r[k],), float("nan"), dtype=dt, device="cuda")
                  for k in range(A.ndim)]
        self.rel = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")

    def item(self):
        return api.make_item(self.Ad, list(self.A.shape), self.r, self.s, self.q, self.core,
                             self.U, self.rel, seed=0, tag=self.tag)

    def result(self):
        return self.core.cpu(), [u.cpu() for u in self.U], self.rel.cpu()


def _single(A, r, s, q, tag):
    q_ = Req(A, r, s, q, tag)
    opts = api.make_opts(A.ndim, q, s, seed=0, tag=tag)
    api.tucker_rsthosvd(q_.Ad, list(A.shape), r, opts, q_.core, q_.U)
    api.tucker_error(q_.Ad, list(A.shape), q_.core, r, q_.U, q_.rel)
    torch.cuda.synchronize()
    return q_.result()


def _same(a, b):
    return (torch.equal(a[0], b[0]) and all(torch.equal(x, y) for x, y in zip(a[1], b[1]))
            and torch.equal(a[2], b[2]))


def _mix(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        shape = [int(rng.integers(8, 48)) for _ in range(3)]
        r = [int(min(rng.integers(2, 8), shape[m] - 1)) for m in range(3)]
        if rng.random() < 0.5:
            A = I.hilbert(shape, dtype=np.float32)
        else:
            A = I.tucker_plus_noise(shape, r, int(rng.integers(1 << 30)), noise=1e-3,
                                    noise_mode="relative", dtype=np.float32)
        out.append((A, r, 4, int(rng.integers(1, 4))))
    return out


def test_server_alone_vs_mix_bitwise(lib):
    A = I.tucker_plus_noise([40, 36, 30], [5, 4, 4], 3, noise=1e-3, noise_mode="relative",
                            dtype=np.float32)
    srv = api.tucker_server_create(pool_bytes=512 << 20, max_active=64)
    try:
        alone = Req(A, [5, 4, 4], 4, 2, tag=7)
        api.tucker_server_submit(srv, alone.item())
        api.tucker_server_drain(srv, 60.0)
        comps = api.tucker_server_poll(srv)
        assert len(comps) == 1 and comps[0]["status"] == 0
        mix = [Req(*m, tag=100 + i) for i, m in enumerate(_mix(24, 5))]
        again = Req(A, [5, 4, 4], 4, 2, tag=7)
        ids = {}
        for i, m in enumerate(mix):
            ids[api.tucker_server_submit(srv, m.item())] = m
            if i == 11:
                ids[api.tucker_server_submit(srv, again.item())] = again
        api.tucker_server_drain(srv, 120.0)
        comps = api.tucker_server_poll(srv, 1024)
        assert sorted(c["id"] for c in comps) == sorted(ids)
        for c in comps:
            assert c["status"] == 0
            assert c["submit_s"] <= c["admit_s"] <= c["done_s"]
    finally:
        api.tucker_server_destroy(srv)
    torch.cuda.synchronize()
    ra, rb = alone.result(), again.result()
    assert _same(ra, rb)
    assert _same(ra, _single(A, [5, 4, 4], 4, 2, tag=7))
    for m in mix[::5]:
        assert _same(m.result(), _single(m.A, m.r, m.s, m.q, m.tag))


def test_server_admission_waits_for_memory(lib):
    """A pool that holds two requests' workspaces: the others queue, are
    admitted as earlier ones finish, and all complete correctly."""
    shape, r = [60, 50, 40], [6, 5, 5]
    A = I.tucker_plus_noise(shape, r, 8, noise=1e-3, noise_mode="relative", dtype=np.float32)
    Ad = api.to_device(A)
    opts = api.make_opts(3, 2, 4)
    ws = api.tucker_workspace_size(Ad, shape, r, opts, 1)
    # a request's pool share is at least the single call's workspace
    srv = api.tucker_server_create(pool_bytes=int(2.4 * ws), max_active=16)
    reqs = [Req(A, r, 4, 2, tag=i) for i in range(6)]
    try:
        for q_ in reqs:
            api.tucker_server_submit(srv, q_.item())
        api.tucker_server_drain(srv, 120.0)
        comps = api.tucker_server_poll(srv, 64)
    finally:
        api.tucker_server_destroy(srv)
    assert len(comps) == 6 and all(c["status"] == 0 for c in comps)
    # never more than two requests held memory at once
    for c in comps:
        live = sum(1 for o in comps if o["admit_s"] <= c["admit_s"] < o["done_s"])
        assert live <= 2
    assert max(c["admit_s"] for c in comps) >= min(c["done_s"] for c in comps)
    ref = _single(A, r, 4, 2, tag=3)
    assert _same(reqs[3].result(), ref)


def test_server_rejects_bad_requests(lib):
    A = I.hilbert([20, 18, 16], dtype=np.float32)
    srv = api.tucker_server_create(pool_bytes=1 << 20, max_active=4)
    try:
        bad = Req(A, [5, 18, 3], 2, 1, tag=0)         # r_2 = n_2
        with pytest.raises(api.TuckerError) as e:
            api.tucker_server_submit(srv, bad.item())
        assert e.value.status == api.TK_EINVAL
        big = I.hilbert([200, 200, 200], dtype=np.float32)
        huge = Req(big, [5, 5, 5], 2, 1, tag=0)       # workspace larger than the pool
        with pytest.raises(api.TuckerError) as e:
            api.tucker_server_submit(srv, huge.item())
        assert e.value.status == api.TK_ENOMEM
    finally:
        api.tucker_server_destroy(srv)
