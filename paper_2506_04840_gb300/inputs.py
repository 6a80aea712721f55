"""Seeded synthetic input tensors (host, numpy).

This module generates inputs only; it holds none of the Tucker method's
arithmetic, and both the CUDA path and the CPU oracle consume what it makes.
Tensors are returned as numpy arrays indexed (i_1, ..., i_d) in Fortran
(column-major, i_1 fastest) order, which is the layout the library reads.

Workloads (the paper's own test tensors are in Section 5.1; the sizes and
recipes of the benchmark workloads are restated here):
* ``hilbert``         a_{i_1..i_d} = 1/(i_1 + ... + i_d - d + 1), 1-based.
* ``tucker_plus_noise`` G x_1 U_1 ... x_d U_d + E, G i.i.d. N(0,1) optionally
                        scaled by decay^(i_1+...+i_d), U_k Haar-orthonormal,
                        E Gaussian with a stated per-entry level.
* ``inverse_radius``  a_ijk = (i^2 + j^2 + k^2)^(-1/2) + Gaussian noise.
* ``superdiagonal``   Section 5.1's tensor C = tendiag(v) x_n A_n with
                        A_n orthogonal (slow / fast / S-shaped v).
* ``sparse_rank_one_sum`` Section 5.1's tensor B: weighted sum of n
                        rank-one terms of sparse vectors.
* ``batch_instances`` uneven order-3/4 Tucker-plus-noise instances.
* ``serving_requests`` Poisson arrivals of mixed-size requests.
"""
import numpy as np


def haar(rng, n, r):
    """n x r matrix with Haar-distributed orthonormal columns (QR of a
    Gaussian with the signs of diag(R) moved into Q)."""
    Z = rng.standard_normal((n, r))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d


def _mode_mult(X, B, k):
    # plain tensor-times-matrix used to BUILD inputs (not the method)
    Xk = np.moveaxis(X, k, 0)
    shp = Xk.shape
    Y = B @ Xk.reshape(shp[0], -1)
    return np.moveaxis(Y.reshape((B.shape[0],) + shp[1:]), 0, k)


def hilbert(shape, dtype=np.float64):
    idx = np.indices(shape, dtype=np.float64)
    s = idx.sum(axis=0) + 1.0                  # (i_1-1)+...+(i_d-1) + 1
    return np.asfortranarray((1.0 / s).astype(dtype))


def tucker_plus_noise(shape, ranks, seed, noise=1e-4, decay=None, noise_mode="core",
                      dtype=np.float32):
    """A = G x_1 U_1 ... x_d U_d + E.

    noise_mode "core": E entries ~ N(0, (noise*||G||/sqrt(N))^2);
    noise_mode "relative": E scaled so that ||E|| = noise * ||X||.
    decay: if given, G entry (i_1..i_d) (1-based) is scaled by decay^(sum i).
    """
    rng = np.random.default_rng(seed)
    d = len(shape)
    G = rng.standard_normal(tuple(ranks))
    if decay is not None:
        idx = np.indices(ranks, dtype=np.float64).sum(axis=0) + d
        G = G * decay ** idx
    Us = [haar(rng, shape[k], ranks[k]) for k in range(d)]
    X = G
    for k in range(d):
        X = _mode_mult(X, Us[k], k)
    N = float(np.prod(shape))
    E = rng.standard_normal(tuple(shape))
    if noise_mode == "core":
        E *= noise * np.linalg.norm(G.ravel()) / np.sqrt(N)
    else:
        E *= noise * np.linalg.norm(X.ravel()) / np.linalg.norm(E.ravel())
    return np.asfortranarray((X + E).astype(dtype))


def inverse_radius(n, seed, noise=1e-6, dtype=np.float32, chunk=64, slices=None):
    """a_ijk = (i^2+j^2+k^2)^(-1/2) (1-based) + N(0, (noise*||A0||/sqrt(N))^2).

    Built slab by slab along the last mode so an n = 1000 cube (4 GB FP32)
    never needs an FP64 copy.  ``slices``: return only the first that many
    slices along the last mode (n x n x slices), bitwise equal to the same
    slices of the whole tensor (same noise level and draws).
    """
    rng = np.random.default_rng(seed)
    i = np.arange(1, n + 1, dtype=np.float64)
    sq = i * i
    ij = sq[:, None] + sq[None, :]
    # ||A0||^2 in FP64, exactly the same sum for every run
    norm2 = 0.0
    for k0 in range(0, n, chunk):
        kk = sq[k0:k0 + chunk]
        norm2 += float(np.sum(1.0 / (ij[:, :, None] + kk[None, None, :])))
    sigma = noise * np.sqrt(norm2) / np.sqrt(float(n) ** 3)
    m = n if slices is None else int(min(max(slices, 1), n))
    A = np.empty((n, n, m), dtype=dtype, order="F")
    for k0 in range(0, m, chunk):
        kk = sq[k0:k0 + chunk]
        slab = 1.0 / np.sqrt(ij[:, :, None] + kk[None, None, :])
        slab += sigma * rng.standard_normal(slab.shape)
        take = min(chunk, m - k0)
        A[:, :, k0:k0 + take] = slab[:, :, :take].astype(dtype)
    return A


def superdiagonal_values(n, kind):
    i = np.arange(1, n + 1, dtype=np.float64)
    if kind == "slow":
        return 1.0 / i ** 2
    if kind == "fast":
        return np.exp(-i / 7.0)
    if kind == "sshape":
        return 0.001 + 1.0 / (1.0 + np.exp(i - 29.0))
    raise ValueError(kind)


def superdiagonal(n, kind, seed, d=3, dtype=np.float64):
    """C = sum_i v_i a1_i o a2_i o a3_i, A_m = orthogonal basis of the column
    space of an n x n Gaussian matrix (Section 5.1, tensor C)."""
    rng = np.random.default_rng(seed)
    v = superdiagonal_values(n, kind)
    As = [haar(rng, n, n) for _ in range(d)]
    X = np.zeros((n,) * d)
    idx = np.arange(n)
    X[(idx,) * d] = v
    for k in range(d):
        X = _mode_mult(X, As[k], k)
    return np.asfortranarray(X.astype(dtype))


def sparse_rank_one_sum(n, seed, gamma=1000.0, heavy=50, density=0.05, power=2,
                        dtype=np.float64):
    """Tensor B of Section 5.1: sum_{i<=heavy} (gamma/i^power) x_i o y_i o z_i
    + sum_{heavy<i<=n} (1/i^power) x_i o y_i o z_i, n terms, x_i, y_i, z_i in
    R^n sparse.  Each vector has ceil(density * n) nonzeros at distinct
    random positions with values uniform on (0, 1) (the entries of a random
    sparse vector of that density).  power = 2: the weights that reproduce
    the errors the paper prints for B (its formula shows power 1)."""
    rng = np.random.default_rng(seed)
    nnz = int(np.ceil(density * n))
    X = np.zeros((n, n, n))
    for i in range(1, n + 1):
        w = (gamma if i <= heavy else 1.0) / float(i) ** power
        idx, val = [], []
        for _ in range(3):
            idx.append(np.sort(rng.choice(n, size=nnz, replace=False)))
            val.append(rng.random(nnz))
        X[np.ix_(*idx)] += w * np.einsum("a,b,c->abc", *val)
    return np.asfortranarray(X.astype(dtype))


def batch_specs(count, seed, lo=32, hi=160, rank_lo=4, rank_hi=16, max_elems=None):
    """Shapes, core ranks and content seeds of ``batch_instances``."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = 3 if rng.random() < 0.5 else 4
        shape = [int(rng.integers(lo, hi + 1)) for _ in range(d)]
        if max_elems is not None:
            while int(np.prod(shape)) > max_elems:
                m = int(np.argmax(shape))
                shape[m] = max(lo // 2, shape[m] // 2)
        ranks = [int(rng.integers(rank_lo, rank_hi + 1)) for _ in range(d)]
        for m in range(d):
            other = int(np.prod([ranks[x] for x in range(d) if x != m]))
            ranks[m] = min(ranks[m], other, shape[m] - 1)
        out.append((shape, ranks, int(rng.integers(0, 2**31 - 1))))
    return out


def tucker_plus_noise_device(shape, ranks, seed, noise=1e-3, dtype=None, device="cuda"):
    """Device-side G x_1 U_1 ... x_d U_d + E with ||E|| = noise * ||X||, made
    with torch's seeded generator (for workloads too large to build on the
    host).  Returns a flat torch tensor in column-major (i_1 fastest) order.
    The draws differ from ``tucker_plus_noise`` for the same seed."""
    import torch
    dtype = torch.float32 if dtype is None else dtype
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    d = len(shape)
    # torch is row-major: hold the tensor with reversed axes, so its flat
    # storage runs i_1 fastest
    X = torch.randn(tuple(reversed(ranks)), generator=g, device=device, dtype=torch.float64)
    for k in range(d):
        Z = torch.randn((shape[k], ranks[k]), generator=g, device=device, dtype=torch.float64)
        Q, R = torch.linalg.qr(Z)
        sgn = torch.sign(torch.diagonal(R))
        sgn[sgn == 0] = 1.0
        Uk = (Q * sgn).to(torch.float32)
        ax = d - 1 - k
        X = torch.movedim(torch.tensordot(Uk, X.to(torch.float32), dims=([1], [ax])), 0, ax)
    X = X.contiguous()
    E = torch.randn(X.shape, generator=g, device=device, dtype=torch.float32)
    E *= noise * torch.linalg.vector_norm(X) / torch.linalg.vector_norm(E)
    X += E
    return X.reshape(-1).to(dtype)


def hilbert_device(shape, dtype=None, device="cuda"):
    """Device-side Hilbert-type tensor 1/(i_1 + ... + i_d - d + 1), flat,
    column-major."""
    import torch
    dtype = torch.float32 if dtype is None else dtype
    s = torch.zeros((1,) * len(shape), dtype=torch.float64, device=device)
    for k, n in enumerate(reversed(shape)):
        ax = torch.arange(n, dtype=torch.float64, device=device)
        view = [1] * len(shape)
        view[k] = n
        s = s + ax.reshape(view)
    return (1.0 / (s + 1.0)).to(dtype).reshape(-1)


def batch_instances(count, seed, lo=32, hi=160, rank_lo=4, rank_hi=16, noise=1e-3,
                    dtype=np.float32, max_elems=None):
    """Uneven instances: order 3 or 4 (probability 1/2 each), sides uniform in
    [lo, hi], core ranks uniform in [rank_lo, rank_hi] clamped so that
    R_m <= prod of the other core ranks, N(0,1) core, Haar factors, noise
    with ||E|| = noise * ||X||.  Returns a list of (tensor, ranks)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = 3 if rng.random() < 0.5 else 4
        shape = [int(rng.integers(lo, hi + 1)) for _ in range(d)]
        if max_elems is not None:
            while int(np.prod(shape)) > max_elems:
                m = int(np.argmax(shape))
                shape[m] = max(lo // 2, shape[m] // 2)
        ranks = [int(rng.integers(rank_lo, rank_hi + 1)) for _ in range(d)]
        for m in range(d):
            other = int(np.prod([ranks[x] for x in range(d) if x != m]))
            ranks[m] = min(ranks[m], other, shape[m] - 1)
        sub = int(rng.integers(0, 2**31 - 1))
        A = tucker_plus_noise(shape, ranks, sub, noise=noise, noise_mode="relative",
                              dtype=dtype)
        out.append((A, ranks))
    return out


def serving_requests(count, seed, rate=200.0, sides=(64, 128, 256, 512, 768),
                     rank_lo=5, rank_hi=40, qs=(1, 2, 3)):
    """Request descriptors for the serving loop: Poisson arrival times at
    ``rate`` per second, per-mode sides uniform over ``sides``, content kind
    (Hilbert-type or random Tucker plus 1e-3 relative noise) 50/50, per-mode
    ranks uniform in [rank_lo, rank_hi] clamped below the side and to the
    product of the other ranks, q uniform over ``qs``.  Content is made by ``request_tensor``."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=count))
    reqs = []
    for i in range(count):
        shape = [int(rng.choice(sides)) for _ in range(3)]
        ranks = [int(min(rng.integers(rank_lo, rank_hi + 1), shape[m] - 1)) for m in range(3)]
        # a Tucker rank needs r_m <= prod of the other ranks (else the last
        # mode's unfolding has fewer columns than r_m)
        for m in range(3):
            ranks[m] = int(min(ranks[m], np.prod([ranks[x] for x in range(3) if x != m])))
        reqs.append(dict(id=i, arrival=float(t[i]), shape=shape, ranks=ranks,
                         q=int(rng.choice(qs)), kind="hilbert" if rng.random() < 0.5 else "tucker",
                         seed=int(rng.integers(0, 2**31 - 1))))
    return reqs


def request_tensor(req, dtype=np.float32):
    if req["kind"] == "hilbert":
        return hilbert(req["shape"], dtype=dtype)
    return tucker_plus_noise(req["shape"], req["ranks"], req["seed"], noise=1e-3,
                             noise_mode="relative", dtype=dtype)
