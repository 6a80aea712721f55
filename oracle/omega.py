"""Oracle Gaussian test matrix Omega_k (Algorithm 2, step "draw a standard
Gaussian matrix"; Algorithm 3, same step; Section 2 defines a standard
Gaussian matrix as one with i.i.d. N(0,1) entries).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper draws Omega_k with MATLAB's ``randn``, which cannot be reproduced,
so the library fixes a counter-based definition and both the oracle (here,
numpy) and the CUDA kernels implement it independently:

* Bits: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
  as easy as 1, 2, 3", SC'11).  Round: (c0,c1,c2,c3) <- (hi(M1*c2)^c1^k0,
  lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0)) with M0 = 0xD2511F53,
  M1 = 0xCD9E8D57; the key is bumped by (0x9E3779B9, 0xBB67AE85) between
  rounds; ten rounds.
* Key = (seed mod 2^32, seed >> 32).
* Entry (j, c) of Omega_k (row j = column index of the mode-k unfolding in
  Kolda order, 0-based; column c in [0, l)) comes from the counter
  (j mod 2^32, j >> 32, c >> 2, (k & 0xff) | (tag << 8)), output word pair
  (w0, w1) for c mod 4 in {0, 1} and (w2, w3) for c mod 4 in {2, 3}.
* Box-Muller on a word pair (wa, wb):
  u1 = (2*(wa >> 9) + 1) * 2^-24  (in (0,1), never 0),
  x  = wb >> 8                    (angle 2*pi*x / 2^24),
  R  = sqrt(-2 ln u1), z_even = R cos(angle), z_odd = R sin(angle).
  ln, cos and sin are evaluated in FP32 by the fixed sequences of correctly
  rounded +, -, *, /, sqrt below (Taylor series of atanh, sin and cos with
  exact octant reduction), so that both implementations agree bit for bit.

Structured test matrices (Section 5.5 compares them with the Gaussian one;
the remark after Algorithm 3 names the Khatri-Rao products):

* Uniform: entries i.i.d. on [-1, 1].  Entry (j, c) takes word c mod 4 of
  the same counter as the Gaussian entry and maps it to
  u = (2*(w >> 8) + 1 - 2^24) * 2^-24, an odd multiple of 2^-24 in (-1, 1)
  (exact in FP32).
* Khatri-Rao (KR-Gaussian, KR-uniform): Omega_k is the Khatri-Rao product
  (column-wise Kronecker product) of one factor per mode m != k, each
  n_m x l with n_m the current size of mode m, ordered so that the row
  index of Omega_k is the unfolding's column index (lowest mode fastest):
  Omega_k(j, c) = prod_{m != k} F_m(i_m(j), c).  Entry (i, c) of F_m comes
  from the counter (i, 2^31 | m, c >> 2, (k & 0xff) | (tag << 8)) -- the
  second word keeps these draws apart from the dense ones -- then
  Box-Muller as above (KR-Gaussian) or the uniform map (KR-uniform).
"""
import numpy as np

_MASK32 = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85


def philox4x32_10(c0, c1, c2, c3, seed):
    """Philox4x32-10 block function on uint32 arrays (broadcast together)."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3))
    k0 = int(seed) & 0xFFFFFFFF
    k1 = (int(seed) >> 32) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * c0          # < 2^64: exact in uint64
        p1 = _M1 * c2
        n0 = (p1 >> np.uint64(32)) ^ c1 ^ np.uint64(k0)
        n1 = p1 & _MASK32
        n2 = (p0 >> np.uint64(32)) ^ c3 ^ np.uint64(k1)
        n3 = p0 & _MASK32
        c0, c1, c2, c3 = n0, n1, n2, n3
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return tuple(x.astype(np.uint32) for x in (c0, c1, c2, c3))


def _f32(h):
    return np.float32(float.fromhex(h))


# Taylor coefficients (1/(2m+1) for atanh; 1/n! for sin/cos), rounded to FP32.
_C3, _C5, _C7, _C9, _C11 = (_f32(h) for h in (
    "0x1.555556p-2", "0x1.99999ap-3", "0x1.24924ap-3", "0x1.c71c72p-4", "0x1.745d18p-4"))
_LN2_HI = _f32("0x1.62e4p-1")          # 11 significant bits: E*LN2_HI is exact
_LN2_LO = _f32("0x1.7f7d1cp-20")       # ln 2 - LN2_HI
_THETA_UNIT = _f32("0x1.921fb6p-22")   # (pi/4) * 2^-21
_S3, _S5, _S7, _S9 = (_f32(h) for h in (
    "-0x1.555556p-3", "0x1.111112p-7", "-0x1.a01a02p-13", "0x1.71de3ap-19"))
_K2, _K4, _K6, _K8, _K10 = (_f32(h) for h in (
    "-0x1p-1", "0x1.555556p-5", "-0x1.6c16c2p-10", "0x1.a01a02p-16", "-0x1.27e4fcp-22"))
_ONE = np.float32(1.0)
_SQRT2_BITS = np.uint32(0x3FB504F3)


def log_u1(wa):
    """ln(u1) with u1 = (2*(wa>>9)+1) * 2^-24, FP32, fixed op sequence.

    u1 = m * 2^-24 with m odd in [1, 2^24).  Write m = f * 2^e with f in
    [1, 2) (exact bit construction), move f into [sqrt(1/2), sqrt(2)], then
    ln f = 2 atanh(s), s = (f-1)/(f+1), by its Taylor series to s^11, and
    ln u1 = (e - 24) ln 2 + ln f with ln 2 split in a high and a low part.
    """
    wa = np.asarray(wa, dtype=np.uint32)
    m = (2 * (wa >> np.uint32(9)).astype(np.int64) + 1)
    _, e1 = np.frexp(m.astype(np.float64))      # m = mant * 2^e1, mant in [0.5, 1): exact
    e = e1.astype(np.int64) - 1                  # floor(log2 m)
    frac = ((m << (23 - e)) & 0x7FFFFF).astype(np.uint32)
    fbits = np.uint32(0x3F800000) | frac
    big = fbits > _SQRT2_BITS
    fbits = np.where(big, fbits - np.uint32(0x00800000), fbits).astype(np.uint32)
    e = np.where(big, e + 1, e)
    f = fbits.view(np.float32)
    s = (f - _ONE) / (f + _ONE)
    z = s * s
    t = _C11 * z
    t = t + _C9
    t = t * z
    t = t + _C7
    t = t * z
    t = t + _C5
    t = t * z
    t = t + _C3
    t = t * z
    t = t + _ONE
    lnf = (s + s) * t
    E = (e - 24).astype(np.float32)
    return E * _LN2_HI + (E * _LN2_LO + lnf)


def cos_sin_2pi(wb):
    """(cos, sin) of 2*pi*x/2^24 with x = wb >> 8, FP32, fixed op sequence.

    Exact octant reduction on the integer x: octant o = x >> 21, remainder
    rem = x mod 2^21; odd octants use the reflected remainder 2^21 - rem, so
    the reduced angle theta = rem' * (pi/4) 2^-21 lies in [0, pi/4].  sin and
    cos of theta by Taylor series (to theta^9 and theta^10), then the octant
    symmetries of sin/cos.
    """
    x = (np.asarray(wb, dtype=np.uint32) >> np.uint32(8)).astype(np.int64)
    octant = x >> 21
    rem = x & 0x1FFFFF
    odd = (octant & 1) == 1
    rr = np.where(odd, 0x200000 - rem, rem)
    theta = rr.astype(np.float32) * _THETA_UNIT
    z = theta * theta
    p = _S9 * z
    p = p + _S7
    p = p * z
    p = p + _S5
    p = p * z
    p = p + _S3
    sin_t = theta + (theta * z) * p
    c = _K10 * z
    c = c + _K8
    c = c * z
    c = c + _K6
    c = c * z
    c = c + _K4
    c = c * z
    c = c + _K2
    cos_t = _ONE + z * c
    # octant o: angle = o*pi/4 + theta (even o) or (o+1)*pi/4 - theta (odd o)
    cos_v = np.select(
        [octant == 0, octant == 1, octant == 2, octant == 3,
         octant == 4, octant == 5, octant == 6, octant == 7],
        [cos_t, sin_t, -sin_t, -cos_t, -cos_t, -sin_t, sin_t, cos_t])
    sin_v = np.select(
        [octant == 0, octant == 1, octant == 2, octant == 3,
         octant == 4, octant == 5, octant == 6, octant == 7],
        [sin_t, cos_t, cos_t, sin_t, -sin_t, -cos_t, -cos_t, -sin_t])
    return cos_v.astype(np.float32), sin_v.astype(np.float32)


def box_muller(wa, wb):
    """Pair of standard normals (FP32) from two Philox words."""
    lnu = log_u1(wa)
    r = np.sqrt(np.float32(-2.0) * lnu)
    cv, sv = cos_sin_2pi(wb)
    return r * cv, r * sv


def omega_rows(k, row0, rows, l, seed=0, tag=0):
    """Rows [row0, row0+rows) of Omega_k, shape (rows, l), FP32.

    k: 0-based mode; tag < 2^24 distinguishes independent draws (instances,
    requests).  Columns >= l of the last group of four are discarded.
    """
    if rows <= 0 or l <= 0:
        return np.zeros((max(rows, 0), max(l, 0)), dtype=np.float32)
    j = np.arange(row0, row0 + rows, dtype=np.uint64)
    groups = (l + 3) // 4
    out = np.empty((rows, groups * 4), dtype=np.float32)
    c3 = np.uint64((int(k) & 0xFF) | (int(tag) << 8))
    for g in range(groups):
        w0, w1, w2, w3 = philox4x32_10(j & _MASK32, j >> np.uint64(32), np.uint64(g), c3, seed)
        za, zb = box_muller(w0, w1)
        zc, zd = box_muller(w2, w3)
        out[:, 4 * g + 0] = za
        out[:, 4 * g + 1] = zb
        out[:, 4 * g + 2] = zc
        out[:, 4 * g + 3] = zd
    return out[:, :l]


OMEGA_GAUSS = "gauss"
OMEGA_UNIFORM = "uniform"
OMEGA_KR_GAUSS = "kr_gauss"
OMEGA_KR_UNIFORM = "kr_uniform"
OMEGA_KINDS = (OMEGA_GAUSS, OMEGA_UNIFORM, OMEGA_KR_GAUSS, OMEGA_KR_UNIFORM)


def uniform_from_word(w):
    """u = (2*(w >> 8) + 1 - 2^24) * 2^-24 in (-1, 1), FP32 (exact)."""
    m = (np.asarray(w, dtype=np.uint32) >> np.uint32(8)).astype(np.int64)
    return ((2 * m + 1 - (1 << 24)).astype(np.float64) * 2.0 ** -24).astype(np.float32)


def uniform_rows(k, row0, rows, l, seed=0, tag=0):
    """Rows [row0, row0+rows) of the dense uniform Omega_k, shape (rows, l), FP32."""
    if rows <= 0 or l <= 0:
        return np.zeros((max(rows, 0), max(l, 0)), dtype=np.float32)
    j = np.arange(row0, row0 + rows, dtype=np.uint64)
    groups = (l + 3) // 4
    out = np.empty((rows, groups * 4), dtype=np.float32)
    c3 = np.uint64((int(k) & 0xFF) | (int(tag) << 8))
    for g in range(groups):
        ws = philox4x32_10(j & _MASK32, j >> np.uint64(32), np.uint64(g), c3, seed)
        for e in range(4):
            out[:, 4 * g + e] = uniform_from_word(ws[e])
    return out[:, :l]


def kr_factor(k, m, n_m, l, gaussian, seed=0, tag=0):
    """Factor F_m (n_m x l, FP32) of mode k's Khatri-Rao test matrix."""
    if n_m <= 0 or l <= 0:
        return np.zeros((max(n_m, 0), max(l, 0)), dtype=np.float32)
    i = np.arange(n_m, dtype=np.uint64)
    groups = (l + 3) // 4
    out = np.empty((n_m, groups * 4), dtype=np.float32)
    c1 = np.uint64((1 << 31) | int(m))
    c3 = np.uint64((int(k) & 0xFF) | (int(tag) << 8))
    for g in range(groups):
        w0, w1, w2, w3 = philox4x32_10(i, c1, np.uint64(g), c3, seed)
        if gaussian:
            out[:, 4 * g + 0], out[:, 4 * g + 1] = box_muller(w0, w1)
            out[:, 4 * g + 2], out[:, 4 * g + 3] = box_muller(w2, w3)
        else:
            for e, w in enumerate((w0, w1, w2, w3)):
                out[:, 4 * g + e] = uniform_from_word(w)
    return out[:, :l]


def omega_matrix(kind, shape, k, l, seed=0, tag=0):
    """Omega_k (prod_{m != k} shape[m] x l) of the given kind, in FP64.

    The Khatri-Rao kinds are formed by the definition: scipy's khatri_rao
    (column-wise Kronecker product, the second operand's row index fastest)
    applied to the factors from the highest mode down to the lowest.
    """
    d = len(shape)
    cols = int(np.prod([shape[m] for m in range(d) if m != k]))
    if kind == OMEGA_GAUSS:
        return omega_rows(k, 0, cols, l, seed=seed, tag=tag).astype(np.float64)
    if kind == OMEGA_UNIFORM:
        return uniform_rows(k, 0, cols, l, seed=seed, tag=tag).astype(np.float64)
    if kind not in (OMEGA_KR_GAUSS, OMEGA_KR_UNIFORM):
        raise ValueError(kind)
    from scipy.linalg import khatri_rao
    gaussian = kind == OMEGA_KR_GAUSS
    Om = None
    for m in range(d):
        if m == k:
            continue
        F = kr_factor(k, m, int(shape[m]), l, gaussian, seed=seed, tag=tag).astype(np.float64)
        Om = F if Om is None else khatri_rao(F, Om)
    if Om is None:      # order-1 tensor: one column index
        Om = np.ones((1, l))
    return Om
