"""Oracle (FP64, numpy) of the fixed-rank Tucker algorithms of the paper.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Conventions (the paper is silent on them; the library uses the same ones):
* Tensors are numpy arrays indexed (i_1, ..., i_d), 0-based.  The mode-k
  unfolding X_(k) is n_k x prod_{m != k} n_m with the remaining indices
  ordered lowest mode fastest (Kolda / Tensor Toolbox order, Section 2
  gives only its size).
* svd_econ returns left singular vectors sorted by descending singular
  value, each column's sign fixed so that its entry of largest magnitude is
  positive (lowest row index on ties).
* l_k = min(r_k + s_k, n_k, columns of the current unfolding).
* Shift rule of Algorithms 2/3: if Sigma(l,l) > alpha_{t-1} then
  alpha_t = (Sigma(l,l) + alpha_{t-1}) / 2, else alpha_t = alpha_{t-1}; the
  subtracted shift in the product is alpha_{t-1} (Algorithm 3 prints it
  without index).
"""
import numpy as np

from .omega import OMEGA_GAUSS, omega_matrix

SHIFT_PAPER = "paper"   # adaptive midpoint shift, Algorithms 2 and 3
SHIFT_NONE = "none"     # alpha = 0 throughout: Algorithm A.1


def unfold(X, k):
    """Mode-k unfolding X_(k) (Section 2), Kolda column order."""
    return np.reshape(np.moveaxis(X, k, 0), (X.shape[k], -1), order="F")


def fold(M, k, shape):
    """Inverse of ``unfold`` for a tensor of the given shape."""
    rest = [shape[m] for m in range(len(shape)) if m != k]
    return np.moveaxis(np.reshape(M, [shape[k]] + rest, order="F"), 0, k)


def mode_product(X, B, k):
    """X x_k B (Section 2): c_{..j..} = sum_{i_k} x_{..i_k..} b_{j i_k}."""
    shape = list(X.shape)
    shape[k] = B.shape[0]
    return fold(B @ unfold(X, k), k, shape)


def fix_signs(Q):
    """Flip columns so the entry of largest |value| is positive."""
    Q = np.array(Q, dtype=np.float64, copy=True)
    if Q.size == 0:
        return Q
    idx = np.argmax(np.abs(Q), axis=0)     # first occurrence on ties
    sgn = np.sign(Q[idx, np.arange(Q.shape[1])])
    sgn[sgn == 0] = 1.0
    return Q * sgn


def svd_econ(Y):
    """[Q, Sigma, ~] = svd(Y, 'econ') (LAPACK), with the sign convention."""
    U, S, _ = np.linalg.svd(np.asarray(Y, dtype=np.float64), full_matrices=False)
    return fix_signs(U), S


def clamp_l(r_k, s_k, n_k, ncols):
    return int(min(r_k + s_k, n_k, ncols))


def sketch(X, k, l, seed=0, tag=0, kind=OMEGA_GAUSS):
    """Y = X_(k) Omega_k (Algorithm 2/3, first svd argument); Omega_k of the
    given kind (Section 5.5) for the current sizes of X."""
    X = np.asarray(X, dtype=np.float64)
    return unfold(X, k) @ omega_matrix(kind, X.shape, k, l, seed, tag)


def shift_update(sigma_l, alpha_prev, rule=SHIFT_PAPER):
    """alpha_t from Sigma(l,l) and alpha_{t-1} (Algorithms 2/3)."""
    if rule == SHIFT_NONE:
        return 0.0
    if sigma_l > alpha_prev:
        return 0.5 * (sigma_l + alpha_prev)
    return alpha_prev


def shifted_power(X, k, Q, alpha, q, rule=SHIFT_PAPER, X_for_step=None):
    """q steps of the inner loop of Algorithm 2/3 on X_(k).

    Step t: [Q, Sigma] = svd(X_(k) (X_(k)^T Q) - alpha_{t-1} Q), then the
    shift update.  ``X_for_step(t)`` may supply a different tensor for step
    t (the BF16 precision form); default X for all steps.
    Returns (Q, Sigma, alpha, alpha_hist, sigma_l_hist).
    """
    S = None
    a_hist, s_hist = [], []
    for t in range(1, q + 1):
        Xt = X if X_for_step is None else X_for_step(t)
        Xk = unfold(np.asarray(Xt, dtype=np.float64), k)
        a_used = 0.0 if rule == SHIFT_NONE else alpha
        Y = Xk @ (Xk.T @ Q) - a_used * Q
        Q, S = svd_econ(Y)
        s_l = S[-1]
        alpha = shift_update(s_l, alpha, rule)
        a_hist.append(alpha)
        s_hist.append(s_l)
    return Q, S, alpha, a_hist, s_hist


def _mode_factor(X, k, r_k, s_k, q, seed, tag, rule, X_for_step=None, kind=OMEGA_GAUSS):
    """Steps of Algorithms 2/3 for one mode: sketch, q shifted powers, U_k."""
    Xk_cols = int(np.prod([X.shape[m] for m in range(X.ndim) if m != k]))
    l = clamp_l(r_k, s_k, X.shape[k], Xk_cols)
    if l < r_k:
        raise ValueError("mode %d: only %d columns for rank %d" % (k, l, r_k))
    Y = sketch(X, k, l, seed, tag, kind)
    Q, S = svd_econ(Y)
    if X_for_step is None or q < 2:
        Q, S2, alpha, a_hist, s_hist = shifted_power(X, k, Q, 0.0, q, rule)
    else:
        # precision form: steps 1..q-1 on the bfloat16 copy; the shift sequence
        # restarts at alpha = 0 for step q, which reads the FP32 tensor (the
        # bfloat16 Sigma(l,l) sits on the rounding floor of the copy and would
        # violate 0 < alpha < sigma_l(A A^T)/2, Section 3.1 item (a))
        Q, _, _, a1, s1 = shifted_power(X_for_step(1), k, Q, 0.0, q - 1, rule)
        Q, S2, alpha, a2, s2 = shifted_power(X_for_step(q), k, Q, 0.0, 1, rule)
        a_hist, s_hist = a1 + a2, s1 + s2
    if S2 is not None:
        S = S2
    return Q[:, :r_k], dict(l=l, alpha=a_hist, sigma_l=s_hist, sigma=S)


def rthosvd(A, r, s, q, seed=0, tag=0, rule=SHIFT_PAPER, omega=OMEGA_GAUSS):
    """Algorithm 2: shifted randomized T-HOSVD.  Returns (G, [U_k], stats).
    ``omega``: the test matrix kind (oracle.omega.OMEGA_KINDS)."""
    A = np.asarray(A, dtype=np.float64)
    d = A.ndim
    s = [s] * d if np.isscalar(s) else list(s)
    Us, stats = [], []
    G = A
    for k in range(d):
        U, st = _mode_factor(A, k, r[k], s[k], q, seed, tag, rule, kind=omega)
        Us.append(U)
        stats.append(st)
        G = mode_product(G, U.T, k)
    return G, Us, stats


def rsthosvd(A, r, s, q, seed=0, tag=0, rule=SHIFT_PAPER, order=None, bf16_power=False,
             omega=OMEGA_GAUSS):
    """Algorithm 3: shifted randomized ST-HOSVD.  Returns (G, [U_k], stats).

    ``order`` is a permutation of the modes (Section 2: any processing order).
    ``bf16_power``: the precision form -- power steps 1..q-1 read the
    current tensor rounded to bfloat16; the sketch and step q read it as
    given; all arithmetic stays FP64.
    """
    G = np.asarray(A, dtype=np.float64)
    d = G.ndim
    s = [s] * d if np.isscalar(s) else list(s)
    order = list(range(d)) if order is None else list(order)
    Us = [None] * d
    stats = [None] * d
    for k in order:
        X_for_step = None
        if bf16_power:
            Gb = round_bf16(G)
            X_for_step = (lambda t, Gb=Gb, Gf=G: Gb if t < q else Gf)
        U, st = _mode_factor(G, k, r[k], s[k], q, seed, tag, rule, X_for_step, kind=omega)
        Us[k] = U
        stats[k] = st
        G = mode_product(G, U.T, k)
    return G, Us, stats


def descending_order(shape):
    """The processing order of Section 3.2: n_{p_1} >= ... >= n_{p_d}, ties
    in ascending mode index."""
    return sorted(range(len(shape)), key=lambda k: (-shape[k], k))


def pve_threshold_index(r_k, l):
    """0-based index of the estimate the Algorithm 4 test scales tol by: the
    (r_k+1)-th (the first one past the kept rank), or the last one when the
    sketch has no column past r_k (l_k = r_k)."""
    return min(r_k, l - 1)


def rthosvd_pve(A, r, s, q_max, tol, seed=0, tag=0, rule=SHIFT_PAPER, omega=OMEGA_GAUSS):
    """Algorithm 2 with the PVE-controlled counts of Algorithm 4 (the
    T-HOSVD version Section 3.3 names and Section 5.6 measures): every
    mode's sketch and power steps act on A, the stopping test as in
    ``rsthosvd_pve``; G = A x_1 U_1^T ... x_d U_d^T.
    Returns (G, [U_k], [q_k], stats)."""
    A = np.asarray(A, dtype=np.float64)
    d = A.ndim
    s = [s] * d if np.isscalar(s) else list(s)
    Us, qs, stats = [], [], []
    for k in range(d):
        _, Uk, qk, stk = rsthosvd_pve(A, r, s, q_max, tol, seed=seed, tag=tag, rule=rule,
                                      order=[k], omega=omega)
        Us.append(Uk[k])
        qs.append(qk[k])
        stats.append(stk[k])
    G = A
    for k in range(d):
        G = mode_product(G, Us[k].T, k)
    return G, Us, qs, stats


def rsthosvd_pve(A, r, s, q_max, tol, seed=0, tag=0, rule=SHIFT_PAPER, order=None,
                 omega=OMEGA_GAUSS):
    """Algorithm 4: Algorithm 3 with the power count of each mode chosen by
    the PVE test.  Returns (G, [U_k], [q_k], stats).

    Per mode k, after the sketch's svd (alpha_0 = 0, sigma_hat = 0), step
    t = 1..q_max: q_k = t; [Q, Sigma] = svd(X_(k)(X_(k)^T Q) - alpha_{t-1} Q);
    sigma_t = diag(Sigma) + alpha_{t-1}; stop when
    max_{i <= r_k} |sigma_t(i) - sigma_hat(i)| <= tol * sigma_t(r_k + 1);
    otherwise the shift update of Algorithm 3 and sigma_hat = sigma_t.
    The stats record sigma_t per step ('sigma_hist'), the shifts and q_k.
    """
    G = np.asarray(A, dtype=np.float64)
    d = G.ndim
    s = [s] * d if np.isscalar(s) else list(s)
    order = list(range(d)) if order is None else list(order)
    Us, qs, stats = [None] * d, [0] * d, [None] * d
    for k in order:
        cols = int(np.prod([G.shape[m] for m in range(d) if m != k]))
        l = clamp_l(r[k], s[k], G.shape[k], cols)
        if l < r[k]:
            raise ValueError("mode %d: only %d columns for rank %d" % (k, l, r[k]))
        Xk = unfold(G, k)
        Q, _ = svd_econ(sketch(G, k, l, seed, tag, omega))
        alpha = 0.0
        sig_hat = np.zeros(l)
        hist, a_hist = [], []
        ridx = pve_threshold_index(r[k], l)
        qk = 0
        for t in range(1, q_max + 1):
            qk = t
            a_used = 0.0 if rule == SHIFT_NONE else alpha
            Q, S = svd_econ(Xk @ (Xk.T @ Q) - a_used * Q)
            sig_t = S + a_used
            hist.append(sig_t)
            if np.max(np.abs(sig_t[:r[k]] - sig_hat[:r[k]])) <= tol * sig_t[ridx]:
                break
            alpha = shift_update(S[-1], alpha, rule)
            a_hist.append(alpha)
            sig_hat = sig_t
        Us[k] = Q[:, :r[k]]
        qs[k] = qk
        stats[k] = dict(l=l, q=qk, sigma_hist=hist, alpha=a_hist)
        G = mode_product(G, Us[k].T, k)
    return G, Us, qs, stats


def holistic(A, r, s, q, seed=0, tag=0, rule=SHIFT_PAPER, st=True, omega=OMEGA_GAUSS):
    """Algorithm B.1 (ST case, shifted power steps) and Algorithm A.2
    (rule=SHIFT_NONE; ST or T-HOSVD case): range finding with all l_k
    columns kept, then a deterministic ST-HOSVD of the small tensor.

    Per mode k in 1..d: Q_k from the sketch and q power steps of Algorithm
    3 on B (ST case; B shrinks as it goes) or on A (T-HOSVD case), keeping
    Q_k with l_k columns; B <- B x_k Q_k^T.  Then {G; V_1..V_d} =
    ST-HOSVD(B, r) (Algorithm 1) and U_k = Q_k V_k.
    Returns (G, [U_k], stats) with stats per mode (l, alpha, sigma of the
    range finder; sigma_small, the singular values of the small tensor's
    unfolding that V_k comes from).
    """
    A = np.asarray(A, dtype=np.float64)
    d = A.ndim
    s = [s] * d if np.isscalar(s) else list(s)
    B = A
    Qs, stats = [], []
    for k in range(d):
        X = B if st else A
        cols = int(np.prod([X.shape[m] for m in range(d) if m != k]))
        l = clamp_l(r[k], s[k], X.shape[k], cols)
        if l < r[k]:
            raise ValueError("mode %d: only %d columns for rank %d" % (k, l, r[k]))
        Q, S = svd_econ(sketch(X, k, l, seed, tag, omega))
        Q, S2, _, a_hist, s_hist = shifted_power(X, k, Q, 0.0, q, rule)
        Qs.append(Q)
        stats.append(dict(l=l, alpha=a_hist, sigma_l=s_hist, sigma=S2 if S2 is not None else S))
        B = mode_product(B, Q.T, k)
    G, Vs = hosvd(B, r, sequential=True)
    # record the spectrum each small mode's V_k was taken from (the
    # singular values of the unfolding Algorithm 1 factors at that step)
    Bk = B
    for k in range(d):
        stats[k]["sigma_small"] = np.linalg.svd(unfold(Bk, k), compute_uv=False)
        Bk = mode_product(Bk, Vs[k].T, k)
    return G, [Q @ V for Q, V in zip(Qs, Vs)], stats


def hosvd(A, r, sequential):
    """Algorithm 1: deterministic T-HOSVD (sequential=False) or ST-HOSVD."""
    A = np.asarray(A, dtype=np.float64)
    G = A
    Us = []
    for k in range(A.ndim):
        X = G if sequential else A
        Q, _ = svd_econ(unfold(X, k))
        U = Q[:, :r[k]]
        Us.append(U)
        G = mode_product(G, U.T, k)
    return G, Us


def reconstruct(G, Us):
    """A_hat = G x_1 U_1 x_2 U_2 ... x_d U_d."""
    X = np.asarray(G, dtype=np.float64)
    for k, U in enumerate(Us):
        X = mode_product(X, U, k)
    return X


def rel_error(A, G, Us):
    """RE = ||A - A_hat|| / ||A|| (Section 5, definition of RE)."""
    A = np.asarray(A, dtype=np.float64)
    return float(np.linalg.norm((A - reconstruct(G, Us)).ravel()) / np.linalg.norm(A.ravel()))


def round_bf16(X):
    """Round to bfloat16 (round to nearest, ties to even) and back to FP64.

    Applied to the FP32 value of each entry (the library keeps FP32 data and
    a bfloat16 shadow of it).
    """
    x = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
    b = x.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    rounded = ((b + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (rounded & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return out.astype(np.float64).reshape(np.shape(X))


def principal_sines(U, V):
    """Sines of the principal angles between range(U) and range(V)."""
    Qu, _ = np.linalg.qr(np.asarray(U, dtype=np.float64))
    Qv, _ = np.linalg.qr(np.asarray(V, dtype=np.float64))
    # singular values of the residual (I - Qv Qv^T) Qu are the sines; this
    # avoids the cancellation of sqrt(1 - cos^2) for small angles
    s = np.linalg.svd(Qu - Qv @ (Qv.T @ Qu), compute_uv=False)
    return np.sort(np.clip(s, 0.0, 1.0))


def separated_block(sigma, r, gap=1e-5):
    """Largest j <= r with (sigma_j^2 - sigma_{j+1}^2)/sigma_1^2 >= gap."""
    sig = np.asarray(sigma, dtype=np.float64)
    best = 0
    for j in range(1, min(r, len(sig) - 1) + 1):
        if (sig[j - 1] ** 2 - sig[j] ** 2) / sig[0] ** 2 >= gap:
            best = j
    return best
