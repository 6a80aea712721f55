"""Plain FP64 CPU oracle of the shifted randomized T-HOSVD / ST-HOSVD method.

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
anything from this package.  The CUDA library never calls it, and it never calls
the CUDA library: the two share no code.  Both consume the seeded input
generators of ``paper_2506_04840_gb300.inputs``, which hold none of the
method's arithmetic.

Modules
-------
``omega``   counter-based Gaussian test matrix (Philox4x32-10 + Box-Muller with
            hand-written FP32 log/sin/cos), re-derived from the published
            definitions; used for Omega_k in Algorithms 2 and 3.
``tucker``  Algorithm 1 (deterministic T-/ST-HOSVD), Algorithm 2 (shifted
            randomized T-HOSVD), Algorithm 3 (shifted randomized ST-HOSVD),
            Algorithm A.1 (the unshifted model, alpha = 0), the relative error
            of Section 5, and the mode-k product of Section 2.

Parity status: every function is pinned by a ``-m "not gpu"`` test against
something other than itself (a third-party Philox, closed forms, printed
values of Table 5.3, dense brute force, algebraic identities).  None is
"parity unpinned".
"""
