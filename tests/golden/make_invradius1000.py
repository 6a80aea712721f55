"""Writes invradius1000.json and invradius1000_factors.npz: the oracle's
result of Algorithm 3 (shifted randomized ST-HOSVD, r = (50,50,50), s = 10,
q = 3, Omega seed 0, tag 0) on the 1000^3 inverse-radius tensor
a_ijk = (i^2+j^2+k^2)^(-1/2) + N(0, (1e-6 ||A0|| / sqrt(N))^2) (generator seed
3, rounded to FP32 as the library reads it), in the plain form and in the
precision form (power steps 1..q-1 on the bfloat16-rounded tensor, the shift
restarting for step q; all arithmetic FP64).

Stored per form: the relative error ||A - A_hat|| / ||A|| (Section 5's
definition), and per mode the final singular values of the shifted product,
the shift history, the size j_k of the well-separated leading block of the
factor (gap (s_j^2 - s_{j+1}^2) / s_1^2 >= 1e-5 on those singular values)
and the factor's first j_k columns (FP32 in the .npz: the parity test checks
principal-angle sines of 1e-5).  Also the tensor's sum and sum of squares in
FP64, so a test can check that it rebuilt the same input.

Run from the repository root:  python tests/golden/make_invradius1000.py
(about 5 minutes and 40 GB of host memory: the reconstruction for the
relative error is formed in FP64).
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import tucker as T            # noqa: E402
from paper_2506_04840_gb300 import inputs as I   # noqa: E402

N, R, S, Q = 1000, [50, 50, 50], 10, 3


def main():
    A = I.inverse_radius(N, seed=3, noise=1e-6)
    A64 = A.astype(np.float64)
    out = {"source": "oracle (FP64) Algorithm 3 on the 1000^3 inverse-radius tensor + 1e-6 "
                     "relative Gaussian noise (generator seed 3, FP32-rounded); r = (50,50,50), "
                     "s = 10, q = 3, Omega seed 0; plain and precision (bfloat16 power) forms",
           "n": N, "r": R, "s": S, "q": Q, "seed": 3,
           "sum": float(np.sum(A64)), "sum_sq": float(np.sum(A64 * A64)), "forms": {}}
    factors = {}
    for name, bf in (("plain", False), ("bf16_power", True)):
        G, Us, st = T.rsthosvd(A64, R, S, Q, bf16_power=bf)
        re = T.rel_error(A64, G, Us)
        modes = []
        for k in range(3):
            sig = np.asarray(st[k]["sigma"], dtype=np.float64)
            j = T.separated_block(sig, R[k])
            modes.append({"sigma": sig.tolist(), "alpha": [float(a) for a in st[k]["alpha"]],
                          "separated_block": int(j)})
            factors["%s_U%d" % (name, k)] = np.asarray(Us[k][:, :j], dtype=np.float32)
        out["forms"][name] = {"rel_err": re, "modes": modes}
        print(name, "RE %.9e" % re, [m["separated_block"] for m in modes], flush=True)
    with open(os.path.join(HERE, "invradius1000.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    np.savez_compressed(os.path.join(HERE, "invradius1000_factors.npz"), **factors)


if __name__ == "__main__":
    main()
