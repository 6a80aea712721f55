"""Writes pve_tensor_B600.json: the oracle's Algorithm 4 (ST-HOSVD with
PVE-controlled counts; r = (20,20,20), s = 10, q_max = 10, tol = 0.5, seed
0, tag 0) on tensor B of Section 5.1 (600^3, generator seed 12, rounded to
FP32 as the library reads it): the counts, the relative error and, per
mode and step, the ratio of the test's left side to its threshold.

Run from the repository root:  python tests/golden/make_pve_tensor_B600.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import tucker as T            # noqa: E402
from paper_2506_04840_gb300 import inputs as I   # noqa: E402


def main():
    A = I.sparse_rank_one_sum(600, 12, dtype=np.float32).astype(np.float64)
    r, s, qmax, tol = [20, 20, 20], 10, 10, 0.5
    G, Us, qs, st = T.rsthosvd_pve(A, r, s, qmax, tol)
    ratios = []
    for k in range(3):
        prev = np.zeros_like(st[k]["sigma_hist"][0])
        rk = []
        for sig in st[k]["sigma_hist"]:
            thr = tol * sig[T.pve_threshold_index(r[k], len(sig))]
            rk.append(float(np.max(np.abs(sig[:r[k]] - prev[:r[k]])) / thr))
            prev = sig
        ratios.append(rk)
    out = {"source": "oracle (FP64) Algorithm 4 on tensor B (Section 5.1, weights gamma/i^2 and "
                     "1/i^2), 600^3, seed 12, FP32-rounded; r = (20,20,20), s = 10, q_max = 10, "
                     "tol = 0.5",
           "r": r, "s": s, "q_max": qmax, "tol": tol, "seed": 12,
           "q": [int(x) for x in qs], "re": T.rel_error(A, G, Us), "test_ratios": ratios}
    with open(os.path.join(HERE, "pve_tensor_B600.json"), "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")


if __name__ == "__main__":
    main()
