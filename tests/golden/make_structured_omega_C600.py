"""Writes structured_omega_C600.json: the oracle's relative errors of
Algorithm 3 (ST-HOSVD, r = (20,20,20), s = 10, q = 1, seed 0, tag 0) on
tensor C of Section 5.1 (600^3, slow decay, generator seed 11, rounded to
FP32 as the library reads it) for each test matrix kind of Section 5.5.

Run from the repository root:  python tests/golden/make_structured_omega_C600.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import omega as om            # noqa: E402
from oracle import tucker as T            # noqa: E402
from paper_2506_04840_gb300 import inputs as I   # noqa: E402


def main():
    A = I.superdiagonal(600, "slow", seed=11, dtype=np.float32).astype(np.float64)
    out = {"source": "oracle (FP64) Algorithm 3 on tensor C (Section 5.1), 600^3, slow decay, "
                     "seed 11, FP32-rounded; r = (20,20,20), s = 10, q = 1; Section 5.5 kinds",
           "n": 600, "r": 20, "s": 10, "q": 1, "seed": 11, "re": {}}
    for kind in om.OMEGA_KINDS:
        G, Us, _ = T.rsthosvd(A, [20, 20, 20], 10, 1, omega=kind)
        out["re"][kind] = T.rel_error(A, G, Us)
    with open(os.path.join(HERE, "structured_omega_C600.json"), "w") as f:
        json.dump(out, f, indent=2)
        f.write("\n")


if __name__ == "__main__":
    main()
