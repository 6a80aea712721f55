"""Helper run in a subprocess: Philox4x32-10 words from Triton's own
implementation (interpreter mode, CPU), used as an independent pin of the
oracle's Philox.  Reads JSON [[seed, c0, c1, c2, c3], ...] on stdin."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"
import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kern(out_ptr, c_ptr, seed, N: tl.constexpr):
    offs = tl.arange(0, N)
    c0 = tl.load(c_ptr + offs * 4 + 0).to(tl.uint32)
    c1 = tl.load(c_ptr + offs * 4 + 1).to(tl.uint32)
    c2 = tl.load(c_ptr + offs * 4 + 2).to(tl.uint32)
    c3 = tl.load(c_ptr + offs * 4 + 3).to(tl.uint32)
    a, b, c, d = tl.random.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + offs * 4 + 0, a.to(tl.int64) & 0xFFFFFFFF)
    tl.store(out_ptr + offs * 4 + 1, b.to(tl.int64) & 0xFFFFFFFF)
    tl.store(out_ptr + offs * 4 + 2, c.to(tl.int64) & 0xFFFFFFFF)
    tl.store(out_ptr + offs * 4 + 3, d.to(tl.int64) & 0xFFFFFFFF)


def main():
    cases = json.load(sys.stdin)
    res = []
    for seed, c0, c1, c2, c3 in cases:
        ctr = torch.tensor([[c0, c1, c2, c3]], dtype=torch.int64).repeat(2, 1)
        out = torch.zeros(8, dtype=torch.int64)
        _kern[(1,)](out, ctr, seed, N=2)
        res.append([int(x) for x in out[:4].tolist()])
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
