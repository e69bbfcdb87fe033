"""Independent Philox4x32-10 outputs from triton's implementation, run by
triton's CPU interpreter (TRITON_INTERPRET=1).  Used only as a pin for the
oracle's generator in tests; nothing on the product path uses triton.

Usage: python philox_triton_reference.py < json [[c0,c1,c2,c3,k0,k1], ...]
prints json [[w0,w1,w2,w3], ...] (uint32 values).
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(seed_ptr, c_ptr, out_ptr, N: tl.constexpr):
    i = tl.arange(0, N)
    seed = tl.load(seed_ptr + i).to(tl.uint64)
    c0 = tl.load(c_ptr + i * 4 + 0).to(tl.uint32)
    c1 = tl.load(c_ptr + i * 4 + 1).to(tl.uint32)
    c2 = tl.load(c_ptr + i * 4 + 2).to(tl.uint32)
    c3 = tl.load(c_ptr + i * 4 + 3).to(tl.uint32)
    w0, w1, w2, w3 = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + i * 4 + 0, w0.to(tl.int64))
    tl.store(out_ptr + i * 4 + 1, w1.to(tl.int64))
    tl.store(out_ptr + i * 4 + 2, w2.to(tl.int64))
    tl.store(out_ptr + i * 4 + 3, w3.to(tl.int64))


def main():
    cases = json.load(sys.stdin)
    n = 1
    while n < len(cases):
        n *= 2
    seeds = torch.zeros(n, dtype=torch.int64)
    ctr = torch.zeros(n * 4, dtype=torch.int64)
    for i, (c0, c1, c2, c3, k0, k1) in enumerate(cases):
        s = (k1 << 32) | k0
        seeds[i] = s - (1 << 64) if s >= (1 << 63) else s
        ctr[4 * i:4 * i + 4] = torch.tensor([c0, c1, c2, c3], dtype=torch.int64)
    out = torch.zeros(n * 4, dtype=torch.int64)
    _philox_kernel[(1,)](seeds, ctr, out, N=n)
    res = [[int(v) & 0xFFFFFFFF for v in out[4 * i:4 * i + 4].tolist()] for i in range(len(cases))]
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
