"""Philox4x32-10 from an independent implementation (triton's, in interpreter mode on the CPU).

Run as a script: reads counters/keys as JSON from stdin and prints the four
output words per counter as JSON. Used only to pin the oracle's generator.
"""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _blocks(out_ptr, c_ptr, seed, n, BLOCK: tl.constexpr):
    i = tl.arange(0, BLOCK)
    m = i < n
    c0 = tl.load(c_ptr + 4 * i + 0, mask=m)
    c1 = tl.load(c_ptr + 4 * i + 1, mask=m)
    c2 = tl.load(c_ptr + 4 * i + 2, mask=m)
    c3 = tl.load(c_ptr + 4 * i + 3, mask=m)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + 4 * i + 0, a, mask=m)
    tl.store(out_ptr + 4 * i + 1, b, mask=m)
    tl.store(out_ptr + 4 * i + 2, c, mask=m)
    tl.store(out_ptr + 4 * i + 3, d, mask=m)


def main():
    req = json.load(sys.stdin)
    res = []
    for seed, ctrs in req:
        c = torch.tensor(np.array(ctrs, dtype=np.uint32).reshape(-1, 4).astype(np.int64)).to(torch.uint32)
        n = c.shape[0]
        out = torch.zeros((n, 4), dtype=torch.uint32)
        block = 1
        while block < n:
            block *= 2
        _blocks[(1,)](out, c, seed, n, BLOCK=block)
        res.append(out.to(torch.int64).numpy().tolist())
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
