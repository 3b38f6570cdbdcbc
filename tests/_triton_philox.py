"""Helper run in a subprocess by test_oracle_rng.py: evaluates Triton's own
Philox4x32-10 (an implementation independent of the oracle) in Triton's CPU
interpreter for the counters/keys given as JSON on stdin; prints JSON words."""
import json
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"
import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kernel(c_ptr, out_ptr, seed, n: tl.constexpr):
    i = tl.arange(0, n)
    c0 = tl.load(c_ptr + i * 4 + 0).to(tl.uint32, bitcast=True)
    c1 = tl.load(c_ptr + i * 4 + 1).to(tl.uint32, bitcast=True)
    c2 = tl.load(c_ptr + i * 4 + 2).to(tl.uint32, bitcast=True)
    c3 = tl.load(c_ptr + i * 4 + 3).to(tl.uint32, bitcast=True)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + i * 4 + 0, a.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 1, b.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 2, c.to(tl.int32, bitcast=True))
    tl.store(out_ptr + i * 4 + 3, d.to(tl.int32, bitcast=True))


def main():
    req = json.load(sys.stdin)
    res = []
    for seed, ctrs in req:
        n = len(ctrs)
        npow = 1 << max(0, (n - 1).bit_length())
        arr = np.zeros((npow, 4), dtype=np.uint32)
        arr[:n] = np.asarray(ctrs, dtype=np.uint64).astype(np.uint32)
        c = torch.from_numpy(arr.view(np.int32).copy())
        out = torch.zeros((npow, 4), dtype=torch.int32)
        _kernel[(1,)](c, out, seed, npow)
        res.append(out.numpy().view(np.uint32)[:n].astype(np.int64).tolist())
    json.dump(res, sys.stdout)


if __name__ == "__main__":
    main()
