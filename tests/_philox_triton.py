"""Helper run in a subprocess: Philox4x32-10 from Triton's CPU interpreter.

Triton's ``philox_impl`` is an independent implementation of the published
Philox4x32 rounds; with TRITON_INTERPRET=1 it runs on the CPU through numpy.
Usage: python _philox_triton.py in.npy out.npy  (in: [n,6] uint32 = ctr[4], key[2]).
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"
import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _kernel(inp, out, n: tl.constexpr):
    idx = tl.arange(0, n)
    c0 = tl.load(inp + idx * 6 + 0)
    c1 = tl.load(inp + idx * 6 + 1)
    c2 = tl.load(inp + idx * 6 + 2)
    c3 = tl.load(inp + idx * 6 + 3)
    k0 = tl.load(inp + idx * 6 + 4)
    k1 = tl.load(inp + idx * 6 + 5)
    a, b, c, d = tl.philox_impl(c0, c1, c2, c3, k0, k1, 10)
    tl.store(out + idx * 4 + 0, a)
    tl.store(out + idx * 4 + 1, b)
    tl.store(out + idx * 4 + 2, c)
    tl.store(out + idx * 4 + 3, d)


def main():
    a = np.load(sys.argv[1]).astype(np.uint32)
    n = a.shape[0]
    assert n & (n - 1) == 0, "power-of-two batch"
    inp = torch.from_numpy(a.reshape(-1).copy())
    out = torch.zeros(n * 4, dtype=torch.uint32)
    _kernel[(1,)](inp, out, n=n)
    np.save(sys.argv[2], out.numpy().reshape(n, 4))


if __name__ == "__main__":
    main()
