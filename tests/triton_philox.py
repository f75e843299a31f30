"""Philox-4x32-10 evaluated by Triton's own library routine (tl.philox) in
Triton's CPU interpreter.  Used only to pin the oracle's generator.

Run as a script: python triton_philox.py in.npz out.npy
in.npz holds 'ctr' (n, 4) uint32 and 'seed' (a uint64 scalar); out.npy
receives the (n, 4) uint32 outputs.  A separate process is used because
the interpreter must be selected before Triton is imported.
"""
import os
import sys

os.environ["TRITON_INTERPRET"] = "1"

import numpy as np  # noqa: E402
import torch  # noqa: E402
import triton  # noqa: E402
import triton.language as tl  # noqa: E402


@triton.jit
def _philox_kernel(c_ptr, out_ptr, seed, n, BLOCK: tl.constexpr):
    offs = tl.program_id(0) * BLOCK + tl.arange(0, BLOCK)
    mask = offs < n
    c0 = tl.load(c_ptr + offs * 4 + 0, mask=mask)
    c1 = tl.load(c_ptr + offs * 4 + 1, mask=mask)
    c2 = tl.load(c_ptr + offs * 4 + 2, mask=mask)
    c3 = tl.load(c_ptr + offs * 4 + 3, mask=mask)
    r0, r1, r2, r3 = tl.philox(seed, c0, c1, c2, c3, 10)
    tl.store(out_ptr + offs * 4 + 0, r0, mask=mask)
    tl.store(out_ptr + offs * 4 + 1, r1, mask=mask)
    tl.store(out_ptr + offs * 4 + 2, r2, mask=mask)
    tl.store(out_ptr + offs * 4 + 3, r3, mask=mask)


def main():
    d = np.load(sys.argv[1])
    ctr = np.ascontiguousarray(d["ctr"].astype(np.uint32))
    seed = int(d["seed"])
    n = ctr.shape[0]
    c = torch.from_numpy(ctr.view(np.int32).reshape(-1).copy()).view(torch.uint32)
    out = torch.zeros(n * 4, dtype=torch.int32).view(torch.uint32)
    BLOCK = 256
    _philox_kernel[(triton.cdiv(n, BLOCK),)](c, out, seed, n, BLOCK=BLOCK)
    np.save(sys.argv[2], out.view(torch.int32).numpy().view(np.uint32).reshape(n, 4))


if __name__ == "__main__":
    main()
