"""Write fullsize_sha256.txt: SHA-256 of the oracle's lower triangle of A·Aᵀ mod p
for the benchmark's full-size inputs (seed 2), one line per workload.

Calls only the oracle and the seeded input generator.  The digest covers the
lower triangle row by row (row i: entries 0..i), each entry a little-endian
uint32.  Run from the repository root:  python tests/golden/make_fullsize_sha256.py
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2001_04109_gb300 import inputs  # noqa: E402

# (n, k, p): the benchmark's workloads that the oracle finishes in minutes
WORKLOADS = [(256, 256, 65521), (4096, 4096, 65521), (4096, 16384, 131071), (8192, 8192, 65521),
             (16384, 4096, 131071), (16383, 4097, 131071), (16384, 16384, 65521)]
SEED = 2


def lower_sha256(C: np.ndarray) -> str:
    h = hashlib.sha256()
    C = np.ascontiguousarray(C.astype("<u4", copy=False))
    for i in range(C.shape[0]):
        h.update(C[i, : i + 1].tobytes())
    return h.hexdigest()


def main():
    out = os.path.join(HERE, "fullsize_sha256.txt")
    lines = ["# n k p seed sha256(lower triangle of A·Aᵀ mod p, rows in order, uint32 LE)",
             "# written by tests/golden/make_fullsize_sha256.py from the oracle"]
    for n, k, p in WORKLOADS:
        t = time.time()
        A = inputs.uniform_residues(n, k, p, seed=SEED).numpy().view(np.uint32)
        digest = lower_sha256(oracle.syrk(A, p, "lower"))
        lines.append(f"{n} {k} {p} {SEED} {digest}")
        print(lines[-1], f"({time.time() - t:.0f} s)", flush=True)
    with open(out, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
