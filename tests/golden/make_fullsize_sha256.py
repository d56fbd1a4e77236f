"""Write fullsize_sha256.txt: SHA-256 of the oracle's lower triangles of
A·Aᵀ mod p for the benchmark's full-size inputs, one line per workload.

Calls only the oracle and the seeded input generator.  A workload's digest
covers its lower triangle row by row (row i: entries 0..i), each entry a
little-endian uint32; the batch's digest covers its problems' triangles in
problem order.  Lines already in the file are kept; missing ones are
computed (--large adds A 32768², p = 8388593: about 75 minutes on 8 cores).
Run from the repository root:  python tests/golden/make_fullsize_sha256.py [--large]
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

OUT = os.path.join(HERE, "fullsize_sha256.txt")
# (n, k, p): the benchmark's single-problem workloads (inputs seeded with 2)
WORKLOADS = [(256, 256, 65521), (4096, 4096, 65521), (4096, 16384, 131071), (8192, 8192, 65521),
             (16384, 4096, 131071), (16383, 4097, 131071), (16384, 16384, 65521)]
LARGE = (32768, 32768, 8388593)
SEED = 2
# the benchmark's batch: count, n and k log-uniform in [lo, hi], p, seed
BATCH = (2048, 32, 2048, 65521, 5)


def lower_update(h, C: np.ndarray) -> None:
    C = np.ascontiguousarray(C.astype("<u4", copy=False))
    for i in range(C.shape[0]):
        h.update(C[i, : i + 1].tobytes())


def workload_digest(n, k, p, seed=SEED) -> str:
    A = inputs.uniform_residues(n, k, p, seed=seed).numpy().view(np.uint32)
    h = hashlib.sha256()
    lower_update(h, oracle.syrk(A, p, "lower"))
    return h.hexdigest()


def batch_digest(count, lo, hi, p, seed) -> str:
    h = hashlib.sha256()
    for t, (n, k) in enumerate(inputs.batch_shapes(count, lo, hi, seed)):
        A = inputs.uniform_residues(n, k, p, seed=seed * 100000 + t).numpy().view(np.uint32)
        lower_update(h, oracle.syrk(A, p, "lower"))
    return h.hexdigest()


def main():
    have = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            if line.strip() and not line.startswith("#"):
                f = line.split()
                have[tuple(f[:-1])] = f[-1]
    todo = [tuple(str(x) for x in (n, k, p, SEED)) for n, k, p in WORKLOADS]
    if "--large" in sys.argv:
        todo.append(tuple(str(x) for x in (*LARGE, SEED)))
    todo.append(("batched",) + tuple(str(x) for x in BATCH))
    for key in todo:
        if key in have:
            continue
        t = time.time()
        if key[0] == "batched":
            have[key] = batch_digest(*(int(x) for x in key[1:]))
        else:
            have[key] = workload_digest(int(key[0]), int(key[1]), int(key[2]), int(key[3]))
        print(" ".join(key), have[key], f"({time.time() - t:.0f} s)", flush=True)
        write(have)
    write(have)


def write(have):
    lines = ["# n k p seed sha256(lower triangle of A·Aᵀ mod p, rows in order, uint32 LE)",
             "# batched count lo hi p seed sha256(the problems' lower triangles in problem order)",
             "# written by tests/golden/make_fullsize_sha256.py from the oracle"]
    lines += [" ".join(key) + " " + d for key, d in have.items()]
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
