"""Full-size parity in the benchmark's launch configuration (marked gpu).

Every workload the benchmark times, at its full size, with the same inputs
(seed 2), plan options (default depth rule, one-SM tiles) and entry point:
sampled output rows -- first and last rows, tile boundaries, rows of every
tile band, near-diagonal entries -- against the oracle computed row by row.
The classical path (depth 0) is checked next to the fast one where the
benchmark compares them.  Every full-size result is also checked whole by
Freivalds' test, C·x ≡ A·(Aᵀ·x) mod p for two random x, in exact integer
arithmetic that shares nothing with the library, and, where
tests/golden/fullsize_sha256.txt holds the oracle's digest of the whole
lower triangle, bit for bit against it.  The batch of 2048 uneven problems
is checked on a seeded sample of problems' rows and, through the stored
digest, on every problem's whole triangle.
"""
import hashlib
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2001_04109_gb300 import ffsyrk, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()


def sample_rows(n, count, seed):
    fixed = [0, 1, 127, 128, 255, 256, n // 2, n - 2, n - 1]
    rng = np.random.default_rng(seed)
    rows = set(r for r in fixed if 0 <= r < n)
    rows.update(int(r) for r in rng.integers(0, n, size=count))
    return np.array(sorted(rows), dtype=np.int64)


def freivalds(A_host, p, C_dev, seed, vectors=2):
    """C·x ≡ A·(Aᵀ·x) mod p for random x, C the full symmetric matrix of the lower triangle.

    Exact in uint64 (residues < 2^24, sums of ≤ 2^15 products < 2^61, in row
    chunks); a wrong entry anywhere in the triangle escapes one vector with
    probability at most 1/p.  Independent of the library and of the oracle.
    """
    A = A_host.numpy().view(np.uint32).astype(np.uint64) % np.uint64(p)
    n, k = A.shape
    P = np.uint64(p)
    C = C_dev.cpu().numpy().view(np.uint32)
    rng = np.random.default_rng(seed)
    chunk = 2048
    for _ in range(vectors):
        x = rng.integers(0, p, size=n, dtype=np.uint64)
        # A·(Aᵀ·x), with k and n ≤ 2^15 terms per sum
        atx = np.zeros(k, dtype=np.uint64)
        for r0 in range(0, n, chunk):
            atx = (atx + (A[r0:r0 + chunk].T @ x[r0:r0 + chunk]) % P) % P
        want = (A @ atx) % P
        # tril(C)·x + tril(C, −1)ᵀ·x
        got = np.zeros(n, dtype=np.uint64)
        for r0 in range(0, n, chunk):
            L = np.tril(C[r0:r0 + chunk].astype(np.uint64), k=r0)          # rows r0.., lower part
            got[r0:r0 + chunk] = (got[r0:r0 + chunk] + (L @ x) % P) % P
            S = np.tril(C[r0:r0 + chunk].astype(np.uint64), k=r0 - 1)      # strict lower part
            got = (got + (S.T @ x[r0:r0 + chunk]) % P) % P
        assert np.array_equal(got, want), "Freivalds check failed: some entry of C is wrong"


def _golden():
    """The digest script of tests/golden (its hashing is the one the stored digests used)."""
    import importlib.util
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "make_fullsize_sha256.py")
    spec = importlib.util.spec_from_file_location("make_fullsize_sha256", path)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def stored_digests():
    """Key → SHA-256 of the oracle's lower triangles (tests/golden/fullsize_sha256.txt):
    (n, k, p) for seed-2 workloads, ("batched", count, lo, hi, p, seed) for the batch."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize_sha256.txt")
    out = {}
    if os.path.exists(path):
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            f = line.split()
            if f[0] == "batched":
                out[("batched",) + tuple(int(x) for x in f[1:6])] = f[6]
            elif int(f[3]) == 2:
                out[(int(f[0]), int(f[1]), int(f[2]))] = f[4]
    return out


def lower_sha256(C_dev) -> str:
    h = hashlib.sha256()
    _golden().lower_update(h, C_dev.cpu().numpy().view(np.uint32))
    return h.hexdigest()


def check_rows(A_host, p, C_dev, rows):
    want = oracle.syrk_rows(A_host.numpy(), p, rows)
    got = C_dev[torch.from_numpy(rows).cuda()].cpu().numpy().view(np.uint32)
    for t, r in enumerate(rows):
        bad = np.flatnonzero(got[t, : r + 1] != want[t, : r + 1])
        assert bad.size == 0, f"row {r}: {bad.size} entries differ (first at column {bad[0]})"


# (n, k, p, depths): the benchmark's workloads; None = the default depth rule
WORKLOADS = [
    (256, 256, 65521, [0]),
    (4096, 4096, 65521, [None, 1]),
    (8192, 8192, 65521, [0, 1]),
    (16384, 4096, 131071, [None, 1]),
    (4096, 16384, 131071, [None, 1]),
    (16383, 4097, 131071, [None, 1]),
    (16384, 16384, 65521, [None]),
]


@pytest.mark.parametrize("n,k,p,depths", WORKLOADS, ids=[f"{n}x{k}_p{p}" for n, k, p, _ in WORKLOADS])
def test_workload_sampled_rows(n, k, p, depths):
    A = inputs.uniform_residues(n, k, p, seed=2, device="cuda")  # the same matrix on any device
    A_host = A.cpu()
    rows = sample_rows(n, 24, seed=n + k)
    for levels in depths:
        C = torch.zeros((n, n), dtype=torch.int32, device="cuda")
        plan = ffsyrk.Plan(p, n, k, levels=levels)
        plan(A, C)
        plan.sync_status()
        check_rows(A_host, p, C, rows)
        freivalds(A_host, p, C, seed=n + k + (levels or 0))
        digest = stored_digests().get((n, k, p))
        if digest is not None:  # the whole triangle, bit for bit, against the oracle's
            assert lower_sha256(C) == digest, f"lower triangle differs from the oracle ({levels})"
        plan.close()
        del C
    torch.cuda.empty_cache()


def test_large_d3_three_levels_sampled_rows():
    # A 32768×32768 (4 GiB), p = 8388593: three digits, the depth the benchmark times
    n = k = 32768
    p = 8388593
    A = inputs.uniform_residues(n, k, p, seed=2, device="cuda")
    A_host = A.cpu()
    C = torch.zeros((n, n), dtype=torch.int32, device="cuda")
    plan = ffsyrk.Plan(p, n, k, levels=3)
    plan(A, C)
    plan.sync_status()
    check_rows(A_host, p, C, sample_rows(n, 48, seed=7))
    freivalds(A_host, p, C, seed=32768)
    digest = stored_digests().get((n, k, p))
    if digest is not None:  # the whole triangle against the oracle's
        assert lower_sha256(C) == digest, "lower triangle differs from the oracle"
    plan.close()
    del A, C
    torch.cuda.empty_cache()


def test_batched_2048_uneven_sampled_problems():
    p, seed = 65521, 5
    shapes = inputs.batch_shapes(2048, 32, 2048, seed)
    As = [inputs.uniform_residues(n, k, p, seed=seed * 100000 + t, device="cuda")
          for t, (n, k) in enumerate(shapes)]
    Cs = ffsyrk.batched(As, p)
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    picks = sorted(set(int(t) for t in rng.integers(0, len(shapes), size=12)) |
                   {int(np.argmin([n * n * k for n, k in shapes])), int(np.argmax([n for n, _ in shapes]))})
    for t in picks:
        n, _ = shapes[t]
        rows = sample_rows(n, 16, seed=t)
        check_rows(As[t].cpu(), p, Cs[t], rows)
    digest = stored_digests().get(("batched", 2048, 32, 2048, p, seed))
    if digest is not None:  # every problem's whole triangle against the oracle's
        g = _golden()
        h = hashlib.sha256()
        for C in Cs:
            g.lower_update(h, C.cpu().numpy().view(np.uint32))
        assert h.hexdigest() == digest, "some problem of the batch differs from the oracle"
