"""Pins of the schoolbook oracle against facts outside itself (CPU only).

Brute force against Python big integers, closed forms, and invariants of
C = A·Aᵀ mod p.  A plausible mistake in the oracle (a dropped reduction of
the inputs, an overflowing running sum, a transposed index, a missing term)
fails at least one of these.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2001_04109_gb300 import inputs


def bigint_syrk_full(A, p):
    A = [[int(x) for x in row] for row in A]
    n = len(A)
    return [[sum(A[i][l] * A[j][l] for l in range(len(A[i]))) % p for j in range(n)]
            for i in range(n)]


@pytest.mark.parametrize("p", [3, 5, 7])
def test_brute_force_all_tiny_matrices(p):
    # every A in F_p^{n×k} with n·k ≤ 4
    for n, k in [(1, 1), (1, 2), (2, 1), (1, 3), (3, 1), (1, 4), (2, 2), (4, 1)]:
        for vals in itertools.product(range(p), repeat=n * k):
            A = np.array(vals, dtype=np.uint32).reshape(n, k)
            want = bigint_syrk_full(A, p)
            got = oracle.syrk(A, p, "full", threads=1)
            assert got.tolist() == want, (p, A.tolist())


@pytest.mark.parametrize("seed", range(6))
def test_random_small_arbitrary_u32(seed):
    rng = np.random.default_rng(seed)
    for p in [3, 65521, 131071, 8388593, 16777213]:
        n, k = int(rng.integers(1, 9)), int(rng.integers(1, 9))
        A = rng.integers(0, 1 << 32, size=(n, k), dtype=np.uint64).astype(np.uint32)
        want = np.array(bigint_syrk_full(A, p), dtype=np.uint32)
        full = oracle.syrk(A, p, "full", threads=2)
        lo = oracle.syrk(A, p, "lower", threads=3)
        upr = oracle.syrk(A, p, "upper", threads=1)
        assert np.array_equal(full, want)
        assert np.array_equal(lo, np.tril(want))
        assert np.array_equal(upr, np.triu(want))


def test_identity_and_constants():
    p = 65521
    n = 37
    A = np.eye(n, dtype=np.uint32)
    assert np.array_equal(oracle.syrk(A, p, "full"), np.eye(n, dtype=np.uint32))
    k = 50
    ones = np.ones((n, k), dtype=np.uint32)
    assert np.all(oracle.syrk(ones, p, "full") == k % p)
    # A[i][l] = c_i  ->  C[i][j] = k·c_i·c_j
    c = np.arange(1, n + 1, dtype=np.uint64) * 977 % p
    A = np.repeat(c[:, None], k, axis=1).astype(np.uint32)
    want = (np.outer(c, c) % p) * k % p
    assert np.array_equal(oracle.syrk(A, p, "full"), want.astype(np.uint32))


def test_single_nonzero_column_is_rank_one():
    p = 131071
    rng = np.random.default_rng(1)
    A = np.zeros((20, 9), dtype=np.uint32)
    col = rng.integers(0, p, size=20, dtype=np.uint64)
    A[:, 4] = col
    want = np.outer(col, col) % p
    assert np.array_equal(oracle.syrk(A, p, "full"), want.astype(np.uint32))


@pytest.mark.parametrize("p", [65521, 8388593, 16777213])
def test_long_k_max_entries_exercises_periodic_reduction(p):
    # (p−1)² ≡ 1, so an all-(p−1) matrix gives k mod p everywhere; k spans
    # more than two reduction periods of the running sum.
    k = 70001
    A = np.full((3, k), p - 1, dtype=np.uint32)
    assert np.all(oracle.syrk(A, p, "full") == k % p)
    # entries ≥ p are reduced first: p + 1 ≡ 1
    A = np.full((2, k), p + 1, dtype=np.uint32)
    assert np.all(oracle.syrk(A, p, "full") == k % p)


def test_symmetry_and_row_scaling():
    p = 8388593
    A = inputs.uniform_residues(41, 33, p, seed=11).numpy().view(np.uint32)
    C = oracle.syrk(A, p, "full")
    assert np.array_equal(C, C.T)
    s, i = 12345, 7
    B = A.copy().astype(np.uint64)
    B[i] = B[i] * s % p
    D = oracle.syrk(B.astype(np.uint32), p, "full").astype(np.uint64)
    Cu = C.astype(np.uint64)
    want = Cu.copy()
    want[i, :] = Cu[i, :] * s % p
    want[:, i] = Cu[:, i] * s % p
    want[i, i] = Cu[i, i] * s % p * s % p
    assert np.array_equal(D, want)


def test_rows_match_full_and_edge_cases():
    p = 131071
    A = inputs.uniform_residues(30, 19, p, seed=5).numpy().view(np.uint32)
    full = oracle.syrk(A, p, "full")
    rows = [0, 29, 13, 13]
    assert np.array_equal(oracle.syrk_rows(A, p, rows), full[rows])
    # k = 0: the empty sum
    assert np.all(oracle.syrk(np.zeros((4, 0), dtype=np.uint32), p, "full") == 0)
    assert oracle.syrk(np.zeros((0, 5), dtype=np.uint32), p).shape == (0, 0)
    with pytest.raises(ValueError):
        oracle.syrk_rows(A, p, [30])


@pytest.mark.parametrize("seed", range(4))
def test_update_against_big_integers(seed):
    # C ← α·A·Aᵀ + β·C on one triangle (Section 4.2, Table 4), written out in
    # Python integers: only the triangle changes, α and β reduce mod p
    rng = np.random.default_rng(100 + seed)
    for p in [5, 65521, 131071, 8388593]:
        n, k = int(rng.integers(1, 8)), int(rng.integers(1, 8))
        A = rng.integers(0, 1 << 32, size=(n, k), dtype=np.uint64).astype(np.uint32)
        C0 = rng.integers(0, p, size=(n, n), dtype=np.uint64).astype(np.uint32)
        alpha, beta = int(rng.integers(0, 1 << 32)), int(rng.integers(0, 1 << 32))
        full = bigint_syrk_full(A, p)
        for uplo in ["lower", "upper"]:
            got = oracle.syrk_update(A, p, alpha, C0, beta, uplo)
            for i in range(n):
                for j in range(n):
                    inside = j <= i if uplo == "lower" else j >= i
                    want = (alpha * full[i][j] + beta * int(C0[i, j])) % p if inside else int(C0[i, j])
                    assert int(got[i, j]) == want, (p, uplo, i, j)


def test_update_special_cases():
    # α = 1, β = 0 is the product; α = 0 scales C; β = 1 accumulates
    p = 65521
    A = inputs.uniform_residues(9, 13, p, seed=8).numpy().view(np.uint32)
    C0 = inputs.uniform_residues(9, 9, p, seed=9).numpy().view(np.uint32)
    P = oracle.syrk(A, p, "lower")
    low = np.tril(np.ones((9, 9), dtype=bool))
    got = oracle.syrk_update(A, p, 1, C0, 0)
    assert np.array_equal(got[low], P[low]) and np.array_equal(got[~low], C0[~low])
    got = oracle.syrk_update(A, p, 0, C0, 3)
    assert np.array_equal(got[low], (3 * C0[low].astype(np.uint64) % p).astype(np.uint32))
    got = oracle.syrk_update(A, p, 1, C0, 1)
    assert np.array_equal(got[low], ((P[low].astype(np.uint64) + C0[low]) % p).astype(np.uint32))


def test_fullsize_digests_cover_the_benchmark_workloads():
    # tests/golden/fullsize_sha256.txt is written by make_fullsize_sha256.py
    # from the oracle alone; the GPU full-size tests compare whole triangles
    # against it with the script's own hashing (lower_update).
    import hashlib
    import importlib.util
    import os
    import numpy as np
    import oracle
    from paper_2001_04109_gb300 import inputs
    here = os.path.dirname(os.path.abspath(__file__))
    rows = [ln.split() for ln in open(os.path.join(here, "golden", "fullsize_sha256.txt"))
            if ln.strip() and not ln.startswith("#")]
    have = {(int(r[0]), int(r[1]), int(r[2])) for r in rows if r[0] != "batched" and len(r[4]) == 64}
    for w in [(256, 256, 65521), (4096, 4096, 65521), (4096, 16384, 131071), (8192, 8192, 65521),
              (16384, 4096, 131071), (16383, 4097, 131071), (16384, 16384, 65521)]:
        assert w in have, w
    spec = importlib.util.spec_from_file_location(
        "make_fullsize_sha256", os.path.join(here, "golden", "make_fullsize_sha256.py"))
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    # a workload's digest: the rows of its lower triangle in order
    A = inputs.uniform_residues(37, 23, 65521, seed=2).numpy().view(np.uint32)
    C = oracle.syrk(A, 65521, "lower")
    flat = np.concatenate([C[i, : i + 1] for i in range(37)]).astype("<u4").tobytes()
    assert g.workload_digest(37, 23, 65521) == hashlib.sha256(flat).hexdigest()
    # a batch's digest: the problems' triangles in problem order, built as the GPU test builds it
    shapes = inputs.batch_shapes(5, 32, 64, 5)
    h = hashlib.sha256()
    for t, (n, k) in enumerate(shapes):
        At = inputs.uniform_residues(n, k, 65521, seed=5 * 100000 + t).numpy().view(np.uint32)
        g.lower_update(h, oracle.syrk(At, 65521, "lower"))
    assert g.batch_digest(5, 32, 64, 65521, 5) == h.hexdigest()
