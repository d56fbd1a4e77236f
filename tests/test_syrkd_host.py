"""Diagonal scaling (Algorithm 5, syrkd) on the host and in the oracle (CPU only).

The library factors D = Diag(d) as Δ·Δᵀ without field extensions (Algorithm
4, nrsyf, for pairs of non-squares); the product A·D·Aᵀ is then the plain
symmetric product of Ā = [A 0]·Δ.  Checked here: Δ·Δᵀ restricted to A's
columns is exactly D for random d with squares, non-squares (odd and even
counts) and zeros; the oracle's A·D·Aᵀ against Python big integers and
against its own A·Aᵀ for D = I and D = c·I.
"""
import numpy as np
import pytest

import oracle
from paper_2001_04109_gb300 import ffsyrk


def is_square(x, p):
    return x % p == 0 or pow(x, (p - 1) // 2, p) == 1


@pytest.mark.parametrize("p", [3, 5, 7, 11, 13, 65521, 131071, 131041, 8388593, 16777213])
@pytest.mark.parametrize("seed", range(3))
def test_factor_gives_delta_delta_t_equal_d(p, seed):
    rng = np.random.default_rng(seed * 1000 + p % 997)
    for k in [0, 1, 2, 3, 7, 20]:
        d = [int(x) for x in rng.integers(0, 1 << 32, size=k, dtype=np.uint64)]
        if k >= 3:
            d[0] = 0          # zero is a square
            d[1] = p * 5 + 3  # reduced mod p
        kk, partner, u, v = ffsyrk.syrkd_factor(p, d)
        nonsq = sum(1 for x in d if not is_square(x % p, p))
        assert kk == k + (nonsq % 2)
        Delta = [[0] * kk for _ in range(kk)]
        for c in range(kk):
            Delta[c][c] = u[c] % p
            if partner[c] >= 0:
                assert partner[partner[c]] == c  # columns come in pairs
                Delta[partner[c]][c] = v[c] % p
            else:
                assert v[c] == 0
        DDt = [[sum(Delta[i][t] * Delta[j][t] for t in range(kk)) % p for j in range(kk)]
               for i in range(kk)]
        for i in range(k):
            for j in range(k):
                assert DDt[i][j] == (d[i] % p if i == j else 0), (p, d, i, j)


def test_oracle_syrkd_against_big_integers():
    rng = np.random.default_rng(5)
    for p in [5, 65521, 8388593]:
        for _ in range(4):
            n, k = int(rng.integers(1, 7)), int(rng.integers(1, 7))
            A = rng.integers(0, 1 << 32, size=(n, k), dtype=np.uint64).astype(np.uint32)
            d = rng.integers(0, 1 << 32, size=k, dtype=np.uint64).astype(np.uint32)
            want = [[sum(int(A[i, l]) * int(d[l]) * int(A[j, l]) for l in range(k)) % p
                     for j in range(n)] for i in range(n)]
            assert oracle.syrkd(A, d, p, "full").tolist() == want


def test_oracle_syrkd_reduces_to_syrk():
    p = 131071
    rng = np.random.default_rng(6)
    A = rng.integers(0, 1 << 32, size=(17, 23), dtype=np.uint64).astype(np.uint32)
    P = oracle.syrk(A, p, "lower").astype(np.uint64)
    assert np.array_equal(oracle.syrkd(A, np.ones(23, np.uint32), p, "lower"), P.astype(np.uint32))
    assert np.array_equal(oracle.syrkd(A, np.full(23, 9, np.uint32), p, "lower"),
                          (9 * P % p).astype(np.uint32))


def test_oracle_syrkbd_against_big_integers():
    rng = np.random.default_rng(15)
    for p in [3, 7, 65521, 131071]:
        for _ in range(5):
            n, k = int(rng.integers(1, 7)), int(rng.integers(1, 8))
            A = rng.integers(0, 1 << 32, size=(n, k), dtype=np.uint64).astype(np.uint32)
            d = rng.integers(0, 1 << 32, size=k, dtype=np.uint64).astype(np.uint32)
            e = rng.integers(0, 1 << 32, size=max(k - 1, 0), dtype=np.uint64).astype(np.uint32)
            B = [[0] * k for _ in range(k)]
            for l in range(k):
                B[l][l] = int(d[l])
                if l + 1 < k:
                    B[l][l + 1] = B[l + 1][l] = int(e[l])
            want = [[sum(int(A[i, a]) * B[a][b] * int(A[j, b]) for a in range(k) for b in range(k)) % p
                     for j in range(n)] for i in range(n)]
            assert oracle.syrkbd(A, d, e, p, "full").tolist() == want


def test_oracle_syrkbd_special_cases():
    p = 65521
    rng = np.random.default_rng(16)
    A = rng.integers(0, 1 << 32, size=(9, 6), dtype=np.uint64).astype(np.uint32)
    d = rng.integers(0, p, size=6)
    # e = 0: the diagonal product
    assert np.array_equal(oracle.syrkbd(A, d, np.zeros(5, np.uint32), p, "lower"),
                          oracle.syrkd(A, d, p, "lower"))
    # one antidiagonal block [[0, b], [b, 0]] on columns (2, 3): b·(a2·a3ᵀ + a3·a2ᵀ)
    b = 12345
    dz = np.zeros(6, np.uint32)
    e = np.zeros(5, np.uint32)
    e[2] = b
    R = A.astype(object) % p
    want = (b * (np.outer(R[:, 2], R[:, 3]) + np.outer(R[:, 3], R[:, 2]))) % p
    assert oracle.syrkbd(A, dz, e, p, "full").tolist() == want.tolist()


def random_block_diag(k, p, rng):
    """d, e of a symmetric block-diagonal B with every kind of 2×2 block."""
    d = [int(x) for x in rng.integers(0, p, size=k)]
    e = [0] * max(k - 1, 0)
    j = 0
    while j + 1 < k:
        kind = int(rng.integers(0, 5))
        if kind == 0:          # 1×1 block
            j += 1
            continue
        e[j] = int(rng.integers(1, p))
        if kind == 1:          # antidiagonal [[0, β], [β, 0]] (the paper's odd-p case)
            d[j] = d[j + 1] = 0
        elif kind == 2:        # [[0, β], [β, γ]], γ ≠ 0 (the antitriangular form)
            d[j] = 0
            d[j + 1] = int(rng.integers(1, p))
        elif kind == 3:        # [[x, β], [β, 0]]
            d[j + 1] = 0
        j += 2
    return d, e


@pytest.mark.parametrize("p", [3, 5, 7, 13, 97, 40961, 65521, 65537, 131071, 8388593])
def test_block_factor_gives_w_w_t_equal_b(p):
    rng = np.random.default_rng(p % 1009)
    for k in [0, 1, 2, 3, 6, 11, 24]:
        for _ in range(6):
            d, e = random_block_diag(k, p, rng)
            kk, terms = ffsyrk.syrkbd_factor(p, d, e)
            assert kk in (k, k + 1)
            W = [[0] * kk for _ in range(k)]
            for c, ts in enumerate(terms):
                assert len(ts) <= 4
                for src, coef in ts:
                    assert 0 <= src < k and W[src][c] == 0   # merged sources
                    W[src][c] = coef
            for i in range(k):
                for j in range(k):
                    got = sum(W[i][t] * W[j][t] for t in range(kk)) % p
                    want = d[i] if i == j else (e[min(i, j)] if abs(i - j) == 1 else 0)
                    assert got == want % p, (p, d, e, i, j)


def test_block_factor_rejects_overlapping_blocks_and_matches_syrkd():
    p = 65521
    with pytest.raises(ValueError):
        ffsyrk.syrkbd_factor(p, [1, 2, 3, 4], [5, 6, 0])
    # e ≡ 0 mod p closes no block; e = None is Algorithm 5 alone
    d = [3, 0, 17, 5, 65520]
    kk1, t1 = ffsyrk.syrkbd_factor(p, d, [p, 0, 2 * p, 0])
    kk2, t2 = ffsyrk.syrkbd_factor(p, d, None)
    kk3, partner, u, v = ffsyrk.syrkd_factor(p, d)
    assert kk1 == kk2 == kk3 and t1 == t2
    for c in range(kk3):
        want = {}
        if c < len(d) and u[c]:
            want[c] = u[c]
        if partner[c] >= 0 and partner[c] < len(d) and v[c]:
            want[partner[c]] = v[c]
        assert dict(t2[c]) == want
