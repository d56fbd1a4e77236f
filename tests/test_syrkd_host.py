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
