"""The oracle's Hermitian product over F_{p²} (Section 3.2), pinned (CPU only).

F_{p²} = F_p[i]/(i² − r) with r a non-square.  The oracle writes the
conjugate as x − y·i; here conjugation is computed independently as the
Frobenius map x ↦ x^p by repeated multiplication in the field, and C = A·Aᴴ
is summed in Python integers.  Also: C is Hermitian (Re C symmetric, Im C
antisymmetric with a zero diagonal), and for one column the diagonal is the
field norm x·x̄ = a² − r·b² ∈ F_p.
"""
import numpy as np
import pytest

import oracle


def nonsquare(p, which=0):
    ns = [x for x in range(2, p) if pow(x, (p - 1) // 2, p) == p - 1]
    return ns[which % len(ns)]


def fmul(x, y, p, r):
    (a, b), (c, d) = x, y
    return ((a * c + r * b * d) % p, (a * d + b * c) % p)


def frobenius(x, p, r):
    out, base, e = (1, 0), x, p
    while e:
        if e & 1:
            out = fmul(out, base, p, r)
        base = fmul(base, base, p, r)
        e >>= 1
    return out


@pytest.mark.parametrize("p", [3, 7, 11, 13, 65521, 131071])
def test_herk_against_frobenius_conjugate(p):
    rng = np.random.default_rng(p)
    for which in range(2):
        r = nonsquare(p, which * 3)
        for _ in range(3):
            n, k = int(rng.integers(1, 6)), int(rng.integers(1, 6))
            A = rng.integers(0, 1 << 32, size=(n, 2 * k), dtype=np.uint64).astype(np.uint32)
            X = [[(int(A[j, 2 * t]) % p, int(A[j, 2 * t + 1]) % p) for t in range(k)] for j in range(n)]
            Cre, Cim = oracle.herk(A, p, r, "full")
            for j in range(n):
                for l in range(n):
                    s = (0, 0)
                    for t in range(k):
                        term = fmul(X[j][t], frobenius(X[l][t], p, r), p, r)
                        s = ((s[0] + term[0]) % p, (s[1] + term[1]) % p)
                    assert (int(Cre[j, l]), int(Cim[j, l])) == s, (p, r, j, l)


def test_herk_hermitian_and_norm():
    p, r = 65521, nonsquare(65521)
    rng = np.random.default_rng(3)
    A = rng.integers(0, p, size=(9, 14)).astype(np.uint32)
    Cre, Cim = oracle.herk(A, p, r, "full")
    assert np.array_equal(Cre, Cre.T)
    assert np.array_equal((Cim.astype(np.int64) + Cim.T.astype(np.int64)) % p, np.zeros((9, 9)))
    assert np.all(np.diag(Cim) == 0)
    # one column: the diagonal holds the norms a² − r·b²
    A1 = A[:, :2]
    Cre1, Cim1 = oracle.herk(A1, p, r, "lower")
    for j in range(9):
        a, b = int(A1[j, 0]), int(A1[j, 1])
        assert int(Cre1[j, j]) == (a * a - r * b * b) % p and Cim1[j, j] == 0
    # triangles agree with the full product
    lo = oracle.herk(A, p, r, "lower")
    up = oracle.herk(A, p, r, "upper")
    m = np.tril(np.ones((9, 9), bool))
    assert np.array_equal(lo[0][m], Cre[m]) and np.array_equal(lo[1][m], Cim[m])
    assert np.array_equal(up[0][m.T], Cre[m.T]) and np.array_equal(up[1][m.T], Cim[m.T])
