"""Algorithm 1 of arXiv 2001.04109, C = W(A, B) -- TEST INFRASTRUCTURE.

The Winograd variant of Strassen's 2×2 block product (Section 2, Algorithm
1): 8 block pre-additions s1..s4 (rows of A) and t1..t4 (columns of B), 7
block products p1..p7, 7 block post-additions c1..c7, so 15 additions in
all.  Exact arithmetic in Python integers, every value kept in [0, p).  The
paper's fsyrk computes the two general products P3 = A22·S4ᵀ and P4 = S1·S2ᵀ
of Algorithm 2 this way, with one fewer recursive level than the syrk
recursion above them (Section 4.2, the "G1-i"/"G3-i" variants); see
:func:`oracle.alg2.syrk`'s ``winograd`` argument.
"""
from __future__ import annotations

import numpy as np


def _obj(X) -> np.ndarray:
    return np.array(X, dtype=object)


def step(A, B, p: int, mul) -> dict:
    """One level of Algorithm 1 on even-sized A (m×k) and B (k×n).

    ``mul`` computes the 7 block products.  Returns every intermediate value
    under the paper's names and C = [[c3, c7], [c4, c5]].
    """
    A = _obj(A) % p
    B = _obj(B) % p
    m, k = A.shape
    k2, n = B.shape
    assert k == k2 and m % 2 == 0 and k % 2 == 0 and n % 2 == 0
    h, w, v = m // 2, k // 2, n // 2
    a11, a12, a21, a22 = A[:h, :w], A[:h, w:], A[h:, :w], A[h:, w:]
    b11, b12, b21, b22 = B[:w, :v], B[:w, v:], B[w:, :v], B[w:, v:]
    # pre-additions on the rows of A and on the columns of B
    s1 = (a11 - a21) % p
    s2 = (a21 + a22) % p
    s3 = (s2 - a11) % p
    s4 = (a12 - s3) % p
    t1 = (b22 - b12) % p
    t2 = (b12 - b11) % p
    t3 = (b11 + t1) % p
    t4 = (b21 - t3) % p
    # the 7 products
    p1 = mul(a11, b11)
    p2 = mul(a12, b21)
    p3 = mul(a22, t4)
    p4 = mul(s1, t1)
    p5 = mul(s3, t3)
    p6 = mul(s4, b22)
    p7 = mul(s2, t2)
    # post-additions
    c1 = (p1 + p5) % p
    c2 = (c1 + p4) % p
    c3 = (p1 + p2) % p
    c4 = (c2 + p3) % p
    c5 = (c2 + p7) % p
    c6 = (c1 + p7) % p
    c7 = (c6 + p6) % p
    C = np.zeros((m, n), dtype=object)
    C[:h, :v] = c3
    C[:h, v:] = c7
    C[h:, :v] = c4
    C[h:, v:] = c5
    return dict(s1=s1, s2=s2, s3=s3, s4=s4, t1=t1, t2=t2, t3=t3, t4=t4, p1=p1, p2=p2, p3=p3,
                p4=p4, p5=p5, p6=p6, p7=p7, c1=c1, c2=c2, c3=c3, c4=c4, c5=c5, c6=c6, c7=c7, C=C)


def product(A, B, p: int, levels: int) -> np.ndarray:
    """A·B mod p by ``levels`` levels of Algorithm 1, then the classical product.

    Odd dimensions are zero padded to even ones at each level (zero rows of
    A and zero columns of B give zero rows and columns of C; zero columns of
    A against zero rows of B add nothing).
    """
    A = _obj(A) % p
    B = _obj(B) % p
    m, k = A.shape
    n = B.shape[1]
    if levels <= 0 or min(m, k, n) < 2:
        return A.dot(B) % p
    m2, k2, n2 = m + m % 2, k + k % 2, n + n % 2
    Ap = np.zeros((m2, k2), dtype=object)
    Ap[:m, :k] = A
    Bp = np.zeros((k2, n2), dtype=object)
    Bp[:k, :n] = B

    def mul(X, Z):
        return product(X, Z, p, levels - 1)

    return step(Ap, Bp, p, mul)["C"][:m, :n]
