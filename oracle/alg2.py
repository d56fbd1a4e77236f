"""Algorithm 2 (syrk) of arXiv 2001.04109, step by step -- TEST INFRASTRUCTURE.

Exact arithmetic in Python integers (numpy ``object`` arrays), every value
kept in [0, p).  Written from Section 3 (Algorithm 2, its Require/Ensure
lines and Prop. 3.1) in the paper's notation; it is slow on purpose and only
meant for small blocks.  Two things it makes visible that the tests pin:

* recursive calls return only the lower triangle (the strict upper part is
  zero), which is why Algorithm 2 has to mirror Low(U1) into Up(U1) before
  the full additions U2 = U1 + P4 and U4 = U2 + P3;
* odd dimensions are handled by zero padding, A·Aᵀ = [A 0]·[A 0]ᵀ (Section
  3.1, "Any field with prime characteristic"), and zero rows only add zero
  rows and columns to C.
"""
from __future__ import annotations

import numpy as np

from . import field
from . import winograd as _winograd


def _obj(X) -> np.ndarray:
    return np.array(X, dtype=object)


def low(X) -> np.ndarray:
    """Lower triangle (diagonal included); the strict upper part set to 0."""
    X = _obj(X)
    out = X.copy()
    n = X.shape[0]
    for i in range(n):
        for j in range(i + 1, X.shape[1]):
            out[i, j] = 0
    return out


def up_strict(X) -> np.ndarray:
    X = _obj(X)
    return X - low(X)


def classical_syrk(A, p: int) -> np.ndarray:
    """Low(A·Aᵀ) mod p by the plain definition (the recursion's base case)."""
    A = _obj(A) % p
    return low(A.dot(A.T) % p)


def skew_y(p: int, w: int, layout: str = "interleaved", params: dict | None = None) -> np.ndarray:
    return _obj(field.y_matrix(p, w, layout=layout, params=params))


def pad_to(A, rows: int, cols: int) -> np.ndarray:
    A = _obj(A)
    out = np.zeros((rows, cols), dtype=object)
    out[: A.shape[0], : A.shape[1]] = A
    return out


def step(A, p: int, Y, syrk_rec, mirror: bool = True, gemm=None) -> dict:
    """One level of Algorithm 2 on an even-sized A with a (k/2)×(k/2) Y.

    ``syrk_rec`` computes the three recursive products (lower triangle
    only); ``gemm(X, Z)`` the two general products X·Z (default: the
    classical product).  Returns every intermediate value under the paper's
    names.
    """
    A = _obj(A) % p
    n, k = A.shape
    h, w = n // 2, k // 2
    A11, A12 = A[:h, :w], A[:h, w:]
    A21, A22 = A[h:, :w], A[h:, w:]
    Y = _obj(Y) % p
    # 4 additions and 2 multiplications by Y
    S1 = (A21 - A11).dot(Y) % p
    S2 = (A22 - A21.dot(Y)) % p
    S3 = (S1 - A22) % p
    S4 = (S3 + A12) % p
    # 3 recursive syrk (P1, P2, P5) and 2 general (P3, P4) products
    P1 = syrk_rec(A11)
    P2 = syrk_rec(A12)
    if gemm is None:
        def gemm(X, Z):
            return X.dot(Z) % p
    P3 = _obj(gemm(A22, S4.T)) % p
    P4 = _obj(gemm(S1, S2.T)) % p
    P5 = syrk_rec(S3)
    # 2 symmetric (half) additions
    U1 = (low(P1) + low(P5)) % p
    U3 = (low(P1) + low(P2)) % p
    # mirror, then 2 complete additions
    if mirror:
        U1 = (U1 + up_strict(U1.T)) % p
    U2 = (U1 + P4) % p
    U4 = (U2 + P3) % p
    # 1 half addition: Low(U5) = Low(U2) + Low(P4ᵀ)
    U5 = (low(U2) + low(P4.T)) % p
    C = np.zeros((n, n), dtype=object)
    C[:h, :h] = low(U3)
    C[h:, :h] = U4
    C[h:, h:] = low(U5)
    return dict(S1=S1, S2=S2, S3=S3, S4=S4, P1=P1, P2=P2, P3=P3, P4=P4, P5=P5,
                U1=U1, U2=U2, U3=U3, U4=U4, U5=U5, C=C, Y=Y)


def syrk(A, p: int, levels: int, layout: str = "interleaved", params: dict | None = None,
         mirror: bool = True, winograd: int = 0) -> np.ndarray:
    """Low(A·Aᵀ) mod p by ``levels`` levels of Algorithm 2, then the classical base case.

    Odd sizes are zero padded: rows to an even count, columns to an even
    count (a multiple of 4 when Y has the 2×2 form, whose dimension k/2 must
    be even).  The same Y constants are used at every level.  With
    ``winograd`` > 0 the two general products of a level with ``levels``
    levels to go use min(winograd, levels − 1) levels of Algorithm 1 (the
    paper's G-i variants take levels − 1, Section 4.2).
    """
    A = _obj(A) % p
    n, k = A.shape
    if levels <= 0 or n < 2 or k < 2:
        return classical_syrk(A, p)
    prm = params or field.y_params(p)
    kmul = 4 if prm["form"] == "2x2" else 2
    n2 = n + (n % 2)
    k2 = -(-k // kmul) * kmul
    Ap = pad_to(A, n2, k2)
    Y = skew_y(p, k2 // 2, layout=layout, params=prm)

    def rec(X):
        return syrk(X, p, levels - 1, layout=layout, params=prm, mirror=mirror,
                    winograd=winograd)

    sw = min(max(winograd, 0), levels - 1)

    def gemm(X, Z):
        return _winograd.product(X, Z, p, sw)

    C = step(Ap, p, Y, rec, mirror=mirror, gemm=gemm)["C"]
    return C[:n, :n]


def classical_dc(A, p: int, levels: int) -> np.ndarray:
    """Classical 2×2 divide and conquer (4 recursive syrk + 2 general products).

    C11 = A11A11ᵀ + A12A12ᵀ, C21 = A21A11ᵀ + A22A12ᵀ, C22 = A21A21ᵀ + A22A22ᵀ;
    the "Syrk-i" rows of Table 5 and the classical divide and conquer the
    paper compares against in Section 4.2.
    """
    A = _obj(A) % p
    n, k = A.shape
    if levels <= 0 or n < 2 or k < 2:
        return classical_syrk(A, p)
    n2, k2 = n + n % 2, k + k % 2
    Ap = pad_to(A, n2, k2)
    h, w = n2 // 2, k2 // 2
    A11, A12, A21, A22 = Ap[:h, :w], Ap[:h, w:], Ap[h:, :w], Ap[h:, w:]

    def rec(X):
        return classical_dc(X, p, levels - 1)

    C = np.zeros((n2, n2), dtype=object)
    C[:h, :h] = (rec(A11) + rec(A12)) % p
    C[h:, :h] = (A21.dot(A11.T) + A22.dot(A12.T)) % p
    C[h:, h:] = (rec(A21) + rec(A22)) % p
    return C[:n, :n]
